// hot_background.cu -- the analytic cube fields of background subtraction (Warren 2013,
// Sec. "Background Subtraction": the force of the uniform background is removed inside a
// surrounding cube by the analytic field of the cube; outside it, the cubes that are not
// expanded -- leaves taken particle by particle, and empty octants of opened cells -- are
// removed by their analytic fields as well).
//
// Per sink group: every cube of its cube list and its surrounding cube S, each a uniform
// cube of density -rho (rho = M / L^3 over the root cube), evaluated at each sink by the
// closed form of hot_box.cuh and added to the accelerations and potentials that the
// interaction kernel wrote.  In the mixed mode the corners relative to the sink are
// formed in float64 and the closed form runs in float32; the cubes are near the group
// (they failed the acceptance test, or surround it), so the eight corner terms cancel
// mildly.
#include "hot_common.cuh"

__device__ __forceinline__ float hb_log(float v) { return logf(v); }
__device__ __forceinline__ double hb_log(double v) { return log(v); }
__device__ __forceinline__ float hb_atan(float v) { return atanf(v); }
__device__ __forceinline__ double hb_atan(double v) { return atan(v); }
__device__ __forceinline__ float hb_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double hb_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float hb_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double hb_div(double a, double b) { return a / b; }

#include "hot_box.cuh"

namespace {

constexpr int BW = 4;  // warps per block

template <class T>
__global__ void __launch_bounds__(BW * 32) k_bg_box(
    int64_t ngroup, const int32_t *__restrict__ gcell, const int32_t *__restrict__ cbegin,
    const int32_t *__restrict__ ccount, const double *__restrict__ spos, const uint32_t *__restrict__ perm,
    const int64_t *__restrict__ off_box, const int32_t *__restrict__ l_box, const int32_t *__restrict__ gS,
    const double *__restrict__ cen, const double *__restrict__ half, const double *__restrict__ rho_p, double G,
    unsigned *__restrict__ work, double *__restrict__ acc, double *__restrict__ pot)
{
    const unsigned lane = lane_id();
    const T Grho = (T)(-G * *rho_p);
    for (;;) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(work, 1u);
        const int64_t g = __shfl_sync(0xffffffffu, g0, 0);
        if (g >= ngroup) break;
        const int32_t gc = gcell[g];
        const int64_t b0 = cbegin[gc], n = ccount[gc];
        const int64_t e0 = off_box[g], ne = off_box[g + 1] - e0;
        for (int64_t s0 = 0; s0 < n; s0 += 32) {
            const int64_t s = b0 + s0 + lane;
            if (s0 + lane >= n) continue;
            const double px = spos[3 * s + 0], py = spos[3 * s + 1], pz = spos[3 * s + 2];
            T ax = T(0), ay = T(0), az = T(0), ph = T(0);
            for (int64_t k = 0; k <= ne; ++k) {
                const int64_t q = k < ne ? (int64_t)l_box[e0 + k] : (int64_t)gS[g];
                const double h = half[q];
                const T lo[3] = {(T)((cen[3 * q + 0] - h) - px), (T)((cen[3 * q + 1] - h) - py),
                                 (T)((cen[3 * q + 2] - h) - pz)};
                const T hi[3] = {(T)((cen[3 * q + 0] + h) - px), (T)((cen[3 * q + 1] + h) - py),
                                 (T)((cen[3 * q + 2] + h) - pz)};
                box_field<T>(T(0), T(0), T(0), lo, hi, Grho, ax, ay, az, ph);
            }
            const int64_t i = perm[s];
            acc[3 * i + 0] += (double)ax;
            acc[3 * i + 1] += (double)ay;
            acc[3 * i + 2] += (double)az;
            if (pot) pot[i] += (double)ph;
        }
    }
}

}  // namespace

int hot_impl_bg_box(hot_ctx *c, double *acc, double *pot)
{
    cudaStream_t s = c->st;
    unsigned *work = (unsigned *)(c->sizes.p + 48);
    HOT_CK(cudaMemsetAsync(work, 0, sizeof(unsigned), s));
    HOT_COUNT_LAUNCH();
    if (c->prm.precision == HOT_FP64)
        k_bg_box<double><<<c->nsm * 8, BW * 32, 0, s>>>(c->ngroup, c->gcell.p, c->cbegin.p, c->ccount.p, c->spos.p,
                                                        c->idx.p, c->off_box.p, c->l_box.p, c->bg_gS.p, c->bg_cen.p,
                                                        c->bg_half.p, c->bg_rho.p, c->prm.G, work, acc, pot);
    else
        k_bg_box<float><<<c->nsm * 8, BW * 32, 0, s>>>(c->ngroup, c->gcell.p, c->cbegin.p, c->ccount.p, c->spos.p,
                                                       c->idx.p, c->off_box.p, c->l_box.p, c->bg_gS.p, c->bg_cen.p,
                                                       c->bg_half.p, c->bg_rho.p, c->prm.G, work, acc, pot);
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}
