// hot_interact.cu -- M2P and P2P interactions of every sink group with its lists
// (Warren 2013, Sec. "Improving instruction-level parallelism": an m x n block of m
// source cells and n sink particles; the source data is reorganised once per block
// and shared by the n sinks).
//
// One warp per sink group (dynamic work counter).  The group's sinks map to lanes; when
// a group has fewer than 32 sinks, each sink gets floor(32/n) lanes that split the
// source lists and are combined at the end.  Source cell records and source particles
// are staged in shared memory per chunk and read as warp-wide broadcasts.
//
// Mixed precision (T = float): all interaction arithmetic in float32 on coordinates
// relative to the group centre g.  float64 is used only for the absolute positions and
// the offsets z_c - g and x_i - g (rounded to float32 afterwards).  Each lane sums a
// chunk in plain float32 and adds the chunk total into a compensated (Kahan) pair; the
// pairs are combined in float64.  T = double runs the same code in float64.
#include "hot_common.cuh"
#include "generated.cuh"

namespace {

constexpr int IW = 4;   // warps per block
constexpr int SRC = 64; // staged source particles per P2P chunk

template <int P>
struct ChunkCells {
    static constexpr int value = P <= 4 ? 32 : 16;
};

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v)
{
    float y = __fsub_rn(v, comp);
    float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}
__device__ __forceinline__ void kahan_add(double &sum, double &comp, double v) { sum += v; }

template <int P, class T>
struct Smem {
    static constexpr int CH = ChunkCells<P>::value;
    static constexpr int RL = HOT_REC_LEN[P];
    T rec[CH][RL];
    T off[CH][4];
    T src[SRC][4];
    int32_t sidx[SRC];
    double red[32][4];
};

template <int P, class T>
__global__ void __launch_bounds__(IW * 32) k_interact(
    int64_t ngroup, const int32_t *__restrict__ gcell, const double *__restrict__ gcen,
    const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount, const double *__restrict__ spos,
    const double *__restrict__ smass, const float4 *__restrict__ prel, const double *__restrict__ ccom,
    const T *__restrict__ rec, const int64_t *__restrict__ off_m2p, const int32_t *__restrict__ l_m2p,
    const int64_t *__restrict__ off_p2p, const int32_t *__restrict__ l_p2p, const uint32_t *__restrict__ perm,
    T eps2, double G, unsigned *__restrict__ work, double *__restrict__ acc_out, double *__restrict__ pot_out)
{
    using S = Smem<P, T>;
    constexpr int CH = S::CH;
    constexpr int RL = S::RL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = reinterpret_cast<S *>(smem_raw)[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const T Gt = (T)G;

    for (;;) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(work, 1u);
        const int64_t g = __shfl_sync(0xffffffffu, g0, 0);
        if (g >= ngroup) break;
        const int32_t gc = gcell[g];
        const int64_t gb = cbegin[gc];
        const int n = ccount[gc];
        const double gx = gcen[3 * g + 0], gy = gcen[3 * g + 1], gz = gcen[3 * g + 2];
        const int64_t m0 = off_m2p[g], m1 = off_m2p[g + 1];
        const int64_t p0 = off_p2p[g], p1 = off_p2p[g + 1];

        for (int s0 = 0; s0 < n; s0 += 32) {
            const int ns = n - s0 < 32 ? n - s0 : 32;
            const int nsplit = 32 / ns;
            const int si = (int)lane % ns;
            const int sj = (int)lane / ns;
            const bool active = sj < nsplit;
            const int64_t s = gb + s0 + si;
            const T xi = (T)(spos[3 * s + 0] - gx);
            const T yi = (T)(spos[3 * s + 1] - gy);
            const T zi = (T)(spos[3 * s + 2] - gz);
            T sum[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};

            // ---- M2P over the cell list ----
            for (int64_t e0 = m0; e0 < m1; e0 += CH) {
                const int ne = (int)(m1 - e0 < CH ? m1 - e0 : CH);
                for (int k = 0; k < ne; ++k) {
                    const int32_t cell = l_m2p[e0 + k];
                    const T *src = rec + (int64_t)cell * RL;
                    for (int q = lane; q < RL; q += 32) sm.rec[k][q] = src[q];
                }
                if ((int)lane < ne) {
                    const int32_t cell = l_m2p[e0 + lane];
                    sm.off[lane][0] = (T)(ccom[3 * (int64_t)cell + 0] - gx);
                    sm.off[lane][1] = (T)(ccom[3 * (int64_t)cell + 1] - gy);
                    sm.off[lane][2] = (T)(ccom[3 * (int64_t)cell + 2] - gz);
                }
                __syncwarp();
                if (active) {
                    T ph = 0, ax = 0, ay = 0, az = 0;
                    for (int k = sj; k < ne; k += nsplit)
                        m2p_eval<P, T>(&sm.rec[k][0], xi - sm.off[k][0], yi - sm.off[k][1], zi - sm.off[k][2], ph,
                                       ax, ay, az);
                    kahan_add(sum[0], cmp[0], ax);
                    kahan_add(sum[1], cmp[1], ay);
                    kahan_add(sum[2], cmp[2], az);
                    kahan_add(sum[3], cmp[3], ph);
                }
                __syncwarp();
            }

            // ---- P2P over the leaf list ----
            int fill = 0;
            auto flush = [&]() {
                __syncwarp();
                if (active) {
                    T ph = 0, ax = 0, ay = 0, az = 0;
                    for (int k = sj; k < fill; k += nsplit) {
                        const T dx = sm.src[k][0] - xi, dy = sm.src[k][1] - yi, dz = sm.src[k][2] - zi;
                        const T r2 = dx * dx + dy * dy + dz * dz + eps2;
                        const bool ok = (r2 > T(0)) && (sm.sidx[k] != (int32_t)s);
                        const T rinv = ok ? hot_rsqrt(r2) : T(0);
                        const T mr = sm.src[k][3] * rinv;
                        const T mr3 = mr * rinv * rinv;
                        ax += mr3 * dx;
                        ay += mr3 * dy;
                        az += mr3 * dz;
                        ph -= mr;
                    }
                    kahan_add(sum[0], cmp[0], Gt * ax);
                    kahan_add(sum[1], cmp[1], Gt * ay);
                    kahan_add(sum[2], cmp[2], Gt * az);
                    kahan_add(sum[3], cmp[3], Gt * ph);
                }
                __syncwarp();
                fill = 0;
            };
            for (int64_t e = p0; e < p1; ++e) {
                const int32_t leaf = l_p2p[e];
                const int64_t lb = cbegin[leaf];
                const int lc = ccount[leaf];
                const double ox = ccom[3 * (int64_t)leaf + 0] - gx;
                const double oy = ccom[3 * (int64_t)leaf + 1] - gy;
                const double oz = ccom[3 * (int64_t)leaf + 2] - gz;
                for (int q0 = 0; q0 < lc; q0 += 32) {
                    const int take = lc - q0 < 32 ? lc - q0 : 32;
                    if (fill + take > SRC) flush();
                    if ((int)lane < take) {
                        const int64_t j = lb + q0 + lane;
                        if constexpr (sizeof(T) == 4) {
                            const float4 v = prel[j];
                            sm.src[fill + lane][0] = v.x + (float)ox;
                            sm.src[fill + lane][1] = v.y + (float)oy;
                            sm.src[fill + lane][2] = v.z + (float)oz;
                            sm.src[fill + lane][3] = v.w;
                        } else {
                            sm.src[fill + lane][0] = (T)(spos[3 * j + 0] - gx);
                            sm.src[fill + lane][1] = (T)(spos[3 * j + 1] - gy);
                            sm.src[fill + lane][2] = (T)(spos[3 * j + 2] - gz);
                            sm.src[fill + lane][3] = (T)smass[j];
                        }
                        sm.sidx[fill + lane] = (int32_t)j;
                    }
                    fill += take;
                }
            }
            if (fill > 0) flush();

            // ---- combine the source splits of each sink in float64, write original order ----
            __syncwarp();
            if (active) {
#pragma unroll
                for (int d = 0; d < 4; ++d) sm.red[lane][d] = (double)sum[d] - (double)cmp[d];
            }
            __syncwarp();
            if (active && sj == 0) {
                double t[4] = {0, 0, 0, 0};
                for (int j = 0; j < nsplit; ++j)
#pragma unroll
                    for (int d = 0; d < 4; ++d) t[d] += sm.red[si + j * ns][d];
                const int64_t i = perm[s];
                acc_out[3 * i + 0] = t[0];
                acc_out[3 * i + 1] = t[1];
                acc_out[3 * i + 2] = t[2];
                if (pot_out) pot_out[i] = t[3];
            }
            __syncwarp();
        }
    }
}

template <int P, class T>
int forces_pt(hot_ctx *c, double *acc, double *pot)
{
    cudaStream_t s = c->st;
    const size_t smem = sizeof(Smem<P, T>) * IW;
    auto kern = k_interact<P, T>;
    HOT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned *work = (unsigned *)(c->sizes.p + 56);
    HOT_CK(cudaMemsetAsync(work, 0, sizeof(int64_t), s));
    const T *rec = nullptr;
    if constexpr (sizeof(T) == 4)
        rec = c->rec32.p;
    else
        rec = c->rec64.p;
    int occ = 0;
    HOT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, IW * 32, smem));
    if (occ < 1) occ = 1;
    const int blocks = c->nsm * occ;
    const T eps2 = (T)(c->prm.eps * c->prm.eps);
    HOT_COUNT_LAUNCH();
    kern<<<blocks, IW * 32, smem, s>>>(c->ngroup, c->gcell.p, c->gcen.p, c->cbegin.p, c->ccount.p, c->spos.p,
                                       c->smass.p, c->prel.p, c->ccom.p, rec, c->off_m2p.p, c->l_m2p.p, c->off_p2p.p,
                                       c->l_p2p.p, c->idx.p, eps2, c->prm.G, work, acc, pot);
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}

template <int P>
int forces_p(hot_ctx *c, double *acc, double *pot)
{
    if (c->prm.precision == HOT_FP64) return forces_pt<P, double>(c, acc, pot);
    return forces_pt<P, float>(c, acc, pot);
}

}  // namespace

int hot_impl_forces(hot_ctx *c, double *acc, double *pot)
{
    hot_tic(c, 4);
    int r;
    switch (c->p_mom) {
        case 0: r = forces_p<0>(c, acc, pot); break;
        case 1: r = forces_p<1>(c, acc, pot); break;
        case 2: r = forces_p<2>(c, acc, pot); break;
        case 3: r = forces_p<3>(c, acc, pot); break;
        case 4: r = forces_p<4>(c, acc, pot); break;
        case 5: r = forces_p<5>(c, acc, pot); break;
        case 6: r = forces_p<6>(c, acc, pot); break;
        default: return HOT_ESTATE;
    }
    hot_toc(c, 4);
    return r;
}

int hot_impl_adjoint(hot_ctx *, const double *, const double *, double *, double *) { return HOT_ESTATE; }
