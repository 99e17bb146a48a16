// hot_interact.cuh -- M2P and P2P interactions of every sink group with its lists
// (Warren 2013, Sec. "Improving instruction-level parallelism": an m x n block of m
// source cells and n sink particles; the source data is reorganised once per block
// and shared by the n sinks).
//
// One warp per work item, a slice of 32 sinks of one group (dynamic work counter over
// the items, which come in descending order of their cost), one sink per lane; when a
// slice has fewer than 32 sinks, each sink gets several lanes that split the source
// lists (combined at the end in float64).  Taking slices rather than whole groups as
// items keeps one large group from being a single warp's work at the end of the launch.
//
// Cell records (the traced coefficients of every accepted cell) are staged per warp in
// shared memory by TMA bulk copies (cp.async.bulk, completion on an mbarrier), double
// buffered: the copies of chunk c+1 are in flight while chunk c is evaluated.  Every
// wait on an mbarrier is bounded; an expired wait sets the status word and the warp
// stops.  Source particles of the P2P list are staged by the lanes.
//
// Mixed precision (T = float): interaction arithmetic in float32 on coordinates relative
// to the group centre g; float64 only for the absolute positions and the offsets z_c - g
// and x_i - g (rounded to float32 afterwards).  Each lane sums a chunk in plain float32
// and adds the chunk total into a compensated (Kahan) pair; pairs are combined in
// float64.  T = double runs the same code in float64.
#pragma once

#include <type_traits>

#include "hot_common.cuh"
#include "generated.cuh"

namespace {

constexpr int IW = 4;    // warps per block
constexpr int SRC = 64;  // staged source particles per P2P chunk
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // try_wait polls before a wait is declared expired

template <int P, class T>
struct Cfg {
    static constexpr int RL = HOT_REC_LEN[P];
    // shared-memory stride of a staged record: 16 bytes of padding, so that lanes reading
    // different records at the same offset hit different banks
    static constexpr int RLS = RL + 16 / (int)sizeof(T);
    // records per staged chunk: 16 up to p = 4 (56-float records; 4.6% faster than 8 at
    // 2^20), 8 above (at p = 6, 16 costs occupancy: 13% slower); 4 in float64
    static constexpr int CH = sizeof(T) == 4 ? (P <= 4 ? 16 : 8) : 4;
};

template <int P, class T>
struct alignas(16) Smem {
    static constexpr int RLS = Cfg<P, T>::RLS;
    static constexpr int CH = Cfg<P, T>::CH;
    T rec[2][CH][RLS];
    T off[2][CH][4];
    T src[SRC][4];
    double red[32][4];
    int32_t sidx[SRC];
    int32_t lex[33], lbeg[32];  // P2P batch: scanned particle offsets and first slots
    T loff[32][3];              // P2P batch: leaf centre offsets
    unsigned long long bar[2];
    unsigned long long probe;   // test setting: a barrier nothing ever arrives on
    unsigned char qo[2][CH];    // order (per-interaction order selection) or periodic image of each staged record
};

// Records of every order (per-interaction order selection): base pointer and length.
template <class T>
struct RecTab {
    const T *rec[HOT_ORDERS];
    int rl[HOT_ORDERS];
};

// The order-q expansion, q <= Q chosen at run time (uniform over the warp except when a
// slice's lanes split the list).
// (R scaled by the record's inv_s, as m2p_eval_s takes it.)
template <int Q, class T>
__device__ __forceinline__ void m2p_eval_order(int q, const T *r, T rx, T ry, T rz, T &ph, T &ax, T &ay, T &az)
{
    if constexpr (Q == 0) {
        m2p_eval_s<0, T>(r, rx, ry, rz, ph, ax, ay, az);
    } else {
        if (q == Q)
            m2p_eval_s<Q, T>(r, rx, ry, rz, ph, ax, ay, az);
        else
            m2p_eval_order<Q - 1, T>(q, r, rx, ry, rz, ph, ax, ay, az);
    }
}

// ---- TMA bulk copy and mbarrier helpers (inline PTX) ----
__device__ __forceinline__ uint32_t sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sptr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sptr(dst)),
        "l"(src), "r"(bytes), "r"(sptr(bar))
        : "memory");
}

// Warp-collective bounded wait: every lane polls until it has observed the phase
// completion itself; the result is the same on all lanes.  Polls use try_wait (which
// may suspend the thread for a while); a limit below the default (a test setting) polls
// with the non-blocking test_wait, so that the limit counts polls of no duration.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t phase, uint32_t limit = WAIT_LIMIT)
{
    uint32_t done = 0;
    const bool quick = limit < WAIT_LIMIT;
    for (uint32_t i = 0; i < limit; ++i) {
        if (!done) {
            if (quick)
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(done)
                    : "r"(sptr(bar)), "r"(phase)
                    : "memory");
            else
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(done)
                    : "r"(sptr(bar)), "r"(phase)
                    : "memory");
        }
        if (__all_sync(0xffffffffu, done)) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v)
{
    float y = __fsub_rn(v, comp);
    float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}
__device__ __forceinline__ void kahan_add(double &sum, double &comp, double v) { sum += v; }

template <class T>
struct Acc {
    T s[4], c[4];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int d = 0; d < 4; ++d) s[d] = c[d] = T(0);
    }
    __device__ __forceinline__ void add(T ax, T ay, T az, T ph)
    {
        kahan_add(s[0], c[0], ax);
        kahan_add(s[1], c[1], ay);
        kahan_add(s[2], c[2], az);
        kahan_add(s[3], c[3], ph);
    }
    __device__ __forceinline__ double get(int d) const { return (double)s[d] - (double)c[d]; }
};

// float32: the running sums and their compensations in pairs, (a_x, a_y) and (a_z, phi), so
// that each step of the compensated sum is one paired instruction for two components; the
// same round-to-nearest operations as kahan_add, a difference x - y taken as x + (-y)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
template <>
struct Acc<float> {
    float2 s01, s23, c01, c23;
    __device__ __forceinline__ void zero() { s01 = s23 = c01 = c23 = make_float2(0.f, 0.f); }
    __device__ __forceinline__ static void kahan2(float2 &s, float2 &c, float2 v)
    {
        const float2 y = __fadd2_rn(v, neg2(c));
        const float2 t = __fadd2_rn(s, y);
        c = __fadd2_rn(__fadd2_rn(t, neg2(s)), neg2(y));
        s = t;
    }
    __device__ __forceinline__ void add(float ax, float ay, float az, float ph)
    {
        kahan2(s01, c01, make_float2(ax, ay));
        kahan2(s23, c23, make_float2(az, ph));
    }
    __device__ __forceinline__ double get(int d) const
    {
        const float sv = d == 0 ? s01.x : d == 1 ? s01.y : d == 2 ? s23.x : s23.y;
        const float cv = d == 0 ? c01.x : d == 1 ? c01.y : d == 2 ? c23.x : c23.y;
        return (double)sv - (double)cv;
    }
};

template <class T>
struct Group {
    int64_t gb;      // first sorted slot of the group's sinks
    int n;           // sinks
    double gx, gy, gz;
    T ghi[3], glo[3];  // group centre as a T pair (hi = rounded, lo = remainder)
    int64_t m0, m1;  // M2P list range
    int64_t p0, p1;  // P2P list range
    int32_t own0, own1;  // pre-order range of the group's cell: its own leaves
    double pL;           // periodic boundaries: side of the cube (0: open)
    int pws;             // periodic boundaries: images within pws cubes on every side
};

// Periodic boundaries: the shift n L of image img (index ((nx + ws) w + ny + ws) w + nz + ws,
// w = 2 ws + 1), the sources of the image being the central ones moved by n L.
template <class T>
__device__ __forceinline__ void image_shift(const Group<T> &G, unsigned img, T &sx, T &sy, T &sz)
{
    const int w = 2 * G.pws + 1;
    sx = (T)((double)((int)(img / (unsigned)(w * w)) - G.pws) * G.pL);
    sy = (T)((double)((int)((img / (unsigned)w) % (unsigned)w) - G.pws) * G.pL);
    sz = (T)((double)((int)(img % (unsigned)w) - G.pws) * G.pL);
}
// Bit of a staged leaf's first slot marking a leaf of a non-central image (slots are below 2^30).
constexpr int32_t IMG_LEAF = 0x40000000;

// Offset z_c - g in T from the hi/lo pairs of the cell (record header slots 2..7) and of
// the group centre: (z_hi - g_hi) + (z_lo - g_lo).
template <class T>
__device__ __forceinline__ void centre_offset(const T *h, const Group<T> &G, T &ox, T &oy, T &oz)
{
    ox = (h[2] - G.ghi[0]) + (h[5] - G.glo[0]);
    oy = (h[3] - G.ghi[1]) + (h[6] - G.glo[1]);
    oz = (h[4] - G.ghi[2]) + (h[7] - G.glo[2]);
}

// M2P over the group's cell list for NS sink positions per lane.  Lane (sink, split sj)
// evaluates cells sj, sj + nsplit, ... of every staged chunk.  Cell indices are loaded
// one chunk ahead of the copies, which run one chunk ahead of the arithmetic.  Returns
// false when a bounded wait expired (status flagged, the warp must stop).
template <int P, class T, int NS, int MODE, bool VQ>
__device__ __forceinline__ bool m2p_list(Smem<P, T> &sm, const Group<T> &G, const int32_t *__restrict__ l_m2p,
                                         const T *__restrict__ rec, const RecTab<T> &rq, const T (&x)[NS][3],
                                         const T (&wt)[NS][4],
                                         int sj, int nsplit, bool active, Acc<T> (&acc)[NS], uint32_t (&phase)[2],
                                         uint32_t wait_limit, bool probe, unsigned *status)
{
    constexpr int CH = Cfg<P, T>::CH;
    constexpr int RL = Cfg<P, T>::RL;
    constexpr uint32_t RB = RL * sizeof(T);
    const unsigned lane = lane_id();
    const int64_t nm = G.m1 - G.m0;
    const int nch = (int)((nm + CH - 1) / CH);
    if (nch == 0) return true;
    if (probe) {
        // test setting: a wait that cannot complete, taken before any copy is issued (so
        // nothing is in flight when it runs out); at most 4096 polls
        if (!mbar_wait(&sm.probe, 0, wait_limit < 4096u ? wait_limit : 4096u)) {
            if (lane == 0) hot_flag(status, HOT_ST_TIMEOUT);
            return false;
        }
    }
    auto chunk_n = [&](int c) { return (int)(nm - (int64_t)c * CH < CH ? nm - (int64_t)c * CH : CH); };
    auto load_idx = [&](int c) {
        return (c < nch && (int)lane < chunk_n(c)) ? l_m2p[G.m0 + (int64_t)c * CH + lane] : 0;
    };
    auto issue = [&](int c, int b, int32_t cell) {
        const int ne = chunk_n(c);
        if constexpr (VQ) {
            // an entry is cell | order << HOT_ORDER_SHIFT; records of each order have their own length
            const uint32_t q = (uint32_t)cell >> HOT_ORDER_SHIFT;
            const int64_t ci = (int64_t)((uint32_t)cell & HOT_CELL_MASK);
            const uint32_t bytes = (int)lane < ne ? (uint32_t)rq.rl[q] * (uint32_t)sizeof(T) : 0u;
            const uint32_t tot = __reduce_add_sync(0xffffffffu, bytes);
            if (lane == 0) mbar_expect_tx(&sm.bar[b], tot);
            __syncwarp();
            if ((int)lane < ne) {
                sm.qo[b][lane] = (unsigned char)q;
                fence_async_smem();
                bulk_g2s(&sm.rec[b][lane][0], rq.rec[q] + ci * rq.rl[q], bytes, &sm.bar[b]);
            }
        } else {
            // periodic boundaries: an entry is cell | image << HOT_IMG_SHIFT
            const bool per = G.pws > 0;
            const uint32_t ci = per ? ((uint32_t)cell & HOT_IMG_CELL_MASK) : (uint32_t)cell;
            if (lane == 0) mbar_expect_tx(&sm.bar[b], (uint32_t)ne * RB);
            __syncwarp();
            if ((int)lane < ne) {
                if (per) sm.qo[b][lane] = (unsigned char)((uint32_t)cell >> HOT_IMG_SHIFT);
                fence_async_smem();
                bulk_g2s(&sm.rec[b][lane][0], rec + (int64_t)ci * RL, RB, &sm.bar[b]);
            }
        }
    };

    issue(0, 0, load_idx(0));
    int32_t nxt = load_idx(1);
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        if (c + 1 < nch) {
            issue(c + 1, b ^ 1, nxt);
            nxt = load_idx(c + 2);
        }
        if (!mbar_wait(&sm.bar[b], phase[b], wait_limit)) {
            // the wait ran out: flag it, let the copies in flight land (default limit) and
            // leave the group
            if (lane == 0) hot_flag(status, HOT_ST_TIMEOUT);
            mbar_wait(&sm.bar[b], phase[b]);
            if (c + 1 < nch) mbar_wait(&sm.bar[b ^ 1], phase[b ^ 1]);
            return false;
        }
        phase[b] ^= 1;
        const int ne = chunk_n(c);
        if ((int)lane < ne) {
            T ox, oy, oz;
            centre_offset(&sm.rec[b][lane][0], G, ox, oy, oz);
            if (!VQ && G.pws > 0) {
                T sx, sy, sz;
                image_shift(G, sm.qo[b][lane], sx, sy, sz);
                ox += sx;
                oy += sy;
                oz += sz;
            }
            // forces: the offset scaled by the record's inv_s (a power of two), negated, with
            // inv_s beside it, so that each evaluation forms (x - o) inv_s = fma(x, inv_s,
            // -o inv_s) exactly; the adjoint's tangent routine takes the offset as it is
            T is = T(1);
            if constexpr (MODE == 0) {
                is = sm.rec[b][lane][0];
                ox = -ox * is;
                oy = -oy * is;
                oz = -oz * is;
            }
            if constexpr (sizeof(T) == 4) {
                *reinterpret_cast<float4 *>(&sm.off[b][lane][0]) = make_float4(ox, oy, oz, is);
            } else {
                sm.off[b][lane][0] = ox;
                sm.off[b][lane][1] = oy;
                sm.off[b][lane][2] = oz;
                sm.off[b][lane][3] = is;
            }
        }
        __syncwarp();
        if (active) {
            T ph[NS], ax[NS], ay[NS], az[NS], dx[NS], dy[NS], dz[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) ph[s] = ax[s] = ay[s] = az[s] = dx[s] = dy[s] = dz[s] = T(0);
            for (int k = sj; k < ne; k += nsplit) {
                const T *r = &sm.rec[b][k][0];
                const T ox = sm.off[b][k][0], oy = sm.off[b][k][1], oz = sm.off[b][k][2], is = sm.off[b][k][3];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    if constexpr (VQ)
                        m2p_eval_order<P, T>(sm.qo[b][k], r, fma(x[s][0], is, ox), fma(x[s][1], is, oy),
                                             fma(x[s][2], is, oz), ph[s], ax[s], ay[s], az[s]);
                    else if constexpr (MODE == 0)
                        m2p_eval_s<P, T>(r, fma(x[s][0], is, ox), fma(x[s][1], is, oy), fma(x[s][2], is, oz), ph[s],
                                         ax[s], ay[s], az[s]);
                    else
                        m2p_tangent<P, T>(r, x[s][0] - ox, x[s][1] - oy, x[s][2] - oz, wt[s][0], wt[s][1], wt[s][2],
                                          ph[s], ax[s], ay[s], az[s], dx[s], dy[s], dz[s]);
                }
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if constexpr (MODE == 0)
                    acc[s].add(ax[s], ay[s], az[s], ph[s]);
                else  // d/dx_i (u.a + v phi) over these cells = (da/dR) u - v a
                    acc[s].add(dx[s] - wt[s][3] * ax[s], dy[s] - wt[s][3] * ay[s], dz[s] - wt[s][3] * az[s], T(0));
            }
        }
        __syncwarp();
    }
    return true;
}

// P2P over the group's leaf list.  Leaf metadata (first slot, count, centre offset) is
// fetched 32 entries at a time, one entry per lane, and broadcast by shuffles; source
// particles are staged SRC at a time with positions relative to g (float32: the
// leaf-relative copy plus the leaf offset).
template <int P, class T, int NS, int MODE, int SOFT>
__device__ __forceinline__ void p2p_list(Smem<P, T> &sm, const Group<T> &G, const int32_t *__restrict__ l_p2p,
                                         const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount,
                                         const T *__restrict__ rec, const float4 *__restrict__ prel,
                                         const double *__restrict__ spos, const double *__restrict__ smass,
                                         const T (&x)[NS][3], const T (&wt)[NS][4], const int32_t (&self)[NS],
                                         int sj, int nsplit, bool active, T eps2, T Gt, Acc<T> (&acc)[NS])
{
    constexpr int RL = Cfg<P, T>::RL;
    // float32 with Plummer smoothing (forces and the adjoint's tangent): the sources of a
    // batch without self or zero-distance pairs are evaluated two per instruction (paired
    // float32 arithmetic), from a staging layout in which one 16-byte load holds the x and y
    // of two sources and the next their z and masses
    constexpr bool PAIRED = sizeof(T) == 4 && SOFT == HOT_SOFT_PLUMMER;
    const unsigned lane = lane_id();
    int fill = 0;
    SoftConst<T> kc{};
    if constexpr (SOFT != HOT_SOFT_PLUMMER) kc = soft_const(eps2);
    // A sink can meet itself, or a source at zero separation, only in a batch holding one
    // of the group's own leaves or when eps = 0; other batches take the loop without the
    // per-pair tests.
    auto flush = [&](bool checked) {
        __syncwarp();
        if (active) {
            T ph[NS], ax[NS], ay[NS], az[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) ph[s] = ax[s] = ay[s] = az[s] = T(0);
            // adjoint: the sink's u is the same for all its sources, so sum_j m/s^3 u is
            // carried as u sum_j m/s^3 (ph holds that sum in this mode)
            auto sweep = [&](auto ck) {
                constexpr bool CK = decltype(ck)::value;
#pragma unroll 2
            for (int k = sj; k < fill; k += nsplit) {
                const T sx = sm.src[k][0], sy = sm.src[k][1], sz = sm.src[k][2], m = sm.src[k][3];
                const int32_t id = CK ? sm.sidx[k] : 0;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const T dx = sx - x[s][0], dy = sy - x[s][1], dz = sz - x[s][2];
                    if constexpr (SOFT != HOT_SOFT_PLUMMER) {
                        // K1: eps2 is the support squared, not added to the separation
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        T f, f2, psi;
                        compact_pair<SOFT>(r2, kc, f, f2, psi);
                        if constexpr (CK) {
                            const bool ok = (r2 > T(0) || kc.e2 > T(0)) && (id != self[s]);
                            f = ok ? f : T(0);
                            f2 = ok ? f2 : T(0);
                            psi = ok ? psi : T(0);
                        }
                        const T mf = m * f;
                        if constexpr (MODE == 0) {
                            ax[s] += mf * dx;
                            ay[s] += mf * dy;
                            az[s] += mf * dz;
                            ph[s] -= m * psi;
                        } else {
                            // the pair term with the tidal tensor f I + f2 d d^T (Plummer below)
                            const T du = dx * wt[s][0] + dy * wt[s][1] + dz * wt[s][2];
                            const T cc = mf * wt[s][3] + m * f2 * du;
                            ph[s] += mf;
                            ax[s] += cc * dx;
                            ay[s] += cc * dy;
                            az[s] += cc * dz;
                        }
                    } else {
                    // from eps^2 up: three fused multiply-adds
                    const T r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
                    T rinv;
                    if constexpr (CK) {
                        const bool ok = (r2 > T(0)) && (id != self[s]);
                        rinv = ok ? hot_rsqrt(r2) : T(0);
                    } else {
                        rinv = hot_rsqrt(r2);
                    }
                    const T mr = m * rinv;
                    const T mr3 = mr * rinv * rinv;
                    if constexpr (MODE == 0) {
                        ax[s] += mr3 * dx;
                        ay[s] += mr3 * dy;
                        az[s] += mr3 * dz;
                        ph[s] -= mr;
                    } else {
                        // d/dx_i (u.a_i + v phi_i) = -G m [u/s^3 - 3 d (d.u)/s^5 + v d/s^3], d = x_j - x_i
                        //   = -G [u sum_j m/s^3 + sum_j (v m/s^3 - 3 m (d.u)/s^5) d]
                        const T du = dx * wt[s][0] + dy * wt[s][1] + dz * wt[s][2];
                        const T cc = mr3 * wt[s][3] - T(3) * mr3 * rinv * rinv * du;
                        ph[s] += mr3;
                        ax[s] += cc * dx;
                        ay[s] += cc * dy;
                        az[s] += cc * dz;
                    }
                    }
                }
            }
            };
            if constexpr (PAIRED) {
                if (!checked) {
                    // pairs of sources (2j, 2j + 1); an odd batch ends with a massless source
                    const int npair = (fill + 1) >> 1;
                    const float4 *s2 = reinterpret_cast<const float4 *>(&sm.src[0][0]);
                    const float2 e22 = make_float2(eps2, eps2), neg1 = make_float2(-1.f, -1.f);
                    float2 nx[NS][3], ax2[NS], ay2[NS], az2[NS], ph2[NS], w2[NS][4];
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) nx[s][d] = make_float2(-x[s][d], -x[s][d]);
#pragma unroll
                        for (int d = 0; d < 4; ++d) w2[s][d] = make_float2(wt[s][d], wt[s][d]);
                        ax2[s] = ay2[s] = az2[s] = ph2[s] = make_float2(0.f, 0.f);
                    }
                    const float2 neg3 = make_float2(-3.f, -3.f);
#pragma unroll 2
                    for (int j = sj; j < npair; j += nsplit) {
                        const float4 a = s2[2 * j], b = s2[2 * j + 1];
                        const float2 px = make_float2(a.x, a.y), py = make_float2(a.z, a.w);
                        const float2 pz = make_float2(b.x, b.y), pm = make_float2(b.z, b.w);
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            const float2 dx = __fadd2_rn(px, nx[s][0]), dy = __fadd2_rn(py, nx[s][1]),
                                         dz = __fadd2_rn(pz, nx[s][2]);
                            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, e22)));
                            const float2 ri = make_float2(hot_rsqrt(r2.x), hot_rsqrt(r2.y));
                            const float2 mr = __fmul2_rn(pm, ri);
                            const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, ri), ri);
                            if constexpr (MODE == 0) {
                                ax2[s] = __ffma2_rn(mr3, dx, ax2[s]);
                                ay2[s] = __ffma2_rn(mr3, dy, ay2[s]);
                                az2[s] = __ffma2_rn(mr3, dz, az2[s]);
                                ph2[s] = __ffma2_rn(mr, neg1, ph2[s]);
                            } else {
                                // the tangent's pair term (see the scalar form below): ph sums
                                // m/s^3, (a) sums (v m/s^3 - 3 m (d.u)/s^5) d
                                const float2 du = __ffma2_rn(dz, w2[s][2], __ffma2_rn(dy, w2[s][1], __fmul2_rn(dx, w2[s][0])));
                                const float2 k5 = __fmul2_rn(__fmul2_rn(mr3, __fmul2_rn(ri, ri)), du);
                                const float2 cc = __ffma2_rn(k5, neg3, __fmul2_rn(mr3, w2[s][3]));
                                ph2[s] = __fadd2_rn(ph2[s], mr3);
                                ax2[s] = __ffma2_rn(cc, dx, ax2[s]);
                                ay2[s] = __ffma2_rn(cc, dy, ay2[s]);
                                az2[s] = __ffma2_rn(cc, dz, az2[s]);
                            }
                        }
                    }
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        ax[s] = ax2[s].x + ax2[s].y;
                        ay[s] = ay2[s].x + ay2[s].y;
                        az[s] = az2[s].x + az2[s].y;
                        ph[s] = ph2[s].x + ph2[s].y;
                    }
                } else {
                    sweep(std::true_type{});
                }
            } else {
                if (checked)
                    sweep(std::true_type{});
                else
                    sweep(std::false_type{});
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if constexpr (MODE == 0) {
                    acc[s].add(Gt * ax[s], Gt * ay[s], Gt * az[s], Gt * ph[s]);
                } else {
                    acc[s].add(-Gt * (wt[s][0] * ph[s] + ax[s]), -Gt * (wt[s][1] * ph[s] + ay[s]),
                               -Gt * (wt[s][2] * ph[s] + az[s]), T(0));
                }
            }
        }
        __syncwarp();
        fill = 0;
    };
    // 32 list entries at a time: their particle counts are scanned across the lanes, then
    // every lane loads particles of the batch (finding its leaf by binary search in the
    // scanned offsets), so the loads of all 32 leaves are in flight together.
    for (int64_t e0 = G.p0; e0 < G.p1; e0 += 32) {
        const int ne = (int)(G.p1 - e0 < 32 ? G.p1 - e0 : 32);
        int32_t lb = 0, lc = 0;
        T ox = T(0), oy = T(0), oz = T(0);
        bool own = false;
        if ((int)lane < ne) {
            // periodic boundaries: an entry is leaf | image << HOT_IMG_SHIFT; the sources of
            // a leaf of a non-central image are marked (IMG_LEAF) so that no sink meets
            // itself there, and carry the image's shift: in the leaf offset (float32), or
            // alone in its place (float64, whose sources are taken relative to g directly)
            const int32_t ent = l_p2p[e0 + lane];
            int32_t leaf = ent;
            T sx = T(0), sy = T(0), sz = T(0);
            bool central = true;
            if (G.pws > 0) {
                const unsigned img = (uint32_t)ent >> HOT_IMG_SHIFT;
                const int w = 2 * G.pws + 1;
                leaf = (int32_t)((uint32_t)ent & HOT_IMG_CELL_MASK);
                central = 2 * (int)img == w * w * w - 1;
                image_shift(G, img, sx, sy, sz);
            }
            own = central && leaf >= G.own0 && leaf < G.own1;
            lb = cbegin[leaf] | (central ? 0 : IMG_LEAF);
            lc = ccount[leaf];
            if constexpr (sizeof(T) == 4) {
                T h[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) h[q] = rec[(int64_t)leaf * RL + q];
                centre_offset(h, G, ox, oy, oz);
                ox += sx;
                oy += sy;
                oz += sz;
            } else {
                ox = sx;
                oy = sy;
                oz = sz;
            }
        }
        // A chunk holding some of the group's own leaves is staged in two passes: its other
        // leaves first, without the per-pair tests, then its own leaves with them.
        const bool anyown = __any_sync(0xffffffffu, own);
        for (int pass = anyown ? 0 : 1; pass < 2; ++pass) {
            const bool mine = !anyown || (own == (pass == 1));
            const bool checked = (anyown && pass == 1) || !(eps2 > T(0));
            const int incl = warp_incl_scan(mine ? lc : 0);
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            sm.lex[lane + 1] = incl;
            if (lane == 0) sm.lex[0] = 0;
            sm.lbeg[lane] = lb;
            sm.loff[lane][0] = ox;
            sm.loff[lane][1] = oy;
            sm.loff[lane][2] = oz;
            __syncwarp();
            // a lane's sources t only grow, so each search starts from the leaf of its last one
            int lo = 0;
            for (int t0 = 0; t0 < tot; t0 += SRC) {
                const int take = tot - t0 < SRC ? tot - t0 : SRC;
                for (int u = lane; u < take; u += 32) {
                    const int t = t0 + u;
                    int hi = ne;  // leaf j with lex[j] <= t < lex[j + 1]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (sm.lex[mid] <= t)
                            lo = mid;
                        else
                            hi = mid;
                    }
                    const int32_t lbv = sm.lbeg[lo];
                    const int64_t s = (int64_t)(lbv & ~IMG_LEAF) + (t - sm.lex[lo]);
                    if constexpr (sizeof(T) == 4) {
                        const float4 v = prel[s];
                        const float vx = v.x + sm.loff[lo][0], vy = v.y + sm.loff[lo][1], vz = v.z + sm.loff[lo][2];
                        if (PAIRED && !checked) {
                            // pair layout: source u in half u & 1 of pair u >> 1
                            float *q = &sm.src[0][0] + 8 * (u >> 1) + (u & 1);
                            q[0] = vx;
                            q[2] = vy;
                            q[4] = vz;
                            q[6] = v.w;
                        } else {
                            // one 16-byte store per source (scalar stores at a 16-byte lane stride
                            // would meet four lanes in each bank)
                            *reinterpret_cast<float4 *>(&sm.src[u][0]) = make_float4(vx, vy, vz, v.w);
                        }
                    } else {
                        sm.src[u][0] = (T)(spos[3 * s + 0] - G.gx) + sm.loff[lo][0];
                        sm.src[u][1] = (T)(spos[3 * s + 1] - G.gy) + sm.loff[lo][1];
                        sm.src[u][2] = (T)(spos[3 * s + 2] - G.gz) + sm.loff[lo][2];
                        sm.src[u][3] = (T)smass[s];
                    }
                    sm.sidx[u] = (lbv & IMG_LEAF) ? -1 : (int32_t)s;
                }
                if constexpr (PAIRED) {
                    if (!checked && (take & 1) && lane == 0) {
                        // the partner of the last source: massless and far away (its pair terms are 0)
                        float *q = &sm.src[0][0] + 8 * (take >> 1) + 1;
                        q[0] = q[2] = q[4] = 1e17f;
                        q[6] = 0.f;
                    }
                }
                fill = take;
                flush(checked);
            }
        }
    }
}

// Groups whose slices run two sinks per lane (p >= 5): more than 32 sinks, and a last
// 64-sink slice at least three quarters full.  A ragged remainder of up to 48 sinks costs
// less as 32-sink slices, whose small last slice splits its lists across spare lanes
// (clustered 2^20, p = 6: 16.5 ms against 18.2 ms with every group of more than 32; the
// lattice 128^3, whose groups hold about 64 sinks, unchanged at 18.9 ms).
__device__ __forceinline__ bool two_sinks_per_lane(int n) { return n > 32 && (n % 64 == 0 || n % 64 > 48); }

// cls: 0 = every group, 1 = groups of one sink per lane, 2 = groups of two sinks per lane.
// Occupancy (measured on the clustered 2^20 and lattice 128^3 workloads): the forces run
// at 5 CTAs per SM (102 registers; 4% faster than 4 at p = 4, 3% at p = 6), at p = 7, 8 at
// 2 (their staged records fill the shared memory of 2 CTAs); the adjoint's tangent
// evaluation at 4 up to p = 4 and at 2 for p >= 5 (no faster at 3 or 4).
// NS = 1: one sink per lane (slices of 32 sinks, spare lanes split the lists);
// NS = 2: two sinks per lane (slices of 64 sinks: the items at even 32-sink positions).
template <int P, class T, int NS, int MODE, int SOFT, bool VQ>
__global__ void __launch_bounds__(IW * 32, MODE == 1 ? (P >= 5 ? 2 : 4) : (P >= 7 || VQ ? 2 : 5)) k_interact(
    const uint32_t *__restrict__ nitem_p, int cls, const int32_t *__restrict__ gcell, const double *__restrict__ gcen,
    const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount, const int32_t *__restrict__ cend,
    const double *__restrict__ spos, const double *__restrict__ smass, const float4 *__restrict__ prel,
    const double *__restrict__ ccom, const T *__restrict__ rec, const int64_t *__restrict__ off_m2p, const int32_t *__restrict__ l_m2p,
    const int64_t *__restrict__ off_p2p, const int32_t *__restrict__ l_p2p, const uint32_t *__restrict__ perm,
    const uint64_t *__restrict__ items, T eps2, double G, unsigned *__restrict__ work, double *__restrict__ acc_out, double *__restrict__ pot_out,
    const T *__restrict__ wsink, double *__restrict__ gsink, uint32_t wait_limit, int probe,
    unsigned *__restrict__ status, const RecTab<T> rq, double per_L, int per_ws)
{
    using S = Smem<P, T>;
    constexpr int CH = Cfg<P, T>::CH;
    constexpr int SL = 32 * NS;  // sinks per slice
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = reinterpret_cast<S *>(smem_raw)[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const T Gt = (T)G;
    if (lane == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_init(&sm.probe, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    uint32_t phase[2] = {0u, 0u};

    const int64_t nitem = *nitem_p;
    for (;;) {
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(work, 1u);
        const int64_t ii = __shfl_sync(0xffffffffu, i0, 0);
        if (ii >= nitem) break;
        const uint64_t item = items[ii];  // largest slice cost first
        const int64_t g = (int64_t)(item >> 32);
        const int s0 = (int)(uint32_t)item;
        if (s0 % SL != 0) continue;  // two sinks per lane: one item per 64-sink slice
        const int32_t gc = gcell[g];
        Group<T> Gr;
        Gr.n = ccount[gc];
        if ((cls == 1 && two_sinks_per_lane(Gr.n)) || (cls == 2 && !two_sinks_per_lane(Gr.n))) continue;
        Gr.gb = cbegin[gc];
        Gr.gx = gcen[3 * g + 0];
        Gr.gy = gcen[3 * g + 1];
        Gr.gz = gcen[3 * g + 2];
        {
            const double gv[3] = {Gr.gx, Gr.gy, Gr.gz};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Gr.ghi[d] = (T)gv[d];
                Gr.glo[d] = (T)(gv[d] - (double)Gr.ghi[d]);
            }
        }
        Gr.m0 = off_m2p[g];
        Gr.m1 = off_m2p[g + 1];
        Gr.p0 = off_p2p[g];
        Gr.p1 = off_p2p[g + 1];
        Gr.own0 = gc;
        Gr.own1 = cend[gc];
        Gr.pL = per_L;
        Gr.pws = per_L > 0.0 ? per_ws : 0;
        {
            const int rem = Gr.n - s0;
            int ns, nsplit, si, sj;
            if (NS == 1) {
                ns = rem < 32 ? rem : 32;
                nsplit = 32 / ns;
                if (nsplit > CH) nsplit = CH;
                si = (int)lane % ns;
                sj = (int)lane / ns;
            } else {
                ns = rem;
                nsplit = 1;
                si = (int)lane;
                sj = 0;
            }
            const bool active = sj < nsplit;
            T x[NS][3], wt[NS][4];
            int32_t self[NS];
            int64_t slot[NS];
            bool valid[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int k = si + 32 * q;
                valid[q] = k < ns;
                slot[q] = Gr.gb + s0 + (valid[q] ? k : ns - 1);
                x[q][0] = (T)(spos[3 * slot[q] + 0] - Gr.gx);
                x[q][1] = (T)(spos[3 * slot[q] + 1] - Gr.gy);
                x[q][2] = (T)(spos[3 * slot[q] + 2] - Gr.gz);
                self[q] = (int32_t)slot[q];
#pragma unroll
                for (int d = 0; d < 4; ++d) wt[q][d] = MODE == 0 ? T(0) : wsink[4 * slot[q] + d];
            }
            Acc<T> acc[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) acc[q].zero();
            if (!m2p_list<P, T, NS, MODE, VQ>(sm, Gr, l_m2p, rec, rq, x, wt, sj, nsplit, active, acc, phase, wait_limit,
                                          probe != 0, status))
                return;
            p2p_list<P, T, NS, MODE, SOFT>(sm, Gr, l_p2p, cbegin, ccount, rec, prel, spos, smass, x, wt, self, sj, nsplit, active,
                               eps2, Gt, acc);
            if (NS == 1) {
                // combine the list splits of each sink in float64
                __syncwarp();
                if (active) {
#pragma unroll
                    for (int d = 0; d < 4; ++d) sm.red[lane][d] = acc[0].get(d);
                }
                __syncwarp();
                if (active && sj == 0) {
                    double t[4] = {0, 0, 0, 0};
                    for (int j = 0; j < nsplit; ++j)
#pragma unroll
                        for (int d = 0; d < 4; ++d) t[d] += sm.red[si + j * ns][d];
                    if constexpr (MODE == 0) {
                        const int64_t i = perm[slot[0]];
                        acc_out[3 * i + 0] = t[0];
                        acc_out[3 * i + 1] = t[1];
                        acc_out[3 * i + 2] = t[2];
                        if (pot_out) pot_out[i] = t[3];
                    } else {
                        gsink[3 * slot[0] + 0] = t[0];
                        gsink[3 * slot[0] + 1] = t[1];
                        gsink[3 * slot[0] + 2] = t[2];
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < NS; ++q)
                    if (valid[q]) {
                        if constexpr (MODE == 0) {
                            const int64_t i = perm[slot[q]];
                            acc_out[3 * i + 0] = acc[q].get(0);
                            acc_out[3 * i + 1] = acc[q].get(1);
                            acc_out[3 * i + 2] = acc[q].get(2);
                            if (pot_out) pot_out[i] = acc[q].get(3);
                        } else {
                            gsink[3 * slot[q] + 0] = acc[q].get(0);
                            gsink[3 * slot[q] + 1] = acc[q].get(1);
                            gsink[3 * slot[q] + 2] = acc[q].get(2);
                        }
                    }
            }
            __syncwarp();
        }
    }
}

template <int P, class T, int NS, int MODE, int SOFT, bool VQ = false>
int launch_interact_s(hot_ctx *c, cudaStream_t s, int cls, unsigned *work, double *acc, double *pot, const T *wsink,
                      double *gsink)
{
    const size_t smem = sizeof(Smem<P, T>) * IW;
    auto kern = k_interact<P, T, NS, MODE, SOFT, VQ>;
    HOT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HOT_CK(cudaMemsetAsync(work, 0, sizeof(unsigned), s));
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
    // records of every order (used under per-interaction order selection)
    static_assert(HOT_PMAX + 1 <= HOT_ORDERS, "order table");
    RecTab<T> rq{};
    for (int q = 0; q <= HOT_PMAX; ++q) {
        rq.rl[q] = HOT_REC_LEN[q];
        if constexpr (sizeof(T) == 4)
            rq.rec[q] = q == P ? c->rec32.p : c->rec32q[q].p;
        else
            rq.rec[q] = q == P ? c->rec64.p : c->rec64q[q].p;
    }
    HOT_COUNT_LAUNCH();
    kern<<<blocks, IW * 32, smem, s>>>(c->slice_off.p + c->ngroup, cls, c->gcell.p, c->gcen.p, c->cbegin.p, c->ccount.p, c->cend.p,
                                       c->spos.p,
                                       c->smass.p, c->prel.p, c->ccom.p, rec, c->off_m2p.p, c->l_m2p.p, c->off_p2p.p,
                                       c->l_p2p.p, c->idx.p, c->items.p, eps2, c->prm.G, work, acc, pot, wsink,
                                       gsink, c->wait_polls ? c->wait_polls : WAIT_LIMIT, c->wait_probe,
                                       c->d_status, rq, c->prm.box > 0.0 ? c->prm.box : 0.0, c->prm.ws);
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}

}  // namespace
