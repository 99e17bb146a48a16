// hot_common.cuh -- context, device buffers, status word and shared device helpers
// of the hashed oct-tree library (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <vector>

#include "hot.h"

// ---------------------------------------------------------------------------
// Status word bits (device side).  Kernels atomicOr a bit and skip the access
// that would have gone wrong; the host turns bits into HOT_E* codes.
// ---------------------------------------------------------------------------
#define HOT_ST_INPUT 1u      // non-finite position/mass
#define HOT_ST_FRONTIER 2u   // traversal frontier scratch too small
#define HOT_ST_HASH 4u       // hash probe limit reached
#define HOT_ST_TIMEOUT 8u    // a bounded wait gave up
#define HOT_ST_INTERNAL 16u  // a consistency check failed (index out of range)

#define HOT_MAXLEVEL 21

// Per-interaction order selection: an M2P list entry is cell | order << HOT_ORDER_SHIFT.
#define HOT_ORDER_SHIFT 27
#define HOT_CELL_MASK ((1u << HOT_ORDER_SHIFT) - 1u)
#define HOT_ORDERS 9  // orders 0..8
// Periodic boundaries: a list entry is cell | image << HOT_IMG_SHIFT, image index
// ((nx + ws) w + ny + ws) w + nz + ws, w = 2 ws + 1.
#define HOT_IMG_SHIFT 24
#define HOT_IMG_CELL_MASK ((1u << HOT_IMG_SHIFT) - 1u)
#define HOT_WS_MAX 2  // (2 ws + 1)^3 images in the 8 bits above HOT_IMG_SHIFT
#define HOT_PFAR 8    // order of the far images' local expansion
#define HOT_BG_PMAX 6 // largest order under background subtraction (its moments go to p + 2)

// Device memory the one-pass traversal may hold in per-group list slots (bytes).
#define HOT_SLOT_BUDGET (16.0 * 1024 * 1024 * 1024)

// Number of kernel launches issued by this library (all contexts), for benchmarks.
extern std::atomic<long long> hot_launch_counter;
#define HOT_COUNT_LAUNCH() hot_launch_counter.fetch_add(1, std::memory_order_relaxed)

// Device bytes held in DBufs by all contexts, and the largest value since the last reset.
extern std::atomic<long long> hot_bytes_held, hot_bytes_peak;
inline void hot_bytes_add(long long d)
{
    long long now = hot_bytes_held.fetch_add(d, std::memory_order_relaxed) + d;
    long long pk = hot_bytes_peak.load(std::memory_order_relaxed);
    while (now > pk && !hot_bytes_peak.compare_exchange_weak(pk, now, std::memory_order_relaxed)) {
    }
}

// ---------------------------------------------------------------------------
// Grow-only device buffer, stream-ordered allocation.
// ---------------------------------------------------------------------------
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t n, cudaStream_t s)
    {
        if (n <= cap && p) return cudaSuccess;
        release(s);
        size_t want = n + n / 8 + 64;
        cudaError_t e = cudaMallocAsync((void **)&p, want * sizeof(T), s);
        if (e == cudaSuccess) {
            cap = want;
            hot_bytes_add((long long)(want * sizeof(T)));
        }
        return e;
    }
    void release(cudaStream_t s)
    {
        if (p) {
            cudaFreeAsync(p, s);
            hot_bytes_add(-(long long)(cap * sizeof(T)));
        }
        p = nullptr;
        cap = 0;
    }
};

enum { ST_TIMING_EVENTS = 14 };

// Per-cell traversal record: centre of mass and the acceptance radius r_c for the
// current tolerance (a cell is accepted for a group iff |z - g| - Delta_max >= r_c).
struct alignas(32) TCell {
    double x, y, z, rc;
};

// The same in float32 for the traversal's pre-test: the centre as a hi/lo pair (hi =
// rounded, lo = remainder) and r_c rounded.
struct alignas(32) TCellF {
    float hx, hy, hz, lx, ly, lz, rc, pad;
};

struct hot_ctx {
    hot_params prm;
    cudaStream_t st = nullptr;
    // second stream: the adjoint's sink pass runs on it beside the source side, forked from
    // and joined back into st by the two events
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the moment translations and the records run on st2 beside the acceptance aggregates
    // and the traversal (forked after the centres of mass, the records after the
    // aggregates); every later use joins them back into st (hot_join_moments)
    cudaEvent_t ev_mfork = nullptr, ev_mcomb = nullptr, ev_mjoin = nullptr;
    bool mom_pending = false;
    int dev = 0, nsm = 0;
    int stage = 0;  // 0 created, 1 tree, 2 moments, 3 lists
    int64_t N = 0;

    // keys and sort
    DBuf<double> part;     // bbox partials
    DBuf<double> frame;    // lo[3], L, scale
    DBuf<uint64_t> key, key2;
    DBuf<uint32_t> idx, idx2;
    DBuf<uint64_t> scan_tmp;
    // one-launch-per-pass radix sort of the keys: per-block digit histograms of all eight
    // passes, the passes' global digit offsets, tile counters, and the tiles' published
    // digit counts (one array per pass, cleared once per sort)
    DBuf<uint32_t> rs_bhist, rs_goff, rs_ctr;
    DBuf<uint32_t> rs_status;
    DBuf<double> spos, smass;  // sorted copies [N][3], [N]

    // tree
    DBuf<uint8_t> lcp, leaflev;
    DBuf<uint32_t> ncell_i, cell_off;
    int64_t ncell = 0, nleaf = 0, maxlevel = 0, ngroup = 0;
    DBuf<uint64_t> ckey;
    DBuf<int32_t> clevel, cbegin, ccount, cparent, cend, child8, cnchild;
    DBuf<int32_t> level_cells;
    std::vector<int64_t> level_off;  // host, HOT_MAXLEVEL + 2 entries
    DBuf<uint64_t> hkey;
    DBuf<int32_t> hval;
    uint64_t hcap = 0;
    DBuf<uint32_t> gflag, goff;
    DBuf<int32_t> gcell;
    DBuf<double> gcen, gdmax;
    DBuf<int64_t> sizes;  // device scratch for counts read back at sync points

    // moments
    int p_mom = -1;
    int reclen = 0;
    DBuf<double> cmass, ccom, cmom, cbmax, cB1, cB2;
    DBuf<uint32_t> item_off;
    DBuf<int32_t> item_cell;
    DBuf<double> item_part;
    DBuf<float> rec32;
    DBuf<double> rec64;
    DBuf<float4> prel;
    // per-interaction order selection (0 <= p_min < p): orders q_lo..p_mom
    int varq = 0, q_lo = 0;
    DBuf<double> cBn;                  // [ncell][p+3]: B_n = sum m |x - z|^n, n = 0..p+2
    DBuf<uint32_t> bn_cnt, bn_off;     // aggregate work items of every cell
    DBuf<int32_t> bn_cell;
    DBuf<double> bn_part;
    DBuf<float> rec32q[HOT_ORDERS];    // records of the orders below p (order p: rec32 / rec64)
    DBuf<double> rec64q[HOT_ORDERS];
    DBuf<double> rcq;                  // [ncell][p - q_lo + 1]: acceptance radius of each order
    DBuf<float> rcqf;                  // the same rounded to float32 (the traversal's pre-test)
    // periodic boundaries: lattice sums D^g psi_far(0) (host copy and device, for the side
    // per_D_L and ws per_D_ws), moment partials and L2P coefficients of the far images
    std::vector<double> per_Dh;
    double per_D_L = 0.0;
    int per_D_ws = 0;
    DBuf<double> per_D, per_part, per_coef;

    // background subtraction: the cubes are the cells [0, C) and the empty octants of the
    // inner cells [C, C + E) (octants that hold no particle, absent from the tree); their
    // centres and half sides, the contrast's Q_{p+1}, Q_{p+2}, the empty octants' parents
    // and octant numbers, the cells' moments about their cube centres to order p + 2 (then
    // their contrast), the mean density, and per tolerance each cube's acceptance record
    int64_t n_empty = 0;
    DBuf<double> bg_cen, bg_half, bg_q, bg_mom, bg_rho, bg_tab;
    DBuf<uint32_t> bg_ecnt, bg_eoff;
    DBuf<int32_t> bg_eparent, bg_eoct;
    DBuf<TCell> bg_tc;
    DBuf<TCellF> bg_tcf;
    // per group: the analytic-cube list (cube indices) and the surrounding cube S
    DBuf<uint32_t> cnt_box;
    DBuf<int64_t> off_box;
    DBuf<int32_t> l_box, bg_gS;
    int64_t n_box = 0, n_box_eval = 0, n_m2p_con = 0, n_m2p_emp = 0;

    // lists
    double tol_lists = 0;
    int64_t n_m2p = 0, n_p2p = 0, n_pairs = 0, n_m2p_int = 0;
    int64_t n_p2p_src = 0;  // P2P source-particle visits: sum over groups of listed leaf sizes
    DBuf<uint32_t> cnt_m2p, cnt_p2p;
    DBuf<int64_t> off_m2p, off_p2p;
    DBuf<int32_t> l_m2p, l_p2p;
    DBuf<int32_t> trav_scratch;
    DBuf<TCell> tcell;
    DBuf<TCellF> tcellf;

    // adjoint
    DBuf<unsigned char> adj_w;   // sink weights (u, v) per sorted slot, T4
    DBuf<float> adj_xhl;         // sorted positions as float hi/lo pairs [N][8]
    DBuf<double> adj_gsink, adj_gp2p, adj_mbar;
    DBuf<uint64_t> tp_key, tp_key2;
    DBuf<uint32_t> tp_val, tp_val2;
    DBuf<int64_t> tp_start, tp_end;
    DBuf<uint32_t> it_cnt, it_off;
    DBuf<int32_t> it_cell;
    DBuf<int64_t> it_a, it_b;
    DBuf<unsigned char> it_part;
    DBuf<unsigned char> adj_pp;  // P2P source-side partial sums per work item and leaf particle
    DBuf<int64_t> adj_roff;      // first partial row of every leaf
    int trav_cap = 2048;
    uint32_t wait_polls = 0;  // interaction kernels' chunk-wait poll limit (0: default)
    int wait_probe = 0;       // test setting: every group's M2P list first waits on a barrier
                              // that nothing completes
    // per-group slot capacities of the one-pass traversal (grown from the counts seen)
    int64_t slot_capm = 2048, slot_capp = 512;
    DBuf<int32_t> slot_m2p, slot_p2p;
    DBuf<uint64_t> gkey, gkey2;      // per-group cost keys of one 32-sink slice (largest first)
    DBuf<uint32_t> gorder, gorder2;  // groups in descending slice cost
    DBuf<uint32_t> slice_cnt, slice_off;  // 32-sink slices per group (sorted order), offsets
    DBuf<uint64_t> items;            // work items of the interaction kernels: group << 32 | first sink

    // status
    unsigned *d_status = nullptr;
    unsigned *h_status = nullptr;

    // timing: pairs of events per stage
    cudaEvent_t ev[ST_TIMING_EVENTS] = {};
    float stage_ms[6] = {0, 0, 0, 0, 0, 0};
    bool ev_used[7] = {false, false, false, false, false, false, false};
};

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
#define HOT_CK(call)                                  \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            return (e_ == cudaErrorMemoryAllocation) \
                       ? HOT_ENOMEM                   \
                       : HOT_ECUDA;                   \
        }                                             \
    } while (0)

static inline int hot_blocks(int64_t n, int threads, int cap = 1 << 30)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// Stage timing: start/stop a CUDA-event pair on the context stream.
static inline void hot_tic(hot_ctx *c, int stage) { cudaEventRecord(c->ev[2 * stage], c->st); }
// st waits for the moment work left on st2 by the last hot_compute_moments.
static inline int hot_join_moments(hot_ctx *c)
{
    if (!c->mom_pending) return 0;
    c->mom_pending = false;
    return cudaStreamWaitEvent(c->st, c->ev_mjoin, 0) == cudaSuccess ? 0 : HOT_ECUDA;
}
static inline void hot_toc(hot_ctx *c, int stage)
{
    cudaEventRecord(c->ev[2 * stage + 1], c->st);
    c->ev_used[stage] = true;
}

// Read the status word (synchronises) and clear it.
int hot_sync_status(hot_ctx *c);

// Exclusive scan of n values (In) into out[0..n] (Out); out[n] = total.
// Device-wide, deterministic.  tmp must hold hot_scan_tmp_elems(n) uint64.
size_t hot_scan_tmp_elems(int64_t n);
int hot_scan_u32_to_u32(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *tmp,
                        cudaStream_t s);
int hot_scan_u32_to_i64(const uint32_t *in, int64_t *out, int64_t n, uint64_t *tmp,
                        cudaStream_t s);

// Stages implemented in separate translation units.
int hot_impl_build(hot_ctx *c, const double *pos, const double *mass, int64_t N);
int hot_impl_moments(hot_ctx *c, int p);
int hot_impl_traverse(hot_ctx *c, double tol);
int hot_impl_forces(hot_ctx *c, double *acc, double *pot);
int hot_impl_forces_vq(hot_ctx *c, double *acc, double *pot);
int hot_impl_far_field(hot_ctx *c, double *acc, double *pot);
int hot_impl_adjoint(hot_ctx *c, const double *g_acc, const double *g_pot, double *g_pos,
                     double *g_mass);
int hot_impl_adjoint_sink(hot_ctx *c, const void *wsink, double *gsink, cudaStream_t s);
int hot_sort_pairs(hot_ctx *c, uint64_t *keys, uint32_t *vals, uint64_t *ktmp, uint32_t *vtmp, int64_t n, int bits);
int hot_impl_bg_box(hot_ctx *c, double *acc, double *pot);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// 1/sqrt(u) in float32: the approximate reciprocal square root with subnormal inputs flushed
// to zero (rsqrt.approx.ftz.f32), one special-function instruction.  Every float32 caller
// passes |R|^2 + eps^2 of an accepted cell or a source pair (normal numbers, or 0 where the
// result is masked); a subnormal argument gives +inf here, where the plain approximation
// gives a value that overflows the same expressions.
__device__ __forceinline__ float hot_rsqrt(float u)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(u));
    return r;
}
__device__ __forceinline__ double hot_rsqrt(double u) { return rsqrt(u); }

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

template <class T>
__device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// Inclusive warp scan.
template <class T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    unsigned l = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (l >= (unsigned)o) v += u;
    }
    return v;
}

// Number of leading equal octal digits (levels) of two particle keys (0..21).
__device__ __forceinline__ int key_lcp_levels(uint64_t a, uint64_t b)
{
    uint64_t x = a ^ b;
    if (x == 0) return HOT_MAXLEVEL;
    return (__clzll((long long)x) - 1) / 3;
}

__device__ __forceinline__ void hot_flag(unsigned *status, unsigned bit) { atomicOr(status, bit); }

// K1 compensating force smoothing of support eps (Sec. "Force Smoothing"; the kernel is
// the unit-mass density 105/(64 pi eps^3) (1 - x^2)(5 - 9 x^2), x = r/eps).  A source of
// mass m at d (r^2 = |d|^2) gives a = G m f d and phi = -G m psi, and f2 = 2 df/d(r^2)
// enters the pair's tidal tensor -G m (f I + f2 d d^T).  For r < eps, u = r^2/eps^2:
//   f = (175/16 - 147/8 u + 135/16 u^2)/eps^3, f2 = (-147/4 + 135/4 u)/eps^5,
//   psi = (105 - 175 u + 147 u^2 - 45 u^3)/(32 eps);
// Newtonian (f = r^-3, f2 = -3 r^-5, psi = 1/r) for r >= eps.  Finite at r = 0 when eps > 0.
// Evaluated in t = 1 - u, where every coefficient has one sign (the powers of u cancel to
// a tenth near the edge, which float32 would pay for):
//   f eps^3 = 1 + 3/2 t + 135/16 t^2,  f2 eps^5 = -(3 + 135/4 t),
//   psi eps = 1 + t/2 + 3/8 t^2 + 45/32 t^3.
template <class T>
struct SoftConst {
    T e2, ie2, ie, ie3, ie5;  // eps^2, 1/eps^2, 1/eps, 1/eps^3, 1/eps^5
};

template <class T>
__device__ __forceinline__ SoftConst<T> soft_const(T eps2)
{
    SoftConst<T> k;
    k.e2 = eps2;
    k.ie2 = T(1) / eps2;
    k.ie = T(1) / sqrt(eps2);  // correctly rounded: a common factor of every inside pair
    k.ie3 = k.ie2 * k.ie;
    k.ie5 = k.ie3 * k.ie2;
    return k;
}

template <class T>
__device__ __forceinline__ void k1_pair(T r2, const SoftConst<T> &k, T &f, T &f2, T &psi)
{
    const bool in = r2 < k.e2;
    const T ri = hot_rsqrt(in ? k.e2 : r2);
    const T ri2 = ri * ri;
    const T t = T(1) - r2 * k.ie2;
    const T fin = (T(1) + t * (T(1.5) + t * T(135.0 / 16.0))) * k.ie3;
    const T f2in = -(T(3) + t * T(135.0 / 4.0)) * k.ie5;
    const T pin = (T(1) + t * (T(0.5) + t * (T(0.375) + t * T(45.0 / 32.0)))) * k.ie;
    f = in ? fin : ri2 * ri;
    f2 = in ? f2in : T(-3) * ri2 * ri2 * ri;
    psi = in ? pin : ri;
}

// Cubic spline force smoothing of support eps (Sec. "Force Smoothing", the kernel of the
// cited SPH code): the unit-mass density 8/(pi eps^3) w(x), x = r/eps, w = 1 - 6x^2 + 6x^3
// for x < 1/2 and 2(1 - x)^3 for 1/2 <= x < 1, zero beyond.  Same pair functions as
// k1_pair (a = G m f d, phi = -G m psi, f2 = 2 df/d(r^2)).  With M(x) the enclosed mass:
//   x < 1/2:  f eps^3 = 32/3 - 192/5 x^2 + 32 x^3,  f2 eps^5 = -384/5 + 96 x,
//             psi eps = 14/5 - 16/3 x^2 + 48/5 x^4 - 32/5 x^5;
//   x >= 1/2, t = 1 - x (M = 1 - 16 t^4 + 128/5 t^5 - 32/3 t^6, from integrating the
//   density 16/pi t^3 inwards from the edge, where M = 1):
//             f = M / r^3,  f2 = 64 t^3 / (eps^3 r^2) - 3 M / r^5   (dM/dx = 64 x^2 t^3),
//             psi = M / r + (16 t^4 - 64/5 t^5) / eps   (psi - M/r has derivative
//             -dM/dx /(eps r) in r and vanishes at the edge);
// Newtonian for r >= eps.  The outer branch is written in t so that its float32 terms do
// not cancel near the edge, where the expanded powers of x sum terms of size 48 to 1.
template <class T>
__device__ __forceinline__ void spline_pair(T r2, const SoftConst<T> &k, T &f, T &f2, T &psi)
{
    const bool in = r2 < k.e2;
    const T ri = hot_rsqrt(r2 > T(0) ? r2 : k.e2);  // r2 = 0 only reaches the inner branch
    const T ri2 = ri * ri;
    const T ri3 = ri2 * ri;
    const T x = r2 * ri * k.ie;  // r / eps (0 at r = 0)
    const T x2 = x * x;
    const T gi = T(32.0 / 3.0) + x2 * (T(-192.0 / 5.0) + T(32) * x);
    const T f2i = T(-384.0 / 5.0) + T(96) * x;
    const T pi_ = T(14.0 / 5.0) + x2 * (T(-16.0 / 3.0) + x2 * (T(48.0 / 5.0) - T(32.0 / 5.0) * x));
    const T t = T(1) - x;
    const T t3 = t * t * t;
    const T t4 = t3 * t;
    const T mo = T(1) - t4 * (T(16) - t * (T(128.0 / 5.0) - T(32.0 / 3.0) * t));
    const T fo = mo * ri3;
    const T f2o = T(64) * t3 * ri2 * k.ie3 - T(3) * mo * ri3 * ri2;
    const T po = mo * ri + t4 * (T(16) - T(64.0 / 5.0) * t) * k.ie;
    const bool inner = x < T(0.5);
    f = in ? (inner ? gi * k.ie3 : fo) : ri3;
    f2 = in ? (inner ? f2i * k.ie5 : f2o) : T(-3) * ri2 * ri3;
    psi = in ? (inner ? pi_ * k.ie : po) : ri;
}

// The pair functions of a kernel of compact support (K1 or the cubic spline).
template <int SOFT, class T>
__device__ __forceinline__ void compact_pair(T r2, const SoftConst<T> &k, T &f, T &f2, T &psi)
{
    if constexpr (SOFT == HOT_SOFT_SPLINE)
        spline_pair(r2, k, f, f2, psi);
    else
        k1_pair(r2, k, f, f2, psi);
}

#endif  // __CUDACC__
