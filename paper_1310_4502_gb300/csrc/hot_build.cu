// hot_build.cu -- bounding cube, Morton keys, LSD radix sort, gather, hashed oct-tree
// and sink groups (Warren 2013: Sec. "Domain Decomposition" -- space-filling-curve keys
// turn the decomposition into a sort; Sec. "Tree Construction and Traversal" -- cells
// are key prefixes addressed through a hash table).
//
// Tree construction is fully parallel over the sorted keys.  With lcp(a, b) the
// number of leading equal octal digits of two keys:
//   * the level-l cell holding particle i has more than leaf_max particles iff some
//     window t in [i - leaf_max, i] has lcp(key_t, key_{t+leaf_max}) >= l, so the
//     level of i's leaf is min(21, 1 + max_t lcp(key_t, key_{t+leaf_max}));
//   * particle i is the first particle of a level-l cell iff lcp(key_{i-1}, key_i) < l,
//     and that cell exists iff its parent was refined, i.e. iff l <= leaf level(i).
// So particle i "owns" the cells of levels lcp(key_{i-1}, key_i)+1 .. leaf level(i);
// a scan of those counts numbers every cell, and the numbering is the depth-first
// pre-order of the tree (children in ascending octant), which also makes every
// subtree a contiguous index range.
#include "hot_common.cuh"

namespace {

constexpr int BT = 256;

// ---------------------------------------------------------------------------
// Bounding cube
// ---------------------------------------------------------------------------
// The minimum and maximum of doubles are exact, so they are taken on integer images of
// the bit patterns that order as the values do (sign bit set: all bits flipped; clear:
// the sign bit set) -- integer compares instead of the float64 pipe, which on this part
// runs at a sixty-fourth of the float32 rate.  The check for non-finite values and
// non-positive masses is a test of the exponent and sign bits.
__device__ __forceinline__ unsigned long long ord_image(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_value(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}
__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
__device__ __forceinline__ bool bits_finite(unsigned long long u)
{
    return (u & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

__global__ void k_bbox_part(const double *__restrict__ pos, const double *__restrict__ mass,
                            int64_t N, double *__restrict__ part, unsigned *status)
{
    unsigned long long lk[3] = {~0ull, ~0ull, ~0ull}, hk[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += 4 * stride) {
        // four particles per thread in flight
        unsigned long long mu[4], xu[4][3];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + q * stride;
            const bool v = i < N;
            mu[q] = v ? (unsigned long long)__double_as_longlong(mass[i]) : 0x3ff0000000000000ull;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                xu[q][d] = v ? (unsigned long long)__double_as_longlong(pos[3 * i + d]) : 0ull;
            if (!v) {
#pragma unroll
                for (int d = 0; d < 3; ++d) xu[q][d] = (unsigned long long)__double_as_longlong(pos[3 * i0 + d]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // mass: finite, not negative, not zero (+0 and -0 alike)
            bad |= !bits_finite(mu[q]) || (mu[q] >> 63) || (mu[q] << 1) == 0ull;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                bad |= !bits_finite(xu[q][d]);
                const unsigned long long k = ord_image(__longlong_as_double((long long)xu[q][d]));
                lk[d] = k < lk[d] ? k : lk[d];
                hk[d] = k > hk[d] ? k : hk[d];
            }
        }
    }
    double lo[3], hi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lo[d] = lk[d] == ~0ull ? INFINITY : ord_value(lk[d]);
        hi[d] = hk[d] == 0ull ? -INFINITY : ord_value(hk[d]);
    }
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) hot_flag(status, HOT_ST_INPUT);
    __shared__ double sh[BT / 32][6];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lo[d] = warp_min(lo[d]);
        hi[d] = warp_max(hi[d]);
    }
    if (lane_id() == 0)
        for (int d = 0; d < 3; ++d) {
            sh[threadIdx.x >> 5][d] = lo[d];
            sh[threadIdx.x >> 5][3 + d] = hi[d];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        int d = threadIdx.x;
        double v = sh[0][d];
        for (int w = 1; w < BT / 32; ++w) v = d < 3 ? fmin(v, sh[w][d]) : fmax(v, sh[w][d]);
        part[6 * blockIdx.x + d] = v;
    }
}

// frame = lo[3], L, 2^21/L.  One warp: lanes take the block partials in turn, then a warp
// reduction (min and max are exact, so the order does not matter).
// One block of BF threads (min and max are exact, so the order of the reduction is free).
constexpr int BF = 256;
__global__ void __launch_bounds__(BF) k_bbox_final(const double *__restrict__ part, int nb, double *__restrict__ frame)
{
    __shared__ double sw[BF / 32][6];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nb; b += BF)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], part[6 * b + d]);
            hi[d] = fmax(hi[d], part[6 * b + 3 + d]);
        }
    for (int d = 0; d < 3; ++d) {
        lo[d] = warp_min(lo[d]);
        hi[d] = warp_max(hi[d]);
    }
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0)
        for (int d = 0; d < 3; ++d) {
            sw[w][d] = lo[d];
            sw[w][3 + d] = hi[d];
        }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int q = 1; q < BF / 32; ++q)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], sw[q][d]);
            hi[d] = fmax(hi[d], sw[q][3 + d]);
        }
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = __dsub_rn(hi[d], lo[d]);
        if (e > ext) ext = e;
    }
    double L = ext > 0.0 ? ext : 1.0;
    for (int d = 0; d < 3; ++d) frame[d] = lo[d];
    frame[3] = L;
    frame[4] = __ddiv_rn(2097152.0, L);
}

// ---------------------------------------------------------------------------
// Keys: magic-number bit spreading of 21-bit integer coordinates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint64_t icoord(double x, double lo, double s)
{
    const double t = __dmul_rn(__dsub_rn(x, lo), s);  // one subtract, one multiply, no contraction
    // floor(t) for 0 <= t < 2^21 from the bit pattern (the integer part of the significand
    // shifted by the exponent), 0 below, 2^21 - 1 above: exact, and on the integer pipe
    // where a rounding conversion would take the float64 one
    const uint64_t u = (uint64_t)__double_as_longlong(t);
    if ((int64_t)u <= 0) return 0ull;  // t <= 0 (the sign bit set, or +0)
    const int e = (int)((u >> 52) & 0x7ffull) - 1023;
    if (e < 0) return 0ull;
    if (e >= 21) return 2097151ull;  // also inf and NaN
    return ((u & 0xfffffffffffffull) | 0x10000000000000ull) >> (52 - e);
}

// ---------------------------------------------------------------------------
// The particle keys' sort: eight LSD passes of 8 bits.
//   * k_keys_hist computes the keys and, in the same pass, the digit histograms of all
//     eight passes (one per block in shared memory; a warp whose keys share a digit adds
//     them at once) and, when the tiles are counted (below), the first pass's tile counts;
//   * k_rs_goff reduces the block histograms and scans them into each pass's global
//     digit offsets;
//   * k_rs_pass ranks a tile of keys by digit in shared memory (stable: warp w
//     holds the tile's w-th run of OS_R * 32 consecutive keys, ranked round by round in
//     lane order) and writes them in digit order, so that each digit's run leaves as
//     contiguous stores.  How many keys of each digit the earlier tiles hold comes one of
//     two ways.  Few tiles: by a decoupled look-back over the counts the tiles publish (a
//     tile publishes its own counts before it looks back, and tiles are numbered in the
//     order their blocks start, so every wait ends), reading OS_LB earlier tiles' words at
//     a time; the tiles of a wave start together, so the last inclusive count a tile finds
//     lies about a wave behind, and the walk's chain of dependent reads is that distance
//     over OS_LB.  Many tiles: k_rs_count counts every tile's digits first (reading the
//     keys once more) and k_rs_tscan scans them digit by digit, so that no tile waits.
// A published word is flag << 30 | count: flag 1 = this tile's count, 2 = the count of this
// tile and all before it, 0 = not yet written (every pass has its own words, cleared once
// per sort).
// ---------------------------------------------------------------------------
constexpr int OS_W = 8;  // warps per block (thread d of the block owns digit d)
// keys per lane: 16 on the look-back path (4096-key tiles keep the chains short; 117
// registers, 2 blocks per SM); 8 when the tiles are counted first (2048-key tiles, 64
// registers: 4 blocks per SM, 9% faster at 256^3 than 4096-key tiles at 2)
constexpr int OS_R_LB = 16, OS_R_SCAN = 8;
template <int R>
struct OsTile {
    static constexpr int TILE = OS_W * R * 32;  // keys per tile
    static constexpr int SMEM = OS_W * 256 * 4 + TILE * 8 + TILE * 4 + 2 * 256 * 4;
};
constexpr uint32_t OS_FLAG_AGG = 1u, OS_FLAG_INC = 2u;
constexpr long OS_POLL_LIMIT = 1l << 20;  // polls of one published word before giving up
constexpr int OS_LB = 32;                  // earlier tiles' words read together in the look-back

__device__ __forceinline__ uint32_t os_pack(uint32_t flag, uint32_t cnt) { return (flag << 30) | cnt; }

// Blocks take tiles of TILE keys in turn; with thist0, each tile's first-pass digit counts
// go to thist0[d * ntiles + tile] (the counted first pass of the sort needs no count of its
// own).
template <int TILE>
__global__ void __launch_bounds__(256) k_keys_hist(const double *__restrict__ pos, int64_t N,
                                                   const double *__restrict__ frame, uint64_t *__restrict__ key,
                                                   uint32_t *__restrict__ idx, uint32_t *__restrict__ bhist,
                                                   uint32_t *__restrict__ thist0)
{
    __shared__ uint32_t h[8][256], h0[256];
    for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) h[k >> 8][k & 255] = 0;
    h0[threadIdx.x] = 0;
    __syncthreads();
    const double s = frame[4], lx = frame[0], ly = frame[1], lz = frame[2];
    const unsigned lane = lane_id();
    const int64_t ntiles = (N + TILE - 1) / TILE;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int r = 0; r < TILE / 256; ++r) {
            const int64_t i = t * TILE + r * 256 + threadIdx.x;
            const bool valid = i < N;
            uint64_t k = 0;
            if (valid) {
                const uint64_t cx = icoord(pos[3 * i + 0], lx, s);
                const uint64_t cy = icoord(pos[3 * i + 1], ly, s);
                const uint64_t cz = icoord(pos[3 * i + 2], lz, s);
                k = (1ull << 63) | (spread3(cx) << 2) | (spread3(cy) << 1) | spread3(cz);
                key[i] = k;
                idx[i] = (uint32_t)i;
            }
            const unsigned vm = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                // a warp whose keys share the digit (the high digits of spatially ordered input)
                // adds once; otherwise every lane adds its own
                const unsigned d = valid ? (unsigned)(k >> (8 * p)) & 255u : 256u;
                const unsigned d0 = __shfl_sync(0xffffffffu, d, 0);
                if (__all_sync(0xffffffffu, d == d0 || !valid)) {
                    if (lane == 0 && vm) {
                        atomicAdd(&h[p][d0], (unsigned)__popc(vm));
                        if (p == 0 && thist0) atomicAdd(&h0[d0], (unsigned)__popc(vm));
                    }
                } else if (valid) {
                    atomicAdd(&h[p][d], 1u);
                    if (p == 0 && thist0) atomicAdd(&h0[d], 1u);
                }
            }
        }
        if (thist0) {
            __syncthreads();
            thist0[(int64_t)threadIdx.x * ntiles + t] = h0[threadIdx.x];
            h0[threadIdx.x] = 0;
            __syncthreads();
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) bhist[(int64_t)blockIdx.x * 2048 + k] = h[k >> 8][k & 255];
}

// The digit histograms of the first npass passes of existing keys (one per block, as in
// k_keys_hist), for hot_sort_pairs.
__global__ void __launch_bounds__(256) k_rs_hist_all(const uint64_t *__restrict__ key, int64_t n, int npass,
                                                     uint32_t *__restrict__ bhist)
{
    __shared__ uint32_t h[8][256];
    for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) h[k >> 8][k & 255] = 0;
    __syncthreads();
    const unsigned lane = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; w0 < n; w0 += nw * 32) {
        const int64_t i = w0 + lane;
        const bool valid = i < n;
        const uint64_t k = valid ? key[i] : 0ull;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        for (int p = 0; p < npass; ++p) {
            const unsigned d = valid ? (unsigned)(k >> (8 * p)) & 255u : 256u;
            const unsigned d0 = __shfl_sync(0xffffffffu, d, 0);
            if (__all_sync(0xffffffffu, d == d0 || !valid)) {
                if (lane == 0) atomicAdd(&h[p][d0], (unsigned)__popc(vm));
            } else if (valid) {
                atomicAdd(&h[p][d], 1u);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) bhist[(int64_t)blockIdx.x * 2048 + k] = h[k >> 8][k & 255];
}

// Block p: digit totals of pass p over the nb block histograms, scanned into goff[p][d].
// 1024 threads: thread (g, d) sums the histograms g, g + 4, ... of digit d (integer sums: the
// order is free).
__global__ void __launch_bounds__(1024) k_rs_goff(const uint32_t *__restrict__ bhist, int nb,
                                                  uint32_t *__restrict__ goff)
{
    __shared__ uint32_t ws[8], part[4][256];
    const int p = blockIdx.x, d = threadIdx.x & 255, g = threadIdx.x >> 8;
    uint32_t t0 = 0, t1 = 0;
    int b = g;
    for (; b + 4 < nb; b += 8) {
        t0 += bhist[(int64_t)b * 2048 + p * 256 + d];
        t1 += bhist[(int64_t)(b + 4) * 2048 + p * 256 + d];
    }
    if (b < nb) t0 += bhist[(int64_t)b * 2048 + p * 256 + d];
    part[g][d] = t0 + t1;
    __syncthreads();
    const uint32_t t = part[0][d] + part[1][d] + part[2][d] + part[3][d];
    const uint32_t inc = warp_incl_scan(t);
    if (g == 0 && lane_id() == 31) ws[d >> 5] = inc;
    __syncthreads();
    if (g != 0) return;
    uint32_t base = 0;
    for (int w = 0; w < (d >> 5); ++w) base += ws[w];
    goff[p * 256 + d] = base + inc - t;
}

// Digit counts of every tile of one pass (the tiles of k_rs_pass), digit-major:
// thist[d * ntiles + tile].
template <int RT>
__global__ void __launch_bounds__(256) k_rs_count(const uint64_t *__restrict__ kin, int64_t N, int shift,
                                                  int64_t ntiles, uint32_t *__restrict__ thist)
{
    constexpr int TILE = OsTile<RT>::TILE;
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * TILE;
    const unsigned lane = lane_id();
    constexpr int R = TILE / 256;
    uint64_t kk[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = t0 + r * 256 + threadIdx.x;
        kk[r] = i < N ? kin[i] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = t0 + r * 256 + threadIdx.x;
        const bool valid = i < N;
        const unsigned d = valid ? (unsigned)(kk[r] >> shift) & 255u : 256u;
        // a warp whose keys share the digit adds once; otherwise every lane adds its own
        const unsigned d0 = __shfl_sync(0xffffffffu, d, 0);
        if (__all_sync(0xffffffffu, d == d0)) {
            if (lane == 0 && d0 < 256u) atomicAdd(&h[d0], 32u);
        } else if (valid) {
            atomicAdd(&h[d], 1u);
        }
    }
    __syncthreads();
    thist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Block d: exclusive scan of digit d's tile counts, in place, plus the pass's global
// offset of d: thist[d * ntiles + tile] becomes the first output slot of the tile's keys
// of digit d.
constexpr int TS_T = 1024, TS_Q = 8, TS_CH = TS_T * TS_Q;  // threads, counts per thread, per chunk
__device__ __forceinline__ int ts_pad(int i) { return i + (i >> 5); }
__global__ void __launch_bounds__(TS_T) k_rs_tscan(uint32_t *__restrict__ thist, int64_t ntiles,
                                                   const uint32_t *__restrict__ goff)
{
    // a chunk of the row is loaded and stored coalesced through shared memory; each
    // thread scans TS_Q consecutive counts
    __shared__ uint32_t sm[TS_CH + TS_CH / 32];
    __shared__ uint32_t ws[TS_T / 32];
    const int d = blockIdx.x;
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    uint32_t *row = thist + (int64_t)d * ntiles;
    uint32_t carry = goff[d];
    for (int64_t c0 = 0; c0 < ntiles; c0 += TS_CH) {
#pragma unroll
        for (int q = 0; q < TS_Q; ++q) {
            const int k = q * TS_T + threadIdx.x;
            sm[ts_pad(k)] = c0 + k < ntiles ? row[c0 + k] : 0u;
        }
        __syncthreads();
        uint32_t v[TS_Q];
        uint32_t sum = 0;
#pragma unroll
        for (int q = 0; q < TS_Q; ++q) {
            v[q] = sm[ts_pad(threadIdx.x * TS_Q + q)];
            sum += v[q];
        }
        const uint32_t inc = warp_incl_scan(sum);
        if (lane == 31) ws[w] = inc;
        __syncthreads();
        if (w == 0) ws[lane] = warp_incl_scan(ws[lane]);  // TS_T / 32 == 32 warp totals
        __syncthreads();
        uint32_t off = carry + inc - sum + (w > 0 ? ws[w - 1] : 0u);
#pragma unroll
        for (int q = 0; q < TS_Q; ++q) {
            sm[ts_pad(threadIdx.x * TS_Q + q)] = off;
            off += v[q];
        }
        carry += ws[TS_T / 32 - 1];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TS_Q; ++q) {
            const int k = q * TS_T + threadIdx.x;
            if (c0 + k < ntiles) row[c0 + k] = sm[ts_pad(k)];
        }
        __syncthreads();
    }
}

// LB = true: one launch per pass, the tiles' offsets found by the decoupled look-back over
// pub (tiles numbered in the order their blocks start); LB = false: the offsets come
// scanned in pub (k_rs_count, k_rs_tscan) and tile = block index.
template <bool LB, int OS_R>
__global__ void __launch_bounds__(OS_W * 32, OS_R <= 8 ? 4 : 2) k_rs_pass(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t N, int shift, const uint32_t *__restrict__ goff, uint32_t *tile_ctr,
    uint32_t *pub, int64_t ntiles, unsigned *status)
{
    constexpr int OS_TILE = OsTile<OS_R>::TILE;
    extern __shared__ __align__(16) unsigned char os_smem[];
    uint64_t *sk = (uint64_t *)os_smem;                                 // [OS_TILE]
    uint32_t *sv = (uint32_t *)(sk + OS_TILE);                          // [OS_TILE]
    uint32_t(*wcnt)[256] = (uint32_t(*)[256])(sv + OS_TILE);            // [OS_W][256]
    uint32_t *toff = (uint32_t *)(wcnt + OS_W);                         // [256] tile-local digit offsets
    uint32_t *gbase = toff + 256;                                       // [256] global first slot
    __shared__ uint32_t s_tile, ws[OS_W];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    if (LB && threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int k = lane; k < 256; k += 32) wcnt[w][k] = 0;
    __syncthreads();
    const int64_t tile = LB ? (int64_t)s_tile : (int64_t)blockIdx.x;
    // counted tiles: the tile's first slot of digit threadIdx.x, loaded beside the keys
    uint32_t gscan = 0;
    if constexpr (!LB) gscan = pub[(int64_t)threadIdx.x * ntiles + tile];
    const int64_t base = tile * OS_TILE + (int64_t)w * (OS_R * 32);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t kk[OS_R];
    uint32_t vv[OS_R];
    uint32_t rk[OS_R];
    // every load of the tile first, so that they are all in flight together (the ranking
    // below orders its rounds through shared memory)
#pragma unroll
    for (int r = 0; r < OS_R; ++r) {
        const int64_t i = base + r * 32 + lane;
        kk[r] = i < N ? kin[i] : 0ull;
        vv[r] = i < N ? vin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < OS_R; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < N;
        const uint64_t k = kk[r];
        const unsigned d = valid ? ((unsigned)(k >> shift) & 255u) : 256u;
        // lanes with the same digit: one ballot per digit bit and one for validity (at 256^3
        // 1.6x faster than __match_any_sync, whose latency stalled the ranking rounds)
        const unsigned vb = __ballot_sync(0xffffffffu, valid);
        unsigned peers = valid ? vb : ~vb;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const bool bit = (d >> q) & 1u;
            const unsigned bq = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bq : ~bq;
        }
        const unsigned rank = __popc(peers & lt);
        const uint32_t b = valid ? wcnt[w][d] : 0u;
        __syncwarp();
        if (valid && rank == 0) wcnt[w][d] = b + __popc(peers);
        __syncwarp();
        rk[r] = valid ? b + rank : 0xffffffffu;
    }
    __syncthreads();
    // thread d: per-warp offsets of digit d within the tile, and the tile's count of d
    const unsigned d = threadIdx.x;
    uint32_t tot = 0;
    for (int ww = 0; ww < OS_W; ++ww) {
        const uint32_t c = wcnt[ww][d];
        wcnt[ww][d] = tot;
        tot += c;
    }
    uint32_t *my = pub + tile * 256 + d;
    if constexpr (!LB) {
        gbase[d] = gscan;
    } else if (tile == 0) {
        atomicExch(my, os_pack(OS_FLAG_INC, tot));
        gbase[d] = goff[d];
    } else {
        atomicExch(my, os_pack(OS_FLAG_AGG, tot));
        uint64_t excl = 0;
        int64_t t = tile - 1;  // the nearest earlier tile not yet added
        long polls = 0;
        bool done = false;
        while (!done) {
            // the words of tiles t, t-1, ..., t-OS_LB+1 (as far as tile 0), read together
            uint32_t v[OS_LB];
#pragma unroll
            for (int k = 0; k < OS_LB; ++k) v[k] = t - k >= 0 ? *((volatile uint32_t *)(pub + (t - k) * 256 + d)) : 0u;
            // add the words in order up to the first inclusive one, stopping at the first
            // not yet written (unrolled and predicated, so that v stays in registers)
            int k = 0;
            bool stop = false;
#pragma unroll
            for (int q = 0; q < OS_LB; ++q) {
                if (!stop && !done) {
                    if (t - q < 0 || (v[q] >> 30) == 0u) {
                        stop = true;
                    } else {
                        excl += v[q] & 0x3fffffffu;
                        k = q + 1;
                        if ((v[q] >> 30) == OS_FLAG_INC || t - q == 0) done = true;
                    }
                }
            }
            if (done) break;
            if (k > 0) {
                t -= k;  // every word read up to k was an aggregate: continue below it
                continue;
            }
            if (++polls > OS_POLL_LIMIT) {
                hot_flag(status, HOT_ST_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
        atomicExch(my, os_pack(OS_FLAG_INC, (uint32_t)(excl + tot)));
        gbase[d] = goff[d] + (uint32_t)excl;
    }
    // tile-local exclusive scan of the digit counts
    const uint32_t inc = warp_incl_scan(tot);
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    uint32_t off = 0;
    for (int ww = 0; ww < w; ++ww) off += ws[ww];
    toff[d] = off + inc - tot;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < OS_R; ++r) {
        if (rk[r] == 0xffffffffu) continue;
        const unsigned dd = (unsigned)(kk[r] >> shift) & 255u;
        const uint32_t lp = toff[dd] + wcnt[w][dd] + rk[r];
        sk[lp] = kk[r];
        sv[lp] = vv[r];
    }
    __syncthreads();
    const int64_t t0 = tile * OS_TILE;
    const int n = (int)(N - t0 < OS_TILE ? N - t0 : OS_TILE);
    for (int i = threadIdx.x; i < n; i += OS_W * 32) {
        const uint64_t k = sk[i];
        const unsigned dd = (unsigned)(k >> shift) & 255u;
        const int64_t dst = (int64_t)gbase[dd] + (i - (int64_t)toff[dd]);
        if (dst < 0 || dst >= N) {  // only after a look-back gave up: never store out of range
            hot_flag(status, HOT_ST_INTERNAL);
            continue;
        }
        kout[dst] = k;
        vout[dst] = sv[i];
    }
}

__global__ void k_gather(const double *__restrict__ pos, const double *__restrict__ mass,
                         const uint32_t *__restrict__ idx, int64_t N, double *__restrict__ spos,
                         double *__restrict__ smass)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    uint32_t i = idx[s];
    spos[3 * s + 0] = pos[3 * (int64_t)i + 0];
    spos[3 * s + 1] = pos[3 * (int64_t)i + 1];
    spos[3 * s + 2] = pos[3 * (int64_t)i + 2];
    smass[s] = mass[i];
}

// ---------------------------------------------------------------------------
// Tree
// ---------------------------------------------------------------------------
// lcp[i] = lcp(key_{i-1}, key_i) (255 for i = 0); win[t] = lcp(key_t, key_{t+leaf_max}).
__global__ void k_lcp(const uint64_t *__restrict__ key, int64_t N, int leaf_max,
                      uint8_t *__restrict__ lcp, uint8_t *__restrict__ win)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint64_t k = key[i];
    lcp[i] = i == 0 ? 255 : (uint8_t)key_lcp_levels(key[i - 1], k);
    win[i] = (i + leaf_max < N) ? (uint8_t)key_lcp_levels(k, key[i + leaf_max]) : 0;
}

__global__ void k_leaflevel(const uint8_t *__restrict__ lcp, const uint8_t *__restrict__ win,
                            int64_t N, int leaf_max, uint8_t *__restrict__ leaflev,
                            uint32_t *__restrict__ ncell_i, int64_t *__restrict__ maxlev)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ll = 0;
    if (i < N) {
        int64_t t0 = i - leaf_max > 0 ? i - leaf_max : 0;
        int64_t t1 = i < N - 1 - leaf_max ? i : N - 1 - leaf_max;
        int dmax = -1;
        for (int64_t t = t0; t <= t1; ++t) dmax = max(dmax, (int)win[t]);
        ll = min(HOT_MAXLEVEL, dmax + 1);
        leaflev[i] = (uint8_t)ll;
        int d = (i == 0) ? -1 : (int)lcp[i];
        ncell_i[i] = ll > d ? (uint32_t)(ll - d) : 0u;
    }
    int m = warp_max(ll);
    if (lane_id() == 0 && m > 0) atomicMax((unsigned long long *)maxlev, (unsigned long long)m);
}

// First j in (i, N] whose key differs from key_i in the first `lev` digits.
__device__ int64_t run_end(const uint64_t *__restrict__ key, int64_t N, int64_t i, int lev)
{
    const uint64_t ki = key[i];
    int64_t lo = i, step = 1, hi;
    // gallop
    for (;;) {
        int64_t j = i + step;
        if (j >= N) {
            hi = N;
            break;
        }
        if (key_lcp_levels(ki, key[j]) < lev) {
            hi = j;
            break;
        }
        lo = j;
        step <<= 1;
    }
    // invariant: key[lo] shares the prefix, hi is the first known non-sharer (or N)
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (key_lcp_levels(ki, key[mid]) >= lev)
            lo = mid;
        else
            hi = mid;
    }
    return hi;
}

// First t in [0, i] whose key shares the first `lev` digits with key_i.
__device__ int64_t run_start(const uint64_t *__restrict__ key, int64_t i, int lev)
{
    const uint64_t ki = key[i];
    int64_t hi = i, step = 1, lo;
    for (;;) {
        int64_t j = i - step;
        if (j < 0) {
            lo = -1;
            break;
        }
        if (key_lcp_levels(ki, key[j]) < lev) {
            lo = j;
            break;
        }
        hi = j;
        step <<= 1;
    }
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (key_lcp_levels(ki, key[mid]) >= lev)
            hi = mid;
        else
            lo = mid;
    }
    return hi;
}

__global__ void k_cells(const uint64_t *__restrict__ key, int64_t N, const uint8_t *__restrict__ lcp,
                        const uint8_t *__restrict__ leaflev, const uint32_t *__restrict__ off,
                        int64_t ncell, uint64_t *__restrict__ ckey, int32_t *__restrict__ clevel,
                        int32_t *__restrict__ cbegin, int32_t *__restrict__ ccount,
                        int32_t *__restrict__ cparent, int32_t *__restrict__ cend,
                        unsigned *status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int d = (i == 0) ? -1 : (int)lcp[i];
    int ll = leaflev[i];
    if (ll <= d) return;
    const uint64_t ki = key[i];
    int64_t c0 = off[i];
    for (int lev = d + 1; lev <= ll; ++lev) {
        int64_t c = c0 + (lev - d - 1);
        if (c >= ncell) {
            hot_flag(status, HOT_ST_INTERNAL);
            return;
        }
        ckey[c] = ki >> (3 * (HOT_MAXLEVEL - lev));
        clevel[c] = lev;
        cbegin[c] = (int32_t)i;
        int64_t e = run_end(key, N, i, lev);
        ccount[c] = (int32_t)(e - i);
        cend[c] = (int32_t)(e < N ? (int64_t)off[e] : ncell);
        if (lev == 0) {
            cparent[c] = -1;
        } else if (lev > d + 1) {
            cparent[c] = (int32_t)(c - 1);
        } else {
            // parent: the level-(lev-1) cell holding i, owned by the first particle t of that run
            int64_t t = run_start(key, i, lev - 1);
            int dt = (t == 0) ? -1 : (int)lcp[t];
            cparent[c] = (int32_t)((int64_t)off[t] + (lev - 1 - dt - 1));
        }
    }
}

__global__ void k_link(const uint64_t *__restrict__ ckey, const int32_t *__restrict__ cparent,
                       const int32_t *__restrict__ clevel, int64_t ncell, int32_t *__restrict__ child8,
                       int32_t *__restrict__ cnchild, int32_t *__restrict__ lvlcnt)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    atomicAdd(&lvlcnt[clevel[c]], 1);
    int32_t p = cparent[c];
    if (p < 0) return;
    child8[8 * (int64_t)p + (int)(ckey[c] & 7u)] = (int32_t)c;
    atomicAdd(&cnchild[p], 1);
}

// level offsets (exclusive scan of 22 counts) on one thread, then scatter.
__global__ void k_level_off(int32_t *lvlcnt, int64_t *levoff, int64_t *sizes)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t run = 0;
    for (int l = 0; l <= HOT_MAXLEVEL; ++l) {
        levoff[l] = run;
        run += lvlcnt[l];
        lvlcnt[l] = 0;  // reused as cursor
    }
    levoff[HOT_MAXLEVEL + 1] = run;
    (void)sizes;
}

__global__ void k_level_scatter(const int32_t *__restrict__ clevel, int64_t ncell,
                                const int64_t *__restrict__ levoff, int32_t *cursor,
                                int32_t *__restrict__ level_cells)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int l = clevel[c];
    int32_t k = atomicAdd(&cursor[l], 1);
    level_cells[levoff[l] + k] = (int32_t)c;
}

__device__ __forceinline__ uint64_t hash64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__global__ void k_hash_insert(const uint64_t *__restrict__ ckey, int64_t ncell, uint64_t *hkey,
                              int32_t *hval, uint64_t mask, unsigned *status)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    uint64_t k = ckey[c];
    uint64_t h = hash64(k) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        unsigned long long prev =
            atomicCAS((unsigned long long *)&hkey[h], 0ull, (unsigned long long)k);
        if (prev == 0ull || prev == k) {
            hval[h] = (int32_t)c;
            return;
        }
        h = (h + 1) & mask;
    }
    hot_flag(status, HOT_ST_HASH);
}

__global__ void k_hash_lookup(const uint64_t *__restrict__ q, int64_t n, const uint64_t *__restrict__ hkey,
                              const int32_t *__restrict__ hval, uint64_t mask, int32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = q[i];
    int32_t r = -1;
    if (k != 0ull) {
        uint64_t h = hash64(k) & mask;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
            uint64_t s = hkey[h];
            if (s == k) {
                r = hval[h];
                break;
            }
            if (s == 0ull) break;
            h = (h + 1) & mask;
        }
    }
    out[i] = r;
}

// Sink groups: topmost cells that are leaves or hold <= group_max particles.
__global__ void k_group_flag(const int32_t *__restrict__ ccount, const int32_t *__restrict__ cparent,
                             const int32_t *__restrict__ cnchild, int64_t ncell, int group_max,
                             uint32_t *__restrict__ flag, int64_t *__restrict__ nleaf)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool leaf = false;
    if (c < ncell) {
        leaf = cnchild[c] == 0;
        bool small = leaf || ccount[c] <= group_max;
        int32_t p = cparent[c];
        bool top = p < 0 || ccount[p] > group_max;
        flag[c] = (small && top) ? 1u : 0u;
    }
    unsigned b = __ballot_sync(0xffffffffu, leaf);
    if (lane_id() == 0 && b) atomicAdd((unsigned long long *)nleaf, (unsigned long long)__popc(b));
}

__global__ void k_group_write(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ goff,
                              int64_t ncell, int32_t *__restrict__ gcell)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    if (flag[c]) gcell[goff[c]] = (int32_t)c;
}

// Group centre = centre of the sinks' bounding box; Delta_max = max |x - g|, evaluated
// with explicit roundings ((dx*dx + dy*dy) + dz*dz, no contraction, IEEE sqrt).
__global__ void k_group_geom(const int32_t *__restrict__ gcell, const uint32_t *__restrict__ ngroup_p,
                             const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount,
                             const double *__restrict__ spos, double *__restrict__ gcen,
                             double *__restrict__ gdmax)
{
    int64_t ngroup = *ngroup_p;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    // min and max on the order-preserving integer images of the coordinates and on the bit
    // patterns of the non-negative squared distances: exact, and off the float64 pipe
    auto wmin = [](unsigned long long v) {
        for (int o = 16; o > 0; o >>= 1) v = umin64(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    };
    auto wmax = [](unsigned long long v) {
        for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    };
    for (int64_t g = warp; g < ngroup; g += nw) {
        int32_t c = gcell[g];
        int64_t b = cbegin[c], n = ccount[c];
        unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
        for (int64_t s = b + lane; s < b + n; s += 32)
            for (int d = 0; d < 3; ++d) {
                const unsigned long long x = ord_image(spos[3 * s + d]);
                lo[d] = umin64(lo[d], x);
                hi[d] = umax64(hi[d], x);
            }
        double cen[3];
        for (int d = 0; d < 3; ++d) cen[d] = __dmul_rn(__dadd_rn(ord_value(wmin(lo[d])), ord_value(wmax(hi[d]))), 0.5);
        unsigned long long r2m = 0ull;
        for (int64_t s = b + lane; s < b + n; s += 32) {
            double dx = __dsub_rn(spos[3 * s + 0], cen[0]);
            double dy = __dsub_rn(spos[3 * s + 1], cen[1]);
            double dz = __dsub_rn(spos[3 * s + 2], cen[2]);
            double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            r2m = umax64(r2m, (unsigned long long)__double_as_longlong(r2));
        }
        const double r2max = __longlong_as_double((long long)wmax(r2m));
        if (lane == 0) {
            for (int d = 0; d < 3; ++d) gcen[3 * g + d] = cen[d];
            gdmax[g] = __dsqrt_rn(r2max);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
// The passes of a sort of n pairs.  Up to OS_SCAN_TILES tiles of 4096 keys a pass is one
// launch (decoupled look-back: the chain of dependent reads stays short); above, the
// tiles' digit counts are counted and scanned first (three launches a pass, no tile waits
// for another): both give every key the same slot.
constexpr int64_t OS_SCAN_TILES = 1024;

static bool rs_scan(int64_t n) { return (n + OsTile<OS_R_LB>::TILE - 1) / OsTile<OS_R_LB>::TILE > OS_SCAN_TILES; }

static int64_t rs_ntiles(int64_t n)
{
    const int64_t t = rs_scan(n) ? OsTile<OS_R_SCAN>::TILE : OsTile<OS_R_LB>::TILE;
    return (n + t - 1) / t;
}

static cudaError_t rs_prepare(hot_ctx *c, int passes, int64_t n)
{
    cudaStream_t s = c->st;
    cudaError_t e;
    const int64_t ntiles = rs_ntiles(n);
    if (rs_scan(n)) return c->rs_status.ensure(256 * (size_t)ntiles, s);
    // every pass's published words, cleared once
    if ((e = c->rs_ctr.ensure(8, s)) != cudaSuccess) return e;
    if ((e = c->rs_status.ensure((size_t)passes * 256 * (size_t)ntiles, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->rs_status.p, 0, sizeof(uint32_t) * passes * 256 * (size_t)ntiles, s)) != cudaSuccess)
        return e;
    return cudaMemsetAsync(c->rs_ctr.p, 0, 8 * sizeof(uint32_t), s);
}

// Passes 0..passes-1 from (ka, va), alternating with (kb, vb): the result is in (ka, va)
// for an even number of passes, in (kb, vb) for an odd one.  counted0: the first pass's
// tile counts are already in rs_status (k_keys_hist).
static cudaError_t rs_passes(hot_ctx *c, uint64_t *ka, uint32_t *va, uint64_t *kb, uint32_t *vb, int64_t n, int passes,
                             bool counted0 = false)
{
    cudaStream_t s = c->st;
    const bool scan = rs_scan(n);
    const int64_t ntiles = rs_ntiles(n);
    constexpr int SM_LB = OsTile<OS_R_LB>::SMEM, SM_SCAN = OsTile<OS_R_SCAN>::SMEM;
    cudaError_t e = scan ? cudaFuncSetAttribute(k_rs_pass<false, OS_R_SCAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_SCAN)
                         : cudaFuncSetAttribute(k_rs_pass<true, OS_R_LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_LB);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < passes; ++pass) {
        if (scan) {
            if (pass > 0 || !counted0) {
                HOT_COUNT_LAUNCH();
                k_rs_count<OS_R_SCAN><<<(unsigned)ntiles, 256, 0, s>>>(ka, n, 8 * pass, ntiles, c->rs_status.p);
            }
            HOT_COUNT_LAUNCH();
            k_rs_tscan<<<256, TS_T, 0, s>>>(c->rs_status.p, ntiles, c->rs_goff.p + 256 * pass);
            HOT_COUNT_LAUNCH();
            k_rs_pass<false, OS_R_SCAN><<<(unsigned)ntiles, OS_W * 32, SM_SCAN, s>>>(
                ka, va, kb, vb, n, 8 * pass, c->rs_goff.p + 256 * pass, nullptr, c->rs_status.p, ntiles, c->d_status);
        } else {
            HOT_COUNT_LAUNCH();
            k_rs_pass<true, OS_R_LB><<<(unsigned)ntiles, OS_W * 32, SM_LB, s>>>(
                ka, va, kb, vb, n, 8 * pass, c->rs_goff.p + 256 * pass, c->rs_ctr.p + pass,
                c->rs_status.p + (size_t)pass * 256 * ntiles, ntiles, c->d_status);
        }
        uint64_t *tk = ka;
        ka = kb;
        kb = tk;
        uint32_t *tv = va;
        va = vb;
        vb = tv;
    }
    return cudaGetLastError();
}

int hot_impl_build(hot_ctx *c, const double *pos, const double *mass, int64_t N)
{
    cudaStream_t s = c->st;
    const int leaf_max = c->prm.leaf_max;
    c->N = N;
    c->stage = 0;
    hot_tic(c, 0);
    // bbox + keys
    int nbb = c->nsm * 4;
    HOT_CK(c->part.ensure(6 * (size_t)nbb, s));
    HOT_CK(c->frame.ensure(8, s));
    HOT_CK(c->key.ensure(N, s));
    HOT_CK(c->key2.ensure(N, s));
    HOT_CK(c->idx.ensure(N, s));
    HOT_CK(c->idx2.ensure(N, s));
    HOT_COUNT_LAUNCH();
    k_bbox_part<<<nbb, BT, 0, s>>>(pos, mass, N, c->part.p, c->d_status);
    HOT_COUNT_LAUNCH();
    k_bbox_final<<<1, BF, 0, s>>>(c->part.p, nbb, c->frame.p);
    // keys with the digit histograms of every pass, then the passes' global offsets
    const int nkb = c->nsm * 4;
    HOT_CK(c->rs_bhist.ensure(2048 * (size_t)nkb, s));
    HOT_CK(c->rs_goff.ensure(2048, s));
    HOT_CK(rs_prepare(c, 8, N));
    HOT_COUNT_LAUNCH();
    k_keys_hist<OsTile<OS_R_SCAN>::TILE><<<nkb, 256, 0, s>>>(pos, N, c->frame.p, c->key.p, c->idx.p, c->rs_bhist.p,
                                                             rs_scan(N) ? c->rs_status.p : nullptr);
    HOT_COUNT_LAUNCH();
    k_rs_goff<<<8, 1024, 0, s>>>(c->rs_bhist.p, nkb, c->rs_goff.p);
    HOT_CK(rs_passes(c, c->key.p, c->idx.p, c->key2.p, c->idx2.p, N, 8, true));
    HOT_CK(c->scan_tmp.ensure(hot_scan_tmp_elems(N + 64), s));
    // 8 passes: sorted data is back in key/idx
    HOT_CK(c->spos.ensure(3 * (size_t)N, s));
    HOT_CK(c->smass.ensure(N, s));
    HOT_COUNT_LAUNCH();
    k_gather<<<hot_blocks(N, BT), BT, 0, s>>>(pos, mass, c->idx.p, N, c->spos.p, c->smass.p);
    hot_toc(c, 0);

    hot_tic(c, 1);
    HOT_CK(c->lcp.ensure(N, s));
    HOT_CK(c->leaflev.ensure(N, s));
    HOT_CK(c->ncell_i.ensure(N + 1, s));
    HOT_CK(c->cell_off.ensure(N + 1, s));
    HOT_CK(c->sizes.ensure(64, s));
    HOT_CK(cudaMemsetAsync(c->sizes.p, 0, 64 * sizeof(int64_t), s));
    uint8_t *win = (uint8_t *)c->key2.p;  // scratch: key2 is free after the sort
    HOT_COUNT_LAUNCH();
    k_lcp<<<hot_blocks(N, BT), BT, 0, s>>>(c->key.p, N, leaf_max, c->lcp.p, win);
    HOT_COUNT_LAUNCH();
    k_leaflevel<<<hot_blocks(N, BT), BT, 0, s>>>(c->lcp.p, win, N, leaf_max, c->leaflev.p, c->ncell_i.p,
                                                   c->sizes.p + 0);
    int r = hot_scan_u32_to_u32(c->ncell_i.p, c->cell_off.p, N, c->scan_tmp.p, s);
    if (r) return r;
    // sizes[1] = ncell (cell_off[N])
    HOT_CK(cudaMemcpyAsync(c->sizes.p + 1, c->cell_off.p + N, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    int64_t hs[2] = {0, 0};
    HOT_CK(cudaMemcpyAsync(hs, c->sizes.p, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HOT_CK(cudaStreamSynchronize(s));
    {
        int e = hot_sync_status(c);
        if (e) return e;
    }
    c->maxlevel = hs[0];
    int64_t ncell = (int64_t)(uint32_t)hs[1];
    c->ncell = ncell;
    HOT_CK(c->ckey.ensure(ncell, s));
    HOT_CK(c->clevel.ensure(ncell, s));
    HOT_CK(c->cbegin.ensure(ncell, s));
    HOT_CK(c->ccount.ensure(ncell, s));
    HOT_CK(c->cparent.ensure(ncell, s));
    HOT_CK(c->cend.ensure(ncell, s));
    HOT_CK(c->child8.ensure(8 * (size_t)ncell, s));
    HOT_CK(c->cnchild.ensure(ncell, s));
    HOT_CK(c->level_cells.ensure(ncell, s));
    HOT_CK(c->gflag.ensure(ncell + 1, s));
    HOT_CK(c->goff.ensure(ncell + 1, s));
    HOT_CK(c->gcell.ensure(ncell, s));
    HOT_CK(c->scan_tmp.ensure(hot_scan_tmp_elems(ncell + N + 64), s));
    HOT_COUNT_LAUNCH();
    k_cells<<<hot_blocks(N, BT), BT, 0, s>>>(c->key.p, N, c->lcp.p, c->leaflev.p, c->cell_off.p, ncell,
                                              c->ckey.p, c->clevel.p, c->cbegin.p, c->ccount.p, c->cparent.p,
                                              c->cend.p, c->d_status);
    HOT_CK(cudaMemsetAsync(c->child8.p, 0xff, 8 * sizeof(int32_t) * (size_t)ncell, s));
    HOT_CK(cudaMemsetAsync(c->cnchild.p, 0, sizeof(int32_t) * (size_t)ncell, s));
    int32_t *lvlcnt = (int32_t *)(c->sizes.p + 8);     // 24 int32 in sizes[8..20)
    int64_t *levoff = c->sizes.p + 24;                 // 23 int64 in sizes[24..47)
    HOT_COUNT_LAUNCH();
    k_link<<<hot_blocks(ncell, BT), BT, 0, s>>>(c->ckey.p, c->cparent.p, c->clevel.p, ncell, c->child8.p,
                                                 c->cnchild.p, lvlcnt);
    HOT_COUNT_LAUNCH();
    k_level_off<<<1, 32, 0, s>>>(lvlcnt, levoff, c->sizes.p);
    HOT_COUNT_LAUNCH();
    k_level_scatter<<<hot_blocks(ncell, BT), BT, 0, s>>>(c->clevel.p, ncell, levoff, lvlcnt, c->level_cells.p);
    // hash table, load <= 1/2
    uint64_t hcap = 1024;
    while (hcap < 2 * (uint64_t)ncell) hcap <<= 1;
    c->hcap = hcap;
    HOT_CK(c->hkey.ensure(hcap, s));
    HOT_CK(c->hval.ensure(hcap, s));
    HOT_CK(cudaMemsetAsync(c->hkey.p, 0, sizeof(uint64_t) * hcap, s));
    HOT_COUNT_LAUNCH();
    k_hash_insert<<<hot_blocks(ncell, BT), BT, 0, s>>>(c->ckey.p, ncell, c->hkey.p, c->hval.p, hcap - 1,
                                                        c->d_status);
    // groups
    HOT_COUNT_LAUNCH();
    k_group_flag<<<hot_blocks(ncell, BT), BT, 0, s>>>(c->ccount.p, c->cparent.p, c->cnchild.p, ncell,
                                                       c->prm.group_max, c->gflag.p, c->sizes.p + 2);
    r = hot_scan_u32_to_u32(c->gflag.p, c->goff.p, ncell, c->scan_tmp.p, s);
    if (r) return r;
    HOT_COUNT_LAUNCH();
    k_group_write<<<hot_blocks(ncell, BT), BT, 0, s>>>(c->gflag.p, c->goff.p, ncell, c->gcell.p);
    HOT_CK(c->gcen.ensure(3 * (size_t)ncell, s));
    HOT_CK(c->gdmax.ensure(ncell, s));
    HOT_COUNT_LAUNCH();
    k_group_geom<<<c->nsm * 8, 256, 0, s>>>(c->gcell.p, c->goff.p + ncell, c->cbegin.p, c->ccount.p,
                                             c->spos.p, c->gcen.p, c->gdmax.p);
    HOT_CK(cudaMemcpyAsync(c->sizes.p + 3, c->goff.p + ncell, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    hot_toc(c, 1);
    int64_t hs2[48];
    HOT_CK(cudaMemcpyAsync(hs2, c->sizes.p, 48 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HOT_CK(cudaStreamSynchronize(s));
    {
        int e = hot_sync_status(c);
        if (e) return e;
    }
    c->nleaf = hs2[2];
    c->ngroup = (int64_t)(uint32_t)hs2[3];
    c->level_off.assign(HOT_MAXLEVEL + 2, 0);
    for (int l = 0; l <= HOT_MAXLEVEL + 1; ++l) c->level_off[l] = hs2[24 + l];
    c->stage = 1;
    return HOT_OK;
}

int hot_impl_lookup(hot_ctx *c, const uint64_t *keys, int64_t n, int32_t *idx)
{
    cudaStream_t s = c->st;
    uint64_t *dk = nullptr;
    int32_t *di = nullptr;
    HOT_CK(cudaMallocAsync((void **)&dk, sizeof(uint64_t) * (n > 0 ? n : 1), s));
    HOT_CK(cudaMallocAsync((void **)&di, sizeof(int32_t) * (n > 0 ? n : 1), s));
    HOT_CK(cudaMemcpyAsync(dk, keys, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s));
    HOT_COUNT_LAUNCH();
    k_hash_lookup<<<hot_blocks(n, BT), BT, 0, s>>>(dk, n, c->hkey.p, c->hval.p, c->hcap - 1, di);
    HOT_CK(cudaMemcpyAsync(idx, di, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(dk, s);
    cudaFreeAsync(di, s);
    HOT_CK(cudaStreamSynchronize(s));
    return HOT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the bounding-cube reduction (see hot_key_frame_noalloc
// in include/hot.h).  Its scratch -- one partial min/max record per block, the
// frame record written by the final reduction and the status word -- lives in this
// file-scope device array, which every GPU that loads the library keeps until exit.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int64_t NOALLOC_PER_BLOCK = (int64_t)BT * 64;  // particles per reduction block
constexpr int NOALLOC_MAX_BLOCKS = 4096;                // => at most 2^26 particles
constexpr int NOALLOC_DOUBLES = 6 * NOALLOC_MAX_BLOCKS + 8 + 1;  // partials, frame, status

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is queried once per device with
// that device current, and reused afterwards.
int noalloc_scratch(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HOT_ECUDA;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return HOT_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        double *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_noalloc_scratch) != cudaSuccess || !p) return HOT_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return HOT_OK;
}

}  // namespace

extern "C" int hot_key_frame_noalloc(const double *pos, const double *mass, int64_t N, double *frame,
                                     void *cuda_stream)
{
    if (!pos || !mass || !frame || N < 1) return HOT_EINVAL;
    if (N > NOALLOC_PER_BLOCK * NOALLOC_MAX_BLOCKS) return HOT_EOVERFLOW;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *scratch = nullptr;
    int e = noalloc_scratch(&scratch);
    if (e) return e;
    double *part = scratch;
    double *fr = scratch + 6 * NOALLOC_MAX_BLOCKS;
    unsigned *status = (unsigned *)(fr + 8);
    const int nb = (int)((N + NOALLOC_PER_BLOCK - 1) / NOALLOC_PER_BLOCK);
    // the status word keeps the previous call's value: clear it
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), s) != cudaSuccess) return HOT_ECUDA;
    // A rejected launch would leave the previous call's frame in the scratch array, so
    // each launch is checked before that record is copied out.
    HOT_COUNT_LAUNCH();
    k_bbox_part<<<nb, BT, 0, s>>>(pos, mass, N, part, status);
    if (cudaGetLastError() != cudaSuccess) return HOT_ECUDA;
    HOT_COUNT_LAUNCH();
    k_bbox_final<<<1, BF, 0, s>>>(part, nb, fr);
    if (cudaGetLastError() != cudaSuccess) return HOT_ECUDA;
    if (cudaMemcpyAsync(frame, fr, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return HOT_ECUDA;
    unsigned bits = 0;
    if (cudaMemcpyAsync(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HOT_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HOT_ECUDA;
    return (bits & HOT_ST_INPUT) ? HOT_EINPUT : HOT_OK;
}

// ---------------------------------------------------------------------------
// Stable sort of (key, value) pairs by the low `bits` bits of the key (LSD passes of
// 8 bits); used to transpose interaction lists and to order the groups by cost.  The
// digit histograms of every pass in one launch, then one launch per pass (k_rs_pass).
// The result is left in keys/vals.
// ---------------------------------------------------------------------------
int hot_sort_pairs(hot_ctx *c, uint64_t *keys, uint32_t *vals, uint64_t *ktmp, uint32_t *vtmp, int64_t n, int bits)
{
    cudaStream_t s = c->st;
    if (n <= 0) return HOT_OK;
    if (n >= (int64_t)1 << 30) return HOT_EOVERFLOW;  // the published counts hold 30 bits
    const int passes = (bits + 7) / 8 < 8 ? (bits + 7) / 8 : 8;
    const int nkb = c->nsm * 4;
    HOT_CK(c->rs_bhist.ensure(2048 * (size_t)nkb, s));
    HOT_CK(c->rs_goff.ensure(2048, s));
    HOT_CK(rs_prepare(c, passes, n));
    HOT_COUNT_LAUNCH();
    k_rs_hist_all<<<nkb, 256, 0, s>>>(keys, n, passes, c->rs_bhist.p);
    HOT_COUNT_LAUNCH();
    k_rs_goff<<<passes, 1024, 0, s>>>(c->rs_bhist.p, nkb, c->rs_goff.p);
    HOT_CK(rs_passes(c, keys, vals, ktmp, vtmp, n, passes));
    if (passes & 1) {
        HOT_CK(cudaMemcpyAsync(keys, ktmp, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        HOT_CK(cudaMemcpyAsync(vals, vtmp, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}
