// hot_scan.cu -- deterministic device-wide exclusive scan (reduce, scan partials, scan tiles).
#include "hot_common.cuh"

namespace {

constexpr int ST = 256;           // threads per block
constexpr int SIPT = 8;           // items per thread
constexpr int STILE = ST * SIPT;  // items per tile

template <class In>
__global__ void k_scan_reduce(const In *__restrict__ in, int64_t n, uint64_t *__restrict__ part)
{
    int64_t base = (int64_t)blockIdx.x * STILE;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < SIPT; ++k) {
        int64_t i = base + k * ST + threadIdx.x;
        if (i < n) s += (uint64_t)in[i];
    }
    s = warp_sum(s);
    __shared__ uint64_t ws[ST / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < ST / 32; ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// One block: exclusive scan of part[0..nb) in place, total into part[nb].
__global__ void k_scan_partials(uint64_t *__restrict__ part, int64_t nb)
{
    const int T = blockDim.x;
    int64_t per = (nb + T - 1) / T;
    int64_t b0 = threadIdx.x * per;
    int64_t b1 = b0 + per < nb ? b0 + per : nb;
    uint64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += part[i];
    // block exclusive scan of s
    __shared__ uint64_t ws[32];
    uint64_t inc = warp_incl_scan(s);
    if (lane_id() == 31) ws[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint64_t v = (threadIdx.x < (unsigned)(T / 32)) ? ws[threadIdx.x] : 0;
        uint64_t vi = warp_incl_scan(v);
        ws[threadIdx.x] = vi - v;
    }
    __syncthreads();
    uint64_t run = ws[threadIdx.x >> 5] + inc - s;
    for (int64_t i = b0; i < b1; ++i) {
        uint64_t v = part[i];
        part[i] = run;
        run += v;
    }
    if (b1 == nb && b0 < b1) part[nb] = run;
    if (nb == 0 && threadIdx.x == 0) part[0] = 0;
}

template <class In, class Out>
__global__ void k_scan_tiles(const In *__restrict__ in, Out *__restrict__ out, int64_t n,
                             const uint64_t *__restrict__ part, int64_t nb)
{
    __shared__ uint64_t tile[STILE];
    __shared__ uint64_t ws[ST / 32];
    int64_t base = (int64_t)blockIdx.x * STILE;
#pragma unroll
    for (int k = 0; k < SIPT; ++k) {
        int64_t i = base + k * ST + threadIdx.x;
        tile[k * ST + threadIdx.x] = (i < n) ? (uint64_t)in[i] : 0;
    }
    __syncthreads();
    uint64_t loc[SIPT];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < SIPT; ++k) {
        loc[k] = tile[threadIdx.x * SIPT + k];
        s += loc[k];
    }
    uint64_t inc = warp_incl_scan(s);
    if (lane_id() == 31) ws[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint64_t wpre = 0;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wpre += ws[w];
    uint64_t run = part[blockIdx.x] + wpre + inc - s;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SIPT; ++k) {
        tile[threadIdx.x * SIPT + k] = run;
        run += loc[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SIPT; ++k) {
        int64_t i = base + k * ST + threadIdx.x;
        if (i < n) out[i] = (Out)tile[k * ST + threadIdx.x];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (Out)part[nb];
}

template <class In, class Out>
int scan_impl(const In *in, Out *out, int64_t n, uint64_t *tmp, cudaStream_t s)
{
    int64_t nb = (n + STILE - 1) / STILE;
    if (nb < 1) nb = 1;
    HOT_COUNT_LAUNCH();
    k_scan_reduce<In><<<(unsigned)nb, ST, 0, s>>>(in, n, tmp);
    HOT_COUNT_LAUNCH();
    k_scan_partials<<<1, 1024, 0, s>>>(tmp, nb);
    HOT_COUNT_LAUNCH();
    k_scan_tiles<In, Out><<<(unsigned)nb, ST, 0, s>>>(in, out, n, tmp, nb);
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}

}  // namespace

size_t hot_scan_tmp_elems(int64_t n) { return (size_t)((n + STILE - 1) / STILE + 2); }

int hot_scan_u32_to_u32(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *tmp, cudaStream_t s)
{
    return scan_impl<uint32_t, uint32_t>(in, out, n, tmp, s);
}

int hot_scan_u32_to_i64(const uint32_t *in, int64_t *out, int64_t n, uint64_t *tmp, cudaStream_t s)
{
    return scan_impl<uint32_t, int64_t>(in, out, n, tmp, s);
}
