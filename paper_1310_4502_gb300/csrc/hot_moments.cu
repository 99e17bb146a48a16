// hot_moments.cu -- cell moments (Eq. "moment tensor": M_a(z) = sum m (x - z)^a about the
// centre of mass z), built as P2M at the leaves and exact binomial translation (M2M,
// "expand M(y0 + Delta) in powers of Delta and recollect") level by level upwards, all in
// float64; the acceptance-test aggregates b_max = max |x - z| and B_n = sum m |x - z|^n
// (n = p+1, p+2) taken from the particles; and the per-cell interaction records.
#include "hot_common.cuh"
#include "generated.cuh"

namespace {

constexpr int MW = 4;  // warps per block
constexpr int CHUNK = 2048;  // particles per aggregate work item

// ---------------------------------------------------------------------------
// P2M at leaves: one warp per leaf.  Also b_max, B_{p+1}, B_{p+2} of the leaf and
// the leaf-relative single-precision particle copy used by the P2P interactions.
// The centre of mass and the acceptance aggregates are float64 (they decide the
// acceptance test); the moment sums run in T on the leaf-relative offsets (float32 in
// the mixed mode, which only feeds float32 interaction records and the float64 M2M)
// and are stored as float64.
// ---------------------------------------------------------------------------
// sqrt(x) to about 1e-13 relative, for the powers of the aggregates (b_max itself is the
// correctly rounded square root of the largest x): the float32 reciprocal square root
// refined by one Newton step in float64 (r0 = x y, r = r0 + (x - r0^2) y/2, error about
// the square of y's), three float64 operations where the correctly rounded root takes
// several times that; outside [1e-36, 1e36] the float64 root.
__device__ __forceinline__ double near_sqrt(double x)
{
    if (!(x >= 1e-36 && x <= 1e36)) return sqrt(x);
    const float y = rsqrtf((float)x);
    const double r0 = x * (double)y;
    return fma(fma(-r0, r0, x), 0.5 * (double)y, r0);
}

// Warp sums of four (two) doubles in six (five) float64 additions per lane instead of
// twenty (ten): the lanes specialise, each exchange halving the quantities a lane
// carries, until each group of 8 (16) lanes reduces one; the totals are returned in every
// lane.  (A float64 addition occupies the pipe for a whole warp instruction however many
// lanes need it, at a sixty-fourth of the float32 rate.)
__device__ __forceinline__ void warp_sum4(double &a, double &b, double &c, double &d)
{
    const unsigned lane = lane_id();
    const bool h = lane & 16, q = lane & 8;
    double k0 = h ? c : a, k1 = h ? d : b;
    k0 += __shfl_xor_sync(0xffffffffu, h ? a : c, 16);
    k1 += __shfl_xor_sync(0xffffffffu, h ? b : d, 16);
    double v = q ? k1 : k0;
    v += __shfl_xor_sync(0xffffffffu, q ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    a = __shfl_sync(0xffffffffu, v, 0);
    b = __shfl_sync(0xffffffffu, v, 8);
    c = __shfl_sync(0xffffffffu, v, 16);
    d = __shfl_sync(0xffffffffu, v, 24);
}
__device__ __forceinline__ void warp_sum2(double &a, double &b)
{
    const unsigned lane = lane_id();
    const bool h = lane & 16;
    double v = h ? b : a;
    v += __shfl_xor_sync(0xffffffffu, h ? a : b, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    a = __shfl_sync(0xffffffffu, v, 0);
    b = __shfl_sync(0xffffffffu, v, 16);
}

__device__ __forceinline__ unsigned long long dmax_bits(unsigned long long a, double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);  // x >= 0
    return u > a ? u : a;
}

// r^(P+1) and r^(P+2) from r and r^2 = |d|^2 by powers of r^2 (three multiplications at
// p = 4 where repeated multiplication by r took six: the float64 pipe is the bound here)
template <int P>
__device__ __forceinline__ void rpow_pair(double r, double r2, double &rp, double &rq)
{
    double h = 1.0;  // r2^floor((P+1)/2)
#pragma unroll
    for (int q = 0; q < (P + 1) / 2; ++q) h *= r2;
    if constexpr ((P + 1) % 2 == 0) {
        rp = h;
        rq = h * r;
    } else {
        rp = h * r;
        rq = h * r2;
    }
}

template <int P, class T>
__global__ void __launch_bounds__(MW * 32) k_p2m_leaf(
    const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount,
    const int32_t *__restrict__ cnchild, int64_t ncell, const double *__restrict__ spos,
    const double *__restrict__ smass, double *__restrict__ cmass, double *__restrict__ ccom,
    double *__restrict__ cmom, double *__restrict__ cbmax, double *__restrict__ cB1,
    double *__restrict__ cB2, float4 *__restrict__ prel)
{
    constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
    __shared__ T pw[MW][32][3][P + 1];
    __shared__ T pm[MW][32];
    __shared__ unsigned char mi[NC][3];
    for (int k = threadIdx.x; k < NC; k += blockDim.x) {
        mi[k][0] = hot_midx[k][0];
        mi[k][1] = hot_midx[k][1];
        mi[k][2] = hot_midx[k][2];
    }
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * MW;
    for (int64_t c = (int64_t)blockIdx.x * MW + w; c < ncell; c += nw) {
        if (cnchild[c] != 0) continue;
        const int64_t b = cbegin[c], n = ccount[c];
        double m = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
        for (int64_t s = b + lane; s < b + n; s += 32) {
            double ms = smass[s];
            m += ms;
            mx += ms * spos[3 * s + 0];
            my += ms * spos[3 * s + 1];
            mz += ms * spos[3 * s + 2];
        }
        warp_sum4(m, mx, my, mz);
        // the centre's three components by lanes 0, 1, 2 in one division (a float64
        // division is a long sequence of warp instructions on this part)
        const double zq = (lane == 1 ? my : (lane == 2 ? mz : mx)) / m;
        const double z[3] = {__shfl_sync(0xffffffffu, zq, 0), __shfl_sync(0xffffffffu, zq, 1),
                             __shfl_sync(0xffffffffu, zq, 2)};
        T acc[(NC + 31) / 32];
#pragma unroll
        for (int q = 0; q < (NC + 31) / 32; ++q) acc[q] = T(0);
        double B1 = 0.0, B2 = 0.0;
        unsigned long long r2max = 0ull;  // bit pattern of the largest |d|^2 (non-negative)
        for (int64_t s0 = b; s0 < b + n; s0 += 32) {
            int64_t s = s0 + lane;
            bool valid = s < b + n;
            double d[3] = {0.0, 0.0, 0.0}, ms = 0.0;
            if (valid) {
                ms = smass[s];
                for (int e = 0; e < 3; ++e) d[e] = spos[3 * s + e] - z[e];
                const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                r2max = dmax_bits(r2max, r2);
                double rp, rq;
                rpow_pair<P>(near_sqrt(r2), r2, rp, rq);
                B1 += ms * rp;
                B2 += ms * rq;
                prel[s] = make_float4((float)d[0], (float)d[1], (float)d[2], (float)ms);
            }
            pm[w][lane] = (T)ms;
            for (int e = 0; e < 3; ++e) {
                const T de = (T)d[e];
                T v = T(1);
                for (int q = 0; q <= P; ++q) {
                    pw[w][lane][e][q] = v;
                    v *= de;
                }
            }
            __syncwarp();
            int cnt = (int)((b + n - s0) < 32 ? (b + n - s0) : 32);
#pragma unroll
            for (int q = 0; q < (NC + 31) / 32; ++q) {
                int a = lane + 32 * q;
                if (a < NC) {
                    int ax = mi[a][0], ay = mi[a][1], az = mi[a][2];
                    T t = T(0);
                    for (int j = 0; j < cnt; ++j)
                        t += pm[w][j] * pw[w][j][0][ax] * pw[w][j][1][ay] * pw[w][j][2][az];
                    acc[q] += t;
                }
            }
            __syncwarp();
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, r2max, o);
            r2max = t > r2max ? t : r2max;
        }
        const double bmax = sqrt(__longlong_as_double((long long)r2max));
        warp_sum2(B1, B2);
#pragma unroll
        for (int q = 0; q < (NC + 31) / 32; ++q) {
            int a = lane + 32 * q;
            if (a < NC) cmom[c * NC + a] = (double)acc[q];
        }
        if (lane == 0) {
            cmass[c] = m;
            ccom[3 * c + 0] = z[0];
            ccom[3 * c + 1] = z[1];
            ccom[3 * c + 2] = z[2];
            cbmax[c] = bmax;
            cB1[c] = B1;
            cB2[c] = B2;
        }
    }
}

// ---------------------------------------------------------------------------
// M2M for the inner cells of one level: one block of 8 warps per cell, warp o
// translating child o (lanes over components), the children's rows summed in child
// order.  M_a(z) = sum_children sum_{b <= a} C(a,b) M_b(z_ch) (z_ch - z)^{a-b}.  The
// binomial translation factorises over the axes, so it is applied as three
// one-dimensional translations (x, then y, then z):
//   T1(i,j,k) = sum_{i' <= i} C(i,i') dx^{i-i'} M(i',j,k),  then likewise in j and in k,
// at most p+1 terms per component and pass, each one fused multiply-add with the
// factor C(e,e') d^{e-e'} taken from a per-child table (float64 throughout).
// CUBE: the moments are about the cells' cube centres cen (background subtraction), which
// are fixed, so nothing but the moments is written.
// ---------------------------------------------------------------------------
constexpr int M2M_W = 8;  // warps per block: one per child octant

__device__ __forceinline__ int mom_index(int i, int j, int k)
{
    const int n = i + j + k;
    return n * (n + 1) * (n + 2) / 6 + (n - i) * (n - i + 1) / 2 + (n - i - j);
}

// Mass and centre of mass of the inner cells of one level from their children (octant
// order), one thread per cell: the traversal's chain needs only these, so the moment
// translations can run beside it.
__global__ void k_com_level(const int32_t *__restrict__ cells, int64_t n, const int32_t *__restrict__ child8,
                            const int32_t *__restrict__ cnchild, double *__restrict__ cmass, double *__restrict__ ccom)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int32_t c = cells[q];
    if (cnchild[c] == 0) return;
    double m = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int32_t k = child8[8 * (int64_t)c + o];
        if (k >= 0) {
            const double mc = cmass[k];
            m += mc;
            mx += mc * ccom[3 * (int64_t)k + 0];
            my += mc * ccom[3 * (int64_t)k + 1];
            mz += mc * ccom[3 * (int64_t)k + 2];
        }
    }
    cmass[c] = m;
    ccom[3 * (int64_t)c + 0] = mx / m;
    ccom[3 * (int64_t)c + 1] = my / m;
    ccom[3 * (int64_t)c + 2] = mz / m;
}

// The same for the levels l1-1 down to l0 in one block (levels of few cells: one launch
// for several of them), a barrier between levels.
__global__ void __launch_bounds__(1024) k_com_levels(const int32_t *__restrict__ cells, const int64_t *__restrict__ levoff,
                                                     int l0, int l1, const int32_t *__restrict__ child8,
                                                     const int32_t *__restrict__ cnchild, double *__restrict__ cmass,
                                                     double *__restrict__ ccom)
{
    for (int l = l1 - 1; l >= l0; --l) {
        const int64_t a = levoff[l], n = levoff[l + 1] - a;
        for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
            const int32_t c = cells[a + q];
            if (cnchild[c] == 0) continue;
            double m = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int32_t k = child8[8 * (int64_t)c + o];
                if (k >= 0) {
                    const double mc = cmass[k];
                    m += mc;
                    mx += mc * ccom[3 * (int64_t)k + 0];
                    my += mc * ccom[3 * (int64_t)k + 1];
                    mz += mc * ccom[3 * (int64_t)k + 2];
                }
            }
            cmass[c] = m;
            ccom[3 * (int64_t)c + 0] = mx / m;
            ccom[3 * (int64_t)c + 1] = my / m;
            ccom[3 * (int64_t)c + 2] = mz / m;
        }
        __syncthreads();
    }
}

// CUBE = false: the cells' mass and centre are those of k_com_level; CUBE = true (the
// contrast expansions of background subtraction): about the given cube centres.
template <int P, bool CUBE = false>
__global__ void __launch_bounds__(M2M_W * 32) k_m2m_level(
    const int32_t *__restrict__ cells, int64_t ncells_lvl, const int32_t *__restrict__ child8,
    const int32_t *__restrict__ cnchild, double *__restrict__ cmass, double *__restrict__ ccom,
    double *__restrict__ cmom)
{
    constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
    constexpr int NF = (P + 1) * (P + 2) / 2;  // factors (e, e') with e' <= e <= P, per axis
    __shared__ double sa[M2M_W][NC], sb[M2M_W][NC];  // a child's moments and partial translations
    __shared__ double fac[M2M_W][3][NF];             // C(e,e') d^(e-e'), d = z_ch - z per axis
    __shared__ double binom[P + 1][P + 1];
    __shared__ unsigned char mi[NC][3];
    __shared__ int32_t sch[M2M_W];
    __shared__ double smc[M2M_W][4];  // child mass and centre
    __shared__ double spz[4];         // parent mass and centre
    for (int k = threadIdx.x; k < NC; k += blockDim.x) {
        mi[k][0] = hot_midx[k][0];
        mi[k][1] = hot_midx[k][1];
        mi[k][2] = hot_midx[k][2];
    }
    for (int k = threadIdx.x; k < (P + 1) * (P + 1); k += blockDim.x) {
        const int n = k / (P + 1), r = k % (P + 1);
        double v = 0.0;
        if (r <= n) {
            v = 1.0;
            for (int t = 1; t <= r; ++t) v = v * (double)(n - r + t) / (double)t;
        }
        binom[n][r] = v;
    }
    const int o = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    for (int64_t q0 = blockIdx.x; q0 < ncells_lvl; q0 += gridDim.x) {
        const int32_t c = cells[q0];
        if (cnchild[c] == 0) continue;  // uniform over the block
        __syncthreads();
        if (threadIdx.x < M2M_W) {
            const int32_t k = child8[8 * (int64_t)c + threadIdx.x];
            sch[threadIdx.x] = k;
            if (k >= 0) {
                smc[threadIdx.x][0] = 0.0;  // (the child's mass: not needed here)
#pragma unroll
                for (int d = 0; d < 3; ++d) smc[threadIdx.x][1 + d] = ccom[3 * (int64_t)k + d];
            }
        }
        __syncthreads();
        // the expansion centre, shared by the block
        if (threadIdx.x == 0) {
#pragma unroll
            for (int d = 0; d < 3; ++d) spz[1 + d] = ccom[3 * (int64_t)c + d];
        }
        __syncthreads();
        const double z[3] = {spz[1], spz[2], spz[3]};
        const int32_t k = sch[o];
        if (k >= 0) {
            for (int g = lane; g < 3 * NF; g += 32) {
                const int d = g / NF, f = g % NF;
                int e = 0;
                while ((e + 1) * (e + 2) / 2 <= f) ++e;
                const int e2 = f - e * (e + 1) / 2;
                const double dd = smc[o][1 + d] - z[d];
                double pw = 1.0;
                for (int t = 0; t < e - e2; ++t) pw *= dd;
                fac[o][d][f] = binom[e][e2] * pw;
            }
            for (int g = lane; g < NC; g += 32) sa[o][g] = cmom[(int64_t)k * NC + g];
            __syncwarp();
            // pass 1 (x): sa -> sb
            for (int a = lane; a < NC; a += 32) {
                const int i = mi[a][0], j = mi[a][1], kk = mi[a][2];
                const double *F = &fac[o][0][i * (i + 1) / 2];
                double t = 0.0;
                for (int i2 = 0; i2 <= i; ++i2) t += F[i2] * sa[o][mom_index(i2, j, kk)];
                sb[o][a] = t;
            }
            __syncwarp();
            // pass 2 (y): sb -> sa
            for (int a = lane; a < NC; a += 32) {
                const int i = mi[a][0], j = mi[a][1], kk = mi[a][2];
                const double *F = &fac[o][1][j * (j + 1) / 2];
                double t = 0.0;
                for (int j2 = 0; j2 <= j; ++j2) t += F[j2] * sb[o][mom_index(i, j2, kk)];
                sa[o][a] = t;
            }
            __syncwarp();
            // pass 3 (z): sa -> sb, the child's contribution
            for (int a = lane; a < NC; a += 32) {
                const int i = mi[a][0], j = mi[a][1], kk = mi[a][2];
                const double *F = &fac[o][2][kk * (kk + 1) / 2];
                double t = 0.0;
                for (int k2 = 0; k2 <= kk; ++k2) t += F[k2] * sa[o][mom_index(i, j, k2)];
                sb[o][a] = t;
            }
        }
        __syncthreads();
        for (int a = threadIdx.x; a < NC; a += blockDim.x) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < M2M_W; ++q)
                if (sch[q] >= 0) t += sb[q][a];
            cmom[(int64_t)c * NC + a] = t;
        }
    }
}

// ---------------------------------------------------------------------------
// Acceptance-test aggregates of inner cells from their particles, split into
// work items of at most CHUNK particles so that large cells spread over the GPU.
// ---------------------------------------------------------------------------
__global__ void k_item_count(const int32_t *__restrict__ ccount, const int32_t *__restrict__ cnchild,
                             int64_t ncell, uint32_t *__restrict__ nitem)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    nitem[c] = cnchild[c] == 0 ? 0u : (uint32_t)((ccount[c] + CHUNK - 1) / CHUNK);
}

__global__ void k_item_cells(const uint32_t *__restrict__ off, int64_t ncell, int32_t *__restrict__ item_cell)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    for (uint32_t k = off[c]; k < off[c + 1]; ++k) item_cell[k] = (int32_t)c;
}

template <int P>
__global__ void __launch_bounds__(MW * 32) k_item_part(
    const int32_t *__restrict__ item_cell, const uint32_t *__restrict__ off,
    const uint32_t *__restrict__ nitem_p, const int32_t *__restrict__ cbegin,
    const int32_t *__restrict__ ccount, const double *__restrict__ ccom,
    const double *__restrict__ spos, const double *__restrict__ smass, double *__restrict__ part)
{
    const int64_t nitem = *nitem_p;
    const unsigned lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * MW;
    for (int64_t it = (int64_t)blockIdx.x * MW + (threadIdx.x >> 5); it < nitem; it += nw) {
        const int32_t c = item_cell[it];
        const int64_t k = it - off[c];
        const int64_t b = cbegin[c] + k * CHUNK;
        const int64_t e0 = cbegin[c] + (int64_t)ccount[c];
        const int64_t e = b + CHUNK < e0 ? b + CHUNK : e0;
        const double z0 = ccom[3 * (int64_t)c + 0], z1 = ccom[3 * (int64_t)c + 1], z2 = ccom[3 * (int64_t)c + 2];
        double B1 = 0.0, B2 = 0.0;
        unsigned long long r2max = 0ull;  // bit pattern of the largest |d|^2 (non-negative)
        for (int64_t s = b + lane; s < e; s += 32) {
            double dx = spos[3 * s + 0] - z0, dy = spos[3 * s + 1] - z1, dz = spos[3 * s + 2] - z2;
            const double r2 = dx * dx + dy * dy + dz * dz;
            r2max = dmax_bits(r2max, r2);
            double rp, rq;
            rpow_pair<P>(near_sqrt(r2), r2, rp, rq);
            double ms = smass[s];
            B1 += ms * rp;
            B2 += ms * rq;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, r2max, o);
            r2max = t > r2max ? t : r2max;
        }
        const double bmax = sqrt(__longlong_as_double((long long)r2max));
        warp_sum2(B1, B2);
        if (lane == 0) {
            part[3 * it + 0] = bmax;
            part[3 * it + 1] = B1;
            part[3 * it + 2] = B2;
        }
    }
}

// One warp per inner cell: lane l takes items l, l + 32, ... (the root holds N / CHUNK
// of them), then a butterfly over the lanes (a fixed order: reproducible).
__global__ void k_item_combine(const uint32_t *__restrict__ off, const int32_t *__restrict__ cnchild,
                               int64_t ncell, const double *__restrict__ part, double *__restrict__ cbmax,
                               double *__restrict__ cB1, double *__restrict__ cB2)
{
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = lane_id();
    if (c >= ncell || cnchild[c] == 0) return;  // uniform over the warp
    double bmax = 0.0, B1 = 0.0, B2 = 0.0;
    for (uint32_t k = off[c] + lane; k < off[c + 1]; k += 32) {
        bmax = fmax(bmax, part[3 * (int64_t)k + 0]);
        B1 += part[3 * (int64_t)k + 1];
        B2 += part[3 * (int64_t)k + 2];
    }
    bmax = warp_max(bmax);
    B1 = warp_sum(B1);
    B2 = warp_sum(B2);
    if (lane == 0) {
        cbmax[c] = bmax;
        cB1[c] = B1;
        cB2[c] = B2;
    }
}

// ---------------------------------------------------------------------------
// Interaction records: scale s = power of two >= b_max (the cell's size when
// b_max = 0), so that single-precision coefficients stay O(1).
// ---------------------------------------------------------------------------
template <int P, class T>
__global__ void k_records(const double *__restrict__ cmom, const double *__restrict__ ccom,
                          const double *__restrict__ cbmax,
                          const int32_t *__restrict__ clevel, int64_t ncell, const double *__restrict__ frame,
                          double G, double eps, int reclen, int mom_stride, T *__restrict__ rec)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double L = frame[3];
    double b = cbmax[c];
    int e;
    double inv_s;
    if (b > 0.0) {
        frexp(b, &e);
        inv_s = ldexp(1.0, -e);
    } else {
        frexp(L, &e);
        inv_s = ldexp(1.0, clevel[c] - e);
    }
    m2p_record<P, T>(cmom + c * mom_stride, ccom + 3 * c, inv_s, G, eps, rec + c * (int64_t)reclen);
}

// ---------------------------------------------------------------------------
// Per-interaction order selection: B_n = sum m |x - z|^n for n = 0..p+2 of every cell
// (the acceptance bound of each order q needs B_{q+1}, B_{q+2}), from the particles in
// work items of CHUNK, summed per cell in item order; and the records of the lower
// orders, from the leading components of the order-p moments.
// ---------------------------------------------------------------------------
__global__ void k_bn_count(const int32_t *__restrict__ ccount, int64_t ncell, uint32_t *__restrict__ nitem)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) nitem[c] = (uint32_t)((ccount[c] + CHUNK - 1) / CHUNK);
}

template <int P>
__global__ void __launch_bounds__(MW * 32) k_bn_part(
    const int32_t *__restrict__ item_cell, const uint32_t *__restrict__ off, const uint32_t *__restrict__ nitem_p,
    const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount, const double *__restrict__ ccom,
    const double *__restrict__ spos, const double *__restrict__ smass, double *__restrict__ part)
{
    constexpr int NB = P + 3;
    const int64_t nitem = *nitem_p;
    const unsigned lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * MW;
    for (int64_t it = (int64_t)blockIdx.x * MW + (threadIdx.x >> 5); it < nitem; it += nw) {
        const int32_t c = item_cell[it];
        const int64_t b = cbegin[c] + (it - off[c]) * CHUNK;
        const int64_t e0 = cbegin[c] + (int64_t)ccount[c];
        const int64_t e = b + CHUNK < e0 ? b + CHUNK : e0;
        const double z0 = ccom[3 * (int64_t)c + 0], z1 = ccom[3 * (int64_t)c + 1], z2 = ccom[3 * (int64_t)c + 2];
        double B[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) B[q] = 0.0;
        for (int64_t s = b + lane; s < e; s += 32) {
            const double dx = spos[3 * s + 0] - z0, dy = spos[3 * s + 1] - z1, dz = spos[3 * s + 2] - z2;
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const double ms = smass[s];
            double rq = 1.0;
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                B[q] += ms * rq;
                rq *= r;
            }
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const double v = warp_sum(B[q]);
            if (lane == 0) part[NB * it + q] = v;
        }
    }
}

// One warp per cell and order: lanes over the items, then a butterfly (a fixed order).
__global__ void k_bn_combine(const uint32_t *__restrict__ off, int64_t ncell, int nb, const double *__restrict__ part,
                             double *__restrict__ cBn)
{
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = lane_id();
    if (i >= ncell * nb) return;  // uniform over the warp
    const int64_t c = i / nb;
    const int q = (int)(i - c * nb);
    double t = 0.0;
    for (uint32_t k = off[c] + lane; k < off[c + 1]; k += 32) t += part[(int64_t)nb * k + q];
    t = warp_sum(t);
    if (lane == 0) cBn[(int64_t)nb * c + q] = t;
}

// Records of order q from moments of stride mom_stride (the order-p moments).
template <class T>
int records_of_order(hot_ctx *c, int q, int mom_stride, double eps_rec, T *dst)
{
    const int64_t nc = c->ncell;
    HOT_COUNT_LAUNCH();
#define HOT_REC_Q(QQ)                                                                                         \
    case QQ:                                                                                                  \
        k_records<QQ, T><<<hot_blocks(nc, 128), 128, 0, c->st>>>(c->cmom.p, c->ccom.p, c->cbmax.p, c->clevel.p, \
                                                                 nc, c->frame.p, c->prm.G, eps_rec,          \
                                                                 HOT_REC_LEN[QQ], mom_stride, dst);           \
        break;
    switch (q) {
        HOT_REC_Q(0)
        HOT_REC_Q(1)
        HOT_REC_Q(2)
        HOT_REC_Q(3)
        HOT_REC_Q(4)
        HOT_REC_Q(5)
        HOT_REC_Q(6)
        HOT_REC_Q(7)
        HOT_REC_Q(8)
        default: return HOT_EINVAL;
    }
#undef HOT_REC_Q
    return HOT_OK;
}

// ---------------------------------------------------------------------------
// Background subtraction (Sec. "Background Subtraction"): the expansion of a cell outside
// a group's surrounding cube is that of its density contrast -- the particles' moments
// about the cube's geometric centre minus those of the uniform density rho = M / L^3
// filling the cube, both to order p -- and the empty octants of opened cells (cubes of
// density -rho) are cells of their own.  Moments are taken to order p + 2 for the sizes
// Q_n = (sum_{|a| = n} n!/a! M_a^2)^(1/2) of the contrast's first two omitted orders,
// which its acceptance test uses.  All float64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v | (v >> 4)) & 0x100f00f00f00f00full;
    v = (v | (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v | (v >> 16)) & 0x1f00000000ffffull;
    v = (v | (v >> 32)) & 0x1fffffull;
    return v;
}

// Cube of every cell: side s = L / 2^level, centre lo + s (i + 1/2) per axis, i the cell's
// integer coordinate at its level (the key's interleaved digits); and rho = M / L^3.
__global__ void k_bg_geom(const uint64_t *__restrict__ ckey, const int32_t *__restrict__ clevel, int64_t ncell,
                          const double *__restrict__ frame, const double *__restrict__ cmass, double *__restrict__ cen,
                          double *__restrict__ half, double *__restrict__ rho)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int l = clevel[c];
    const uint64_t k = l > 0 ? ckey[c] & ((1ull << (3 * l)) - 1ull) : 0ull;
    const uint64_t ix = compact3(k >> 2), iy = compact3(k >> 1), iz = compact3(k);
    const double L = frame[3];
    const double s = L / (double)(1ull << l);
    cen[3 * c + 0] = __dadd_rn(frame[0], __dmul_rn(s, (double)ix + 0.5));
    cen[3 * c + 1] = __dadd_rn(frame[1], __dmul_rn(s, (double)iy + 0.5));
    cen[3 * c + 2] = __dadd_rn(frame[2], __dmul_rn(s, (double)iz + 0.5));
    half[c] = 0.5 * s;
    if (c == 0) *rho = cmass[0] / (L * L * L);
}

// Moments of every leaf about its cube centre to order P2, one warp per leaf (lanes over
// the components).  Per batch of 32 particles each lane stages, for its particle, the
// products m x^i y^j (i + j <= P2) and the powers z^k, so that every component then takes
// one fused multiply-add per particle: sum_s (m x^i y^j)_s (z^k)_s.
constexpr int BGW = 2;  // warps per block of k_bg_p2m (its staging is 14 KB per warp at P2 = 8)

template <int P2>
__global__ void __launch_bounds__(BGW * 32) k_bg_p2m(const int32_t *__restrict__ cbegin,
                                                     const int32_t *__restrict__ ccount,
                                                     const int32_t *__restrict__ cnchild, int64_t ncell,
                                                     const double *__restrict__ spos, const double *__restrict__ smass,
                                                     const double *__restrict__ cen, double *__restrict__ mom)
{
    constexpr int NC = (P2 + 1) * (P2 + 2) * (P2 + 3) / 6;
    constexpr int NXY = (P2 + 1) * (P2 + 2) / 2;  // pairs (i, j), i + j <= P2
    __shared__ double pxy[BGW][NXY][33];          // [pair][particle], padded against bank conflicts
    __shared__ double pz[BGW][P2 + 1][33];
    __shared__ unsigned char cidx[NC][2];         // component -> (pair index, k)
    for (int a = threadIdx.x; a < NC; a += blockDim.x) {
        const int i = hot_midx[a][0], j = hot_midx[a][1];
        // pairs ordered by i, then j: index of (i, j) = sum_{i' < i} (P2 + 1 - i') + j
        cidx[a][0] = (unsigned char)(i * (P2 + 1) - i * (i - 1) / 2 + j);
        cidx[a][1] = hot_midx[a][2];
    }
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    for (int64_t c = (int64_t)blockIdx.x * BGW + w; c < ncell; c += (int64_t)gridDim.x * BGW) {
        if (cnchild[c] != 0) continue;
        const int64_t b = cbegin[c], n = ccount[c];
        const double z[3] = {cen[3 * c + 0], cen[3 * c + 1], cen[3 * c + 2]};
        double acc[(NC + 31) / 32];
#pragma unroll
        for (int q = 0; q < (NC + 31) / 32; ++q) acc[q] = 0.0;
        for (int64_t s0 = b; s0 < b + n; s0 += 32) {
            const int64_t s = s0 + lane;
            const bool valid = s < b + n;
            const double dx = valid ? spos[3 * s + 0] - z[0] : 0.0;
            const double dy = valid ? spos[3 * s + 1] - z[1] : 0.0;
            const double dz = valid ? spos[3 * s + 2] - z[2] : 0.0;
            double mx = valid ? smass[s] : 0.0;  // m x^i
            int k = 0;
            for (int i = 0; i <= P2; ++i) {
                double v = mx;
                for (int j = 0; j <= P2 - i; ++j) {
                    pxy[w][k++][lane] = v;
                    v *= dy;
                }
                mx *= dx;
            }
            double vz = 1.0;
            for (int q = 0; q <= P2; ++q) {
                pz[w][q][lane] = vz;
                vz *= dz;
            }
            __syncwarp();
            const int cnt = (int)((b + n - s0) < 32 ? (b + n - s0) : 32);
#pragma unroll
            for (int q = 0; q < (NC + 31) / 32; ++q) {
                const int a = lane + 32 * q;
                if (a < NC) {
                    const double *px = pxy[w][cidx[a][0]], *qz = pz[w][cidx[a][1]];
                    double t = 0.0;
                    for (int jj = 0; jj < cnt; ++jj) t = fma(px[jj], qz[jj], t);
                    acc[q] += t;
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < (NC + 31) / 32; ++q) {
            const int a = lane + 32 * q;
            if (a < NC) mom[c * NC + a] = acc[q];
        }
    }
}

// Empty octants of every inner cell (none for a leaf).
__global__ void k_bg_ecount(const int32_t *__restrict__ cnchild, int64_t ncell, uint32_t *__restrict__ ecnt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) ecnt[c] = cnchild[c] > 0 ? (uint32_t)(8 - cnchild[c]) : 0u;
}

// Empty octant e = eoff[c] + k (the k-th missing child of c, ascending octants): its parent,
// octant, and cube (side s = half the parent's, lower corner (centre_c - side_c / 2) + s off,
// centre lower corner + s / 2), stored after the cells' cubes.
__global__ void k_bg_efill(const int32_t *__restrict__ child8, const uint32_t *__restrict__ eoff, int64_t ncell,
                           double *__restrict__ cen, double *__restrict__ half, int32_t *__restrict__ eparent,
                           int32_t *__restrict__ eoct)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    uint32_t e = eoff[c];
    if (eoff[c + 1] == e) return;
    const double hc = half[c], s = hc;  // the octant's side is the parent's half side
    for (int o = 0; o < 8; ++o) {
        if (child8[8 * c + o] >= 0) continue;
        const int off[3] = {(o >> 2) & 1, (o >> 1) & 1, o & 1};
        const int64_t q = ncell + e;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double lo = __dadd_rn(__dsub_rn(cen[3 * c + d], hc), off[d] ? s : 0.0);
            cen[3 * q + d] = __dadd_rn(lo, 0.5 * s);
        }
        half[q] = 0.5 * s;
        eparent[e] = (int32_t)c;
        eoct[e] = o;
        ++e;
    }
}

// Moments about its centre of the uniform cube of density rho at every level l (half side
// h = L / 2^(l+1)): rho prod_d int_{-h}^{h} t^(a_d) dt = rho prod_d 2 h^(a_d+1) / (a_d+1),
// zero unless every a_d is even; and the multinomial factors n!/a! of every component.
// One thread per (level, component).
template <int P2>
__global__ void k_bg_cubetab(const double *__restrict__ frame, const double *__restrict__ rho_p,
                             double *__restrict__ tab, double *__restrict__ mcoef)
{
    constexpr int NC2 = (P2 + 1) * (P2 + 2) * (P2 + 3) / 6;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (HOT_MAXLEVEL + 2) * NC2) return;
    const int l = k / NC2, a = k % NC2;
    const int e[3] = {hot_midx[a][0], hot_midx[a][1], hot_midx[a][2]};
    const double h = frame[3] / (double)(2ull << l);
    double v = *rho_p;
    double f = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (e[d] & 1) v = 0.0;
        double t = 2.0 * h;
        for (int s = 0; s < e[d]; ++s) t *= h;
        v *= t / (double)(e[d] + 1);
        for (int s = 2; s <= e[d]; ++s) f *= (double)s;
    }
    tab[k] = v;
    if (l == 0) {
        double fnn = 1.0;
        for (int s = 2; s <= e[0] + e[1] + e[2]; ++s) fnn *= (double)s;
        mcoef[a] = fnn / f;
    }
}

// Contrast of every cube and its records: for a cell, its moments about the cube centre
// minus the uniform cube's (in place, to order P + 2); for an empty octant, minus the
// uniform cube's.  Q_{P+1}, Q_{P+2} to bg_q; the order-P record (scale: a power of two at
// least the half-diagonal) to rec + (ncell + q) * reclen.  The uniform cube's moments come
// from the per-level table (a cell's level; an empty octant's, its parent's plus one).
template <int P, class T>
__global__ void k_bg_records(int64_t ncell, int64_t ncube, const double *__restrict__ cen,
                             const double *__restrict__ half, const int32_t *__restrict__ clevel,
                             const int32_t *__restrict__ eparent, const double *__restrict__ tab,
                             const double *__restrict__ mcoef, double *__restrict__ mom, double *__restrict__ bq,
                             double G, double eps, int reclen, T *__restrict__ rec)
{
    constexpr int P2 = P + 2;
    constexpr int NC2 = (P2 + 1) * (P2 + 2) * (P2 + 3) / 6;
    constexpr int NCP = (P + 1) * (P + 2) * (P + 3) / 6;
    constexpr int N1 = (P + 1) * (P + 2) * (P + 3) / 6, N2 = (P + 2) * (P + 3) * (P + 4) / 6;  // order p+1 and p+2 start
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ncube) return;
    const double h = half[q];
    const int lv = q < ncell ? clevel[q] : clevel[eparent[q - ncell]] + 1;
    const double *u = tab + (int64_t)lv * NC2;
    double M[NCP];
    double q1 = 0.0, q2 = 0.0;
    double *m = q < ncell ? mom + q * NC2 : nullptr;
#pragma unroll 4
    for (int a = 0; a < NC2; ++a) {
        const double v = m ? m[a] - u[a] : -u[a];
        if (m) m[a] = v;
        if (a < NCP) M[a] = v;
        else if (a < N2) q1 += mcoef[a] * v * v;
        else q2 += mcoef[a] * v * v;
    }
    static_assert(N1 == NCP, "order p+1 starts after the order-p components");
    bq[2 * q + 0] = sqrt(q1);
    bq[2 * q + 1] = sqrt(q2);
    const double b = 0.5 * sqrt(3.0) * (2.0 * h);
    int e;
    frexp(b, &e);
    m2p_record<P, T>(M, cen + 3 * q, ldexp(1.0, -e), G, eps, rec + (ncell + q) * (int64_t)reclen);
}

// Background subtraction's moments, cube records and empty octants; the records go after
// the cells' own in rec (which holds 2 ncell + n_empty records).
template <int P, class T>
int bg_records(hot_ctx *c, T *rec)
{
    constexpr int P2 = P + 2;
    constexpr int NC2 = (P2 + 1) * (P2 + 2) * (P2 + 3) / 6;
    cudaStream_t s = c->st;
    const int64_t nc = c->ncell, ncube = nc + c->n_empty;
    HOT_CK(c->bg_mom.ensure((size_t)NC2 * nc, s));
    HOT_CK(c->bg_q.ensure(2 * (size_t)ncube, s));
    HOT_CK(c->bg_tab.ensure((size_t)(HOT_MAXLEVEL + 2) * NC2 + NC2, s));
    HOT_CK(c->bg_eparent.ensure(c->n_empty + 1, s));
    HOT_CK(c->bg_eoct.ensure(c->n_empty + 1, s));
    HOT_COUNT_LAUNCH();
    k_bg_efill<<<hot_blocks(nc, 128), 128, 0, s>>>(c->child8.p, c->bg_eoff.p, nc, c->bg_cen.p, c->bg_half.p,
                                                   c->bg_eparent.p, c->bg_eoct.p);
    HOT_COUNT_LAUNCH();
    k_bg_p2m<P2><<<c->nsm * 16, BGW * 32, 0, s>>>(c->cbegin.p, c->ccount.p, c->cnchild.p, nc, c->spos.p,
                                                  c->smass.p, c->bg_cen.p, c->bg_mom.p);
    for (int l = (int)c->maxlevel - 1; l >= 0; --l) {
        const int64_t a = c->level_off[l], n = c->level_off[l + 1] - a;
        if (n <= 0) continue;
        const int blocks = (int)(n < (int64_t)c->nsm * 8 ? n : (int64_t)c->nsm * 8);
        HOT_COUNT_LAUNCH();
        k_m2m_level<P2, true><<<blocks, M2M_W * 32, 0, s>>>(c->level_cells.p + a, n, c->child8.p, c->cnchild.p,
                                                            nullptr, c->bg_cen.p, c->bg_mom.p);
    }
    double *tab = c->bg_tab.p, *mcoef = c->bg_tab.p + (HOT_MAXLEVEL + 2) * NC2;
    HOT_COUNT_LAUNCH();
    k_bg_cubetab<P2><<<hot_blocks((HOT_MAXLEVEL + 2) * NC2, 128), 128, 0, s>>>(c->frame.p, c->bg_rho.p, tab, mcoef);
    HOT_COUNT_LAUNCH();
    k_bg_records<P, T><<<hot_blocks(ncube, 128), 128, 0, s>>>(nc, ncube, c->bg_cen.p, c->bg_half.p, c->clevel.p,
                                                              c->bg_eparent.p, tab, mcoef, c->bg_mom.p, c->bg_q.p,
                                                              c->prm.G, c->prm.eps, HOT_REC_LEN[P], rec);
    return HOT_OK;
}

// Number of empty octants (synchronises: it sizes the record array) and the cubes' geometry.
int bg_prepare(hot_ctx *c)
{
    cudaStream_t s = c->st;
    const int64_t nc = c->ncell;
    HOT_CK(c->bg_ecnt.ensure(nc + 1, s));
    HOT_CK(c->bg_eoff.ensure(nc + 1, s));
    HOT_CK(c->bg_rho.ensure(1, s));
    HOT_CK(c->scan_tmp.ensure(hot_scan_tmp_elems(nc + 64), s));
    HOT_COUNT_LAUNCH();
    k_bg_ecount<<<hot_blocks(nc, 256), 256, 0, s>>>(c->cnchild.p, nc, c->bg_ecnt.p);
    int r = hot_scan_u32_to_u32(c->bg_ecnt.p, c->bg_eoff.p, nc, c->scan_tmp.p, s);
    if (r) return r;
    uint32_t ne = 0;
    HOT_CK(cudaMemcpyAsync(&ne, c->bg_eoff.p + nc, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    HOT_CK(cudaStreamSynchronize(s));
    c->n_empty = ne;
    HOT_CK(c->bg_cen.ensure(3 * (size_t)(nc + ne), s));
    HOT_CK(c->bg_half.ensure(nc + ne + 1, s));
    HOT_COUNT_LAUNCH();
    k_bg_geom<<<hot_blocks(nc, 128), 128, 0, s>>>(c->ckey.p, c->clevel.p, nc, c->frame.p, c->cmass.p, c->bg_cen.p,
                                                  c->bg_half.p, c->bg_rho.p);
    return HOT_OK;
}

template <int P>
int moments_p(hot_ctx *c)
{
    constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
    cudaStream_t s = c->st;
    const int64_t ncell = c->ncell, N = c->N;
    HOT_CK(c->cmass.ensure(ncell, s));
    HOT_CK(c->ccom.ensure(3 * (size_t)ncell, s));
    HOT_CK(c->cmom.ensure((size_t)NC * ncell, s));
    HOT_CK(c->cbmax.ensure(ncell, s));
    HOT_CK(c->cB1.ensure(ncell, s));
    HOT_CK(c->cB2.ensure(ncell, s));
    HOT_CK(c->prel.ensure(N, s));
    const int grid = c->nsm * 8;
    HOT_COUNT_LAUNCH();
    if (c->prm.precision == HOT_FP64)
        k_p2m_leaf<P, double><<<grid, MW * 32, 0, s>>>(c->cbegin.p, c->ccount.p, c->cnchild.p, ncell, c->spos.p,
                                                       c->smass.p, c->cmass.p, c->ccom.p, c->cmom.p, c->cbmax.p,
                                                       c->cB1.p, c->cB2.p, c->prel.p);
    else
        k_p2m_leaf<P, float><<<grid, MW * 32, 0, s>>>(c->cbegin.p, c->ccount.p, c->cnchild.p, ncell, c->spos.p,
                                                      c->smass.p, c->cmass.p, c->ccom.p, c->cmom.p, c->cbmax.p,
                                                      c->cB1.p, c->cB2.p, c->prel.p);
    {
        // runs of levels of at most COM_ONE cells in one single-block launch each, larger
        // levels in a launch of their own
        constexpr int64_t COM_ONE = 1024;
        const int64_t *levoff = c->sizes.p + 24;  // the build's level offsets on the device
        int hi = (int)c->maxlevel;               // the run is levels [l + 1, hi)
        for (int l = (int)c->maxlevel - 1; l >= -1; --l) {
            const int64_t n = l >= 0 ? c->level_off[l + 1] - c->level_off[l] : 0;
            if (l >= 0 && n <= COM_ONE) continue;  // joins the run
            if (hi > l + 1) {
                HOT_COUNT_LAUNCH();
                k_com_levels<<<1, 1024, 0, s>>>(c->level_cells.p, levoff, l + 1, hi, c->child8.p, c->cnchild.p,
                                                c->cmass.p, c->ccom.p);
            }
            if (l >= 0) {
                const int64_t a = c->level_off[l];
                HOT_COUNT_LAUNCH();
                k_com_level<<<hot_blocks(n, 128), 128, 0, s>>>(c->level_cells.p + a, n, c->child8.p, c->cnchild.p,
                                                               c->cmass.p, c->ccom.p);
            }
            hi = l;
        }
    }
    // the moment translations, and later the records, on the second stream beside the
    // aggregates (and the traversal that follows), except under background subtraction and
    // order selection, whose later steps read the moments here
    const bool fork = !c->prm.background && !(c->prm.p_min >= 0 && c->prm.p_min < P);
    const int reclen = HOT_REC_LEN[P];
    const int64_t max_items = ncell + N * (c->maxlevel + 1) / CHUNK + 1;
    HOT_CK(c->item_off.ensure(ncell + 1, s));
    HOT_CK(c->item_cell.ensure(max_items, s));
    HOT_CK(c->item_part.ensure(3 * (size_t)max_items, s));
    HOT_CK(c->gflag.ensure(ncell + 1, s));
    HOT_CK(c->scan_tmp.ensure(hot_scan_tmp_elems(ncell + 64), s));
    if (fork) {
        if (c->prm.precision == HOT_FP64)
            HOT_CK(c->rec64.ensure((size_t)reclen * ncell, s));
        else
            HOT_CK(c->rec32.ensure((size_t)reclen * ncell, s));
        HOT_CK(cudaEventRecord(c->ev_mfork, s));
        HOT_CK(cudaStreamWaitEvent(c->st2, c->ev_mfork, 0));
    }
    cudaStream_t ms = fork ? c->st2 : s;
    for (int l = (int)c->maxlevel - 1; l >= 0; --l) {
        int64_t a = c->level_off[l], n = c->level_off[l + 1] - a;
        if (n <= 0) continue;
        const int blocks = (int)(n < (int64_t)c->nsm * 8 ? n : (int64_t)c->nsm * 8);
        HOT_COUNT_LAUNCH();
        k_m2m_level<P><<<blocks, M2M_W * 32, 0, ms>>>(c->level_cells.p + a, n, c->child8.p, c->cnchild.p,
                                                      c->cmass.p, c->ccom.p, c->cmom.p);
    }
    // the expansion's kernel: Plummer-softened, or Newtonian under K1 or spline smoothing
    // (whose kernels differ from 1/r only inside eps, which accepted cells keep clear of)
    const double eps_rec = c->prm.softening != HOT_SOFT_PLUMMER ? 0.0 : c->prm.eps;
    // aggregates of inner cells
    HOT_COUNT_LAUNCH();
    k_item_count<<<hot_blocks(ncell, 256), 256, 0, s>>>(c->ccount.p, c->cnchild.p, ncell, c->gflag.p);
    int r = hot_scan_u32_to_u32(c->gflag.p, c->item_off.p, ncell, c->scan_tmp.p, s);
    if (r) {
        if (fork && cudaEventRecord(c->ev_mjoin, ms) == cudaSuccess) c->mom_pending = true;
        return r;
    }
    HOT_COUNT_LAUNCH();
    k_item_cells<<<hot_blocks(ncell, 256), 256, 0, s>>>(c->item_off.p, ncell, c->item_cell.p);
    HOT_COUNT_LAUNCH();
    k_item_part<P><<<c->nsm * 16, MW * 32, 0, s>>>(c->item_cell.p, c->item_off.p, c->item_off.p + ncell,
                                                   c->cbegin.p, c->ccount.p, c->ccom.p, c->spos.p, c->smass.p,
                                                   c->item_part.p);
    HOT_COUNT_LAUNCH();
    k_item_combine<<<hot_blocks(ncell * 32, 256), 256, 0, s>>>(c->item_off.p, c->cnchild.p, ncell, c->item_part.p,
                                                          c->cbmax.p, c->cB1.p, c->cB2.p);
    // records (under background subtraction also those of the cells' contrasts and of the
    // empty octants, after the cells' own); they need the aggregates' b_max
    c->reclen = reclen;
    if (fork) {
        HOT_CK(cudaEventRecord(c->ev_mcomb, s));
        HOT_CK(cudaStreamWaitEvent(ms, c->ev_mcomb, 0));
    }
    int64_t nrec = ncell;
    if constexpr (P <= HOT_BG_PMAX) {
        if (c->prm.background) {
            r = bg_prepare(c);
            if (r) return r;
            nrec = 2 * ncell + c->n_empty;
        }
    }
    if (c->prm.precision == HOT_FP64) {
        if (!fork) HOT_CK(c->rec64.ensure((size_t)reclen * nrec, s));
        HOT_COUNT_LAUNCH();
        k_records<P, double><<<hot_blocks(ncell, 128), 128, 0, ms>>>(c->cmom.p, c->ccom.p, c->cbmax.p, c->clevel.p, ncell, c->frame.p,
                                                                    c->prm.G, eps_rec, reclen, NC, c->rec64.p);
    } else {
        if (!fork) HOT_CK(c->rec32.ensure((size_t)reclen * nrec, s));
        HOT_COUNT_LAUNCH();
        k_records<P, float><<<hot_blocks(ncell, 128), 128, 0, ms>>>(c->cmom.p, c->ccom.p, c->cbmax.p, c->clevel.p, ncell, c->frame.p,
                                                                   c->prm.G, eps_rec, reclen, NC, c->rec32.p);
    }
    if (fork) {
        HOT_CK(cudaEventRecord(c->ev_mjoin, ms));
        c->mom_pending = true;
    }
    if constexpr (P <= HOT_BG_PMAX) {
        if (c->prm.background) {
            r = c->prm.precision == HOT_FP64 ? bg_records<P, double>(c, c->rec64.p)
                                             : bg_records<P, float>(c, c->rec32.p);
            if (r) return r;
        }
    }
    // per-interaction order selection: B_n of every cell and the records of orders p_min..p-1
    c->varq = c->prm.p_min >= 0 && c->prm.p_min < P;
    c->q_lo = c->varq ? c->prm.p_min : P;
    if (c->varq) {
        constexpr int NB = P + 3;
        HOT_CK(c->bn_cnt.ensure(ncell + 1, s));
        HOT_CK(c->bn_off.ensure(ncell + 1, s));
        HOT_CK(c->bn_cell.ensure(max_items, s));
        HOT_CK(c->bn_part.ensure((size_t)NB * max_items, s));
        HOT_CK(c->cBn.ensure((size_t)NB * ncell, s));
        HOT_COUNT_LAUNCH();
        k_bn_count<<<hot_blocks(ncell, 256), 256, 0, s>>>(c->ccount.p, ncell, c->bn_cnt.p);
        r = hot_scan_u32_to_u32(c->bn_cnt.p, c->bn_off.p, ncell, c->scan_tmp.p, s);
        if (r) return r;
        HOT_COUNT_LAUNCH();
        k_item_cells<<<hot_blocks(ncell, 256), 256, 0, s>>>(c->bn_off.p, ncell, c->bn_cell.p);
        HOT_COUNT_LAUNCH();
        k_bn_part<P><<<c->nsm * 16, MW * 32, 0, s>>>(c->bn_cell.p, c->bn_off.p, c->bn_off.p + ncell, c->cbegin.p,
                                                     c->ccount.p, c->ccom.p, c->spos.p, c->smass.p, c->bn_part.p);
        HOT_COUNT_LAUNCH();
        k_bn_combine<<<hot_blocks(ncell * NB * 32, 256), 256, 0, s>>>(c->bn_off.p, ncell, NB, c->bn_part.p, c->cBn.p);
        for (int q = c->q_lo; q < P; ++q) {
            if (c->prm.precision == HOT_FP64) {
                HOT_CK(c->rec64q[q].ensure((size_t)HOT_REC_LEN[q] * ncell, s));
                r = records_of_order<double>(c, q, NC, eps_rec, c->rec64q[q].p);
            } else {
                HOT_CK(c->rec32q[q].ensure((size_t)HOT_REC_LEN[q] * ncell, s));
                r = records_of_order<float>(c, q, NC, eps_rec, c->rec32q[q].p);
            }
            if (r) return r;
        }
    }
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}

}  // namespace

int hot_impl_moments(hot_ctx *c, int p)
{
    hot_tic(c, 2);
    int r;
    switch (p) {
        case 0: r = moments_p<0>(c); break;
        case 1: r = moments_p<1>(c); break;
        case 2: r = moments_p<2>(c); break;
        case 3: r = moments_p<3>(c); break;
        case 4: r = moments_p<4>(c); break;
        case 5: r = moments_p<5>(c); break;
        case 6: r = moments_p<6>(c); break;
        case 7: r = moments_p<7>(c); break;
        case 8: r = moments_p<8>(c); break;
        default: return HOT_EINVAL;
    }
    hot_toc(c, 2);
    if (r == HOT_OK) {
        c->p_mom = p;
        c->stage = 2;
    }
    return r;
}
