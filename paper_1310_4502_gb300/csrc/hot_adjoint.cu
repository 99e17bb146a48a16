// hot_adjoint.cu -- adjoint of the tree force through frozen lists and frozen
// expansion centres: for L = sum_i u_i . a_i + v_i phi_i, dL/dx and dL/dm of every
// particle, where each cell's moments stay functions of its particles' positions and
// masses (moment tensor definition, about the frozen centre).
//
//   sink side    : d/dx_i of every interaction of sink i -- the forward-mode derivative
//                  of the M2P routine along u_i (the Hessian of the expansion applied to
//                  u_i) minus v_i a_i, and the P2P pair terms (interaction kernel, MODE 1)
//   source, M2P  : the interactions are linear in a cell's record coefficients, so
//                  dL/dC accumulates A y^b + B D_u(y^b) over every (sink, cell) pair; the
//                  lists are transposed (cell -> groups) by a stable radix sort so that
//                  each cell's sum is formed by one warp per chunk, in a fixed order;
//                  then dL/dM = (record map)^T dL/dC, pushed down the tree with the
//                  transposed binomial translation and onto the particles with the
//                  transposed P2M at the leaves (float64)
//   source, P2P  : the pair terms seen from the source particle, over the transposed
//                  (leaf -> groups) lists, one warp per leaf
// Every sum has a fixed order: results are reproducible run to run.
#include <type_traits>

#include "hot_common.cuh"
#include "generated.cuh"

namespace {

constexpr int AW = 4;    // warps per block
constexpr int KG = 32;   // groups per source-side work item

template <int P, class T>
struct ACfg {
    static constexpr int RL = HOT_REC_LEN[P];
    static constexpr int NS = HOT_NS[P];
    static constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
};

// Sorted-order sink weights (u, v) and float hi/lo positions.
template <class T>
__global__ void k_adj_prep(const double *__restrict__ g_acc, const double *__restrict__ g_pot,
                           const uint32_t *__restrict__ perm, const double *__restrict__ spos, int64_t N,
                           T *__restrict__ w, float *__restrict__ xhl)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int64_t i = perm[s];
    w[4 * s + 0] = (T)g_acc[3 * i + 0];
    w[4 * s + 1] = (T)g_acc[3 * i + 1];
    w[4 * s + 2] = (T)g_acc[3 * i + 2];
    w[4 * s + 3] = g_pot ? (T)g_pot[i] : T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double x = spos[3 * s + d];
        const float hi = (float)x;
        xhl[8 * s + d] = hi;
        xhl[8 * s + 4 + d] = (float)(x - (double)hi);
    }
}

// (key = target cell, value = group) for every entry of a CSR list, in list order.
__global__ void k_expand_pairs(const int64_t *__restrict__ off, const int32_t *__restrict__ list, int64_t ng,
                               uint64_t *__restrict__ key, uint32_t *__restrict__ val)
{
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= ng) return;
    for (int64_t e = off[g] + lane_id(); e < off[g + 1]; e += 32) {
        key[e] = (uint64_t)(uint32_t)list[e];
        val[e] = (uint32_t)g;
    }
}

// Range [start, end) of every target in the sorted pair array.
__global__ void k_ranges(const uint64_t *__restrict__ key, int64_t n, int64_t *__restrict__ start,
                         int64_t *__restrict__ end)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint64_t k = key[e];
    if (e == 0 || key[e - 1] != k) start[k] = e;
    if (e == n - 1 || key[e + 1] != k) end[k] = e + 1;
}

__global__ void k_item_count_adj(const int64_t *__restrict__ start, const int64_t *__restrict__ end, int64_t ncell,
                                 uint32_t *__restrict__ cnt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    cnt[c] = (uint32_t)((end[c] - start[c] + KG - 1) / KG);
}

__global__ void k_item_fill_adj(const int64_t *__restrict__ start, const int64_t *__restrict__ end,
                                const uint32_t *__restrict__ ioff, int64_t ncell, int32_t *__restrict__ icell,
                                int64_t *__restrict__ ia, int64_t *__restrict__ ib)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int64_t a = start[c];
    const int64_t e = end[c];
    for (uint32_t it = ioff[c]; it < ioff[c + 1]; ++it) {
        icell[it] = (int32_t)c;
        ia[it] = a;
        ib[it] = a + KG < e ? a + KG : e;
        a += KG;
    }
}

// Partial rows of the P2P source side: a leaf with entries gets (its items) x (its
// particles) rows.
__global__ void k_item_rows(const int64_t *__restrict__ start, const int64_t *__restrict__ end,
                            const int32_t *__restrict__ ccount, const int32_t *__restrict__ cnchild, int64_t ncell,
                            uint32_t *__restrict__ rows)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int64_t ne = end[c] - start[c];
    rows[c] = (cnchild[c] != 0 || ne <= 0) ? 0u : (uint32_t)(((ne + KG - 1) / KG) * (int64_t)ccount[c]);
}

// Source side of M2P: one warp per item (one cell, up to KG groups that list it), taken
// from a work counter in the given order (largest first); the sinks of all the item's
// groups are spread over the lanes.  Each lane accumulates the
// coefficient adjoints in registers; the warp sum goes to part[item].
// At p = 6 the 130 coefficient adjoints a lane accumulates fill every register; capped at
// 168 (3 CTAs per SM) the kernel spills a few bytes and runs 6% faster than at 255 (and
// 15% faster than at 4 CTAs).  At p <= 4 (float) 4 CTAs per SM fit without spills and run
// 8% faster than 1-3 (clustered 2^20).
template <int P, class T>
__global__ void __launch_bounds__(AW * 32, P >= 6 ? 3 : (P <= 4 && sizeof(T) == 4 ? 4 : 1)) k_adj_src(
    const uint32_t *__restrict__ nitem_p, const int32_t *__restrict__ icell, const int64_t *__restrict__ ia,
    const int64_t *__restrict__ ib, const uint32_t *__restrict__ tval, const int32_t *__restrict__ gcell,
    const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount, const T *__restrict__ rec,
    const T *__restrict__ w, const float *__restrict__ xhl, const double *__restrict__ spos,
    const uint32_t *__restrict__ iorder, unsigned *__restrict__ work, T *__restrict__ part)
{
    constexpr int RL = ACfg<P, T>::RL;
    constexpr int NS = ACfg<P, T>::NS;
    __shared__ int32_t sbeg[AW][32], spre[AW][33];
    __shared__ T red[AW][32][33];  // transpose of 32 lanes x 32 coefficients (padded row)
    const int wi = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t nitem = *nitem_p;
    for (;;) {
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(work, 1u);
        const int64_t ii = __shfl_sync(0xffffffffu, i0, 0);
        if (ii >= nitem) break;
        const int64_t it = iorder ? (int64_t)iorder[ii] : ii;
        const int32_t c = icell[it];
        const int64_t a = ia[it], b = ib[it];
        const int ng = (int)(b - a);
        const T *h = rec + (int64_t)c * RL;
        const T is = h[0], e2 = h[1];
        int32_t gb = 0, gn = 0;
        if ((int)lane < ng) {
            const int32_t gcl = gcell[tval[a + lane]];
            gb = cbegin[gcl];
            gn = ccount[gcl];
        }
        const int incl = warp_incl_scan(gn);
        sbeg[wi][lane] = gb;
        spre[wi][lane + 1] = incl;
        if (lane == 0) spre[wi][0] = 0;
        __syncwarp();
        const int total = spre[wi][ng];
        T cb[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) cb[q] = T(0);
        // group of sink t: spre[j] <= t < spre[j+1]; t grows, so j only advances (and
        // stays below ng, as t < total = spre[ng])
        int j = 0;
        for (int t = lane; t < total; t += 32) {
            while (spre[wi][j + 1] <= t) ++j;
            const int64_t s = (int64_t)sbeg[wi][j] + (t - spre[wi][j]);
            T rx, ry, rz, wx, wy, wz, wv;
            if constexpr (sizeof(T) == 4) {
                const float4 hi = reinterpret_cast<const float4 *>(xhl)[2 * s];
                const float4 lo = reinterpret_cast<const float4 *>(xhl)[2 * s + 1];
                rx = (hi.x - h[2]) + (lo.x - h[5]);
                ry = (hi.y - h[3]) + (lo.y - h[6]);
                rz = (hi.z - h[4]) + (lo.z - h[7]);
                const float4 ww = reinterpret_cast<const float4 *>(w)[s];
                wx = ww.x;
                wy = ww.y;
                wz = ww.z;
                wv = ww.w;
            } else {
                rx = spos[3 * s + 0] - h[2];
                ry = spos[3 * s + 1] - h[3];
                rz = spos[3 * s + 2] - h[4];
                wx = w[4 * s + 0];
                wy = w[4 * s + 1];
                wz = w[4 * s + 2];
                wv = w[4 * s + 3];
            }
            m2p_cbar<P, T>(is, e2, rx, ry, rz, wx, wy, wz, wv, cb);
        }
        // warp sums, 32 coefficients at a time through shared memory: lane l writes its
        // row, then sums column l (the 32 lanes' values of coefficient c0 + l, in lane order)
#pragma unroll
        for (int c0 = 0; c0 < NS; c0 += 32) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (c0 + q < NS) red[wi][lane][q] = cb[c0 + q];
            __syncwarp();
            if (c0 + (int)lane < NS) {
                T v = T(0);
#pragma unroll 8
                for (int l = 0; l < 32; ++l) v += red[wi][l][lane];
                part[it * NS + c0 + lane] = v;
            }
            __syncwarp();
        }
    }
}

// dL/dC of every cell = sum of its items (fixed order, float64), then dL/dM through the
// transposed record map.  One thread per cell; Mbar must be zero on entry.
template <int P, class T>
__global__ void __launch_bounds__(AW * 32) k_adj_cells(int64_t ncell, const uint32_t *__restrict__ ioff,
                                                       const T *__restrict__ part, const T *__restrict__ rec,
                                                       double G, double *__restrict__ Mbar)
{
    // One warp per cell: the lanes sum the coefficient adjoints of the cell's items
    // (coalesced rows, FP64, items in order), then each lane gathers the moment
    // adjoints it owns through the record-adjoint table (terms in a fixed order).
    constexpr int RL = ACfg<P, T>::RL;
    constexpr int NS = ACfg<P, T>::NS;
    constexpr int NC = ACfg<P, T>::NC;
    constexpr int NE = 2 * P + 2;
    __shared__ double scb[AW][NS];
    __shared__ double sip[AW][NE];
    const int wi = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * AW;
    for (int64_t c = (int64_t)blockIdx.x * AW + wi; c < ncell; c += nw) {
        const uint32_t i0 = ioff[c], i1 = ioff[c + 1];
        if (i0 == i1) continue;
        for (int q = lane; q < NS; q += 32) {
            double t = 0.0;
            for (uint32_t it = i0; it < i1; ++it) t += (double)part[(int64_t)it * NS + q];
            scb[wi][q] = t;
        }
        if (lane == 0) {
            const double inv_s = (double)rec[c * (int64_t)RL];
            double v = 1.0;
            for (int e = 0; e < NE; ++e) {
                sip[wi][e] = v;
                v *= inv_s;
            }
        }
        __syncwarp();
        for (int a = lane; a < NC; a += 32) {
            double t = 0.0;
            const int j0 = radj_start[RADJ_SBASE[P] + a], j1 = radj_start[RADJ_SBASE[P] + a + 1];
            for (int j = j0; j < j1; ++j) t += radj_f[j] * sip[wi][radj_e[j]] * scb[wi][radj_q[j]];
            Mbar[c * NC + a] = G * t;
        }
        __syncwarp();
    }
}

// Top-down: dL/dM of a cell += transposed translation of its parent's dL/dM
// (M_parent = sum_children shift(M_child) with frozen centres).  One warp per cell of
// the level; the parent level is complete.
template <int P>
__global__ void __launch_bounds__(AW * 32) k_adj_l2l(const int32_t *__restrict__ cells, int64_t n,
                                                     const int32_t *__restrict__ cparent,
                                                     const double *__restrict__ ccom, double *__restrict__ Mbar)
{
    constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
    __shared__ double sd[AW][NC], sp[AW][NC];
    __shared__ unsigned char mi[NC][3];
    for (int k = threadIdx.x; k < NC; k += blockDim.x) {
        mi[k][0] = hot_midx[k][0];
        mi[k][1] = hot_midx[k][1];
        mi[k][2] = hot_midx[k][2];
    }
    __syncthreads();
    const int wi = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * AW;
    for (int64_t q0 = (int64_t)blockIdx.x * AW + wi; q0 < n; q0 += nw) {
        const int32_t c = cells[q0];
        const int32_t p = cparent[c];
        if (p < 0) continue;
        const double d[3] = {ccom[3 * (int64_t)c + 0] - ccom[3 * (int64_t)p + 0],
                             ccom[3 * (int64_t)c + 1] - ccom[3 * (int64_t)p + 1],
                             ccom[3 * (int64_t)c + 2] - ccom[3 * (int64_t)p + 2]};
        for (int g = lane; g < NC; g += 32) {
            double v = 1.0;
            for (int e = 0; e < 3; ++e)
                for (int t = 0; t < mi[g][e]; ++t) v *= d[e];
            sd[wi][g] = v;
            sp[wi][g] = Mbar[(int64_t)p * NC + g];
        }
        __syncwarp();
        for (int b = lane; b < NC; b += 32) {
            double t = 0.0;
            // the table is of order 6; for each b its alpha run in canonical order, so the
            // ones of this order (alpha < NC) come first
            for (int j = m2mt_start[b]; j < m2mt_start[b + 1] && m2mt_alpha[j] < NC; ++j)
                t += m2mt_coef[j] * sd[wi][m2mt_gamma[j]] * sp[wi][m2mt_alpha[j]];
            Mbar[(int64_t)c * NC + b] += t;
        }
        __syncwarp();
    }
}

// Source side of P2P: work items of one leaf and up to KG of the groups that list it (a
// leaf in a dense region is listed by thousands of groups, so whole leaves would leave
// a long tail).  One warp per item, taken from a work counter; lanes = leaf particles
// (two per lane when the leaf has more than 32, otherwise one per lane with the staged
// sinks split across the spare lanes).  The sinks of the item's groups are staged PS at
// a time, all their loads in flight together (a scan of the group sizes, then every lane
// loads sinks of the batch).  Per item and leaf particle the sums
//   gx = sum_i [u_i/s^3 - 3 d (d.u_i)/s^5 + v_i d/s^3],  gm = sum_i [u_i.d/s^3 - v_i/s]
// (d = x_j - x_i, s^2 = |d|^2 + eps^2; with K1 smoothing f u_i + (f2 (d.u_i) + v_i f) d and
// (d.u_i) f - v_i psi, the pair functions of k1_pair or spline_pair) go to row roff[leaf] + k n_leaf + j of part (k:
// the item's rank within its leaf); k_adj_p2p_combine adds the items of each leaf in
// order: dL/dx_j += G m_j gx, dL/dm_j += G gm.
constexpr int PS = 128;
constexpr int LMAX = 64;  // leaf particles per pass (two per lane)
// (5 CTAs per SM: 94 registers without spills, 1% faster at 2^18 and 2^20 than the
// compiler's 80 registers with spills at 6)
template <class T, int SOFT>
__global__ void __launch_bounds__(AW * 32, 5) k_adj_p2p_src(
    const uint32_t *__restrict__ nitem_p, const int32_t *__restrict__ icell, const int64_t *__restrict__ ia,
    const int64_t *__restrict__ ib, const uint32_t *__restrict__ tval, const int32_t *__restrict__ gcell,
    const int32_t *__restrict__ cbegin, const int32_t *__restrict__ ccount, const int32_t *__restrict__ cend,
    const double *__restrict__ ccom, const double *__restrict__ spos, const double *__restrict__ smass,
    const float4 *__restrict__ prel, const float *__restrict__ xhl, const T *__restrict__ w, T eps2,
    const uint32_t *__restrict__ ioff,
    const int64_t *__restrict__ roff, unsigned *__restrict__ work, T *__restrict__ part)
{
    __shared__ T ss[AW][PS][4];
    __shared__ T sw[AW][PS][4];
    __shared__ int32_t sid[AW][PS];
    __shared__ int32_t sex[AW][33], sgb[AW][32];
    __shared__ double red[AW][32][4];
    const int wi = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t nitem = *nitem_p;
    SoftConst<T> kc{};
    if constexpr (SOFT != HOT_SOFT_PLUMMER) kc = soft_const(eps2);
    for (;;) {
        unsigned I0 = 0;
        if (lane == 0) I0 = atomicAdd(work, 1u);
        const int64_t it = __shfl_sync(0xffffffffu, I0, 0);
        if (it >= nitem) break;
        const int64_t L = icell[it];
        const int64_t ea = ia[it], eb = ib[it];
        const int64_t lb = cbegin[L];
        T *pout = part + (roff[L] + (it - (int64_t)ioff[L]) * (int64_t)ccount[L]) * 4;
        const int lc = ccount[L];
        const double zx = ccom[3 * L + 0], zy = ccom[3 * L + 1], zz = ccom[3 * L + 2];
        const float zhi[3] = {(float)zx, (float)zy, (float)zz};
        const float zlo[3] = {(float)(zx - (double)zhi[0]), (float)(zy - (double)zhi[1]), (float)(zz - (double)zhi[2])};
        for (int j0 = 0; j0 < lc; j0 += LMAX) {
            const int nj = lc - j0 < LMAX ? lc - j0 : LMAX;
            const bool two = nj > 32;
            const int nsplit = two ? 1 : 32 / nj;
            const int jj = two ? (int)lane : (int)lane % nj, sj = two ? 0 : (int)lane / nj;
            const bool active = sj < nsplit;
            bool val[2];
            int64_t slot[2];
            T xj[2][3], mj[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int jq = jj + 32 * q;
                val[q] = active && jq < nj && (q == 0 || two);
                slot[q] = lb + j0 + (val[q] ? jq : 0);
                if constexpr (sizeof(T) == 4) {
                    const float4 v = prel[slot[q]];
                    xj[q][0] = v.x;
                    xj[q][1] = v.y;
                    xj[q][2] = v.z;
                    mj[q] = v.w;
                } else {
                    xj[q][0] = spos[3 * slot[q] + 0] - zx;
                    xj[q][1] = spos[3 * slot[q] + 1] - zy;
                    xj[q][2] = spos[3 * slot[q] + 2] - zz;
                    mj[q] = smass[slot[q]];
                }
            }
            T gx[2] = {0, 0}, gy[2] = {0, 0}, gz[2] = {0, 0}, gm[2] = {0, 0};
            // float32 with Plummer smoothing: batches without self or zero-distance pairs take
            // two sinks per instruction (paired float32 arithmetic) against each of the lane's
            // sources, the sinks staged pair-interleaved (x0 x1 y0 y1 z0 z1 . . and
            // ux0 ux1 uy0 uy1 uz0 uz1 v0 v1)
            constexpr bool PAIRED = sizeof(T) == 4 && SOFT == HOT_SOFT_PLUMMER;
            // the self pair, or a zero separation, can only occur in a batch holding the group
            // whose cell contains this leaf, or when eps = 0: other batches skip the tests
            auto flush = [&](int fill, bool checked) {
                __syncwarp();
                if constexpr (PAIRED) {
                    if (active && !checked) {
                        const int npair = (fill + 1) >> 1;
                        const float4 *s2 = reinterpret_cast<const float4 *>(&ss[wi][0][0]);
                        const float4 *w4 = reinterpret_cast<const float4 *>(&sw[wi][0][0]);
                        const float2 e22 = make_float2(eps2, eps2), neg1 = make_float2(-1.f, -1.f),
                                     neg3 = make_float2(-3.f, -3.f);
                        float2 xq[2][3], gx2[2], gy2[2], gz2[2], gm2[2];
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
#pragma unroll
                            for (int d = 0; d < 3; ++d) xq[q][d] = make_float2(xj[q][d], xj[q][d]);
                            gx2[q] = gy2[q] = gz2[q] = gm2[q] = make_float2(0.f, 0.f);
                        }
#pragma unroll 2
                        for (int jp = sj; jp < npair; jp += nsplit) {
                            const float4 a = s2[2 * jp], b = s2[2 * jp + 1], c = w4[2 * jp], d = w4[2 * jp + 1];
                            const float2 sx = make_float2(a.x, a.y), sy = make_float2(a.z, a.w), sz = make_float2(b.x, b.y);
                            const float2 ux = make_float2(c.x, c.y), uy = make_float2(c.z, c.w), uz = make_float2(d.x, d.y);
                            const float2 vv = make_float2(d.z, d.w);
                            const float2 nv = __fmul2_rn(vv, neg1);
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                if (!val[q]) continue;
                                const float2 dx = __ffma2_rn(sx, neg1, xq[q][0]), dy = __ffma2_rn(sy, neg1, xq[q][1]),
                                             dz = __ffma2_rn(sz, neg1, xq[q][2]);
                                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, e22)));
                                const float2 ri = make_float2(hot_rsqrt(r2.x), hot_rsqrt(r2.y));
                                const float2 ri2 = __fmul2_rn(ri, ri);
                                const float2 r3 = __fmul2_rn(ri2, ri);
                                const float2 r5 = __fmul2_rn(r3, ri2);
                                const float2 du = __ffma2_rn(dz, uz, __ffma2_rn(dy, uy, __fmul2_rn(dx, ux)));
                                // cd = v r^-3 - 3 r^-5 (d.u)
                                const float2 cd = __ffma2_rn(vv, r3, __fmul2_rn(__fmul2_rn(r5, du), neg3));
                                gx2[q] = __ffma2_rn(cd, dx, __ffma2_rn(r3, ux, gx2[q]));
                                gy2[q] = __ffma2_rn(cd, dy, __ffma2_rn(r3, uy, gy2[q]));
                                gz2[q] = __ffma2_rn(cd, dz, __ffma2_rn(r3, uz, gz2[q]));
                                gm2[q] = __ffma2_rn(nv, ri, __ffma2_rn(du, r3, gm2[q]));
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            gx[q] += gx2[q].x + gx2[q].y;
                            gy[q] += gy2[q].x + gy2[q].y;
                            gz[q] += gz2[q].x + gz2[q].y;
                            gm[q] += gm2[q].x + gm2[q].y;
                        }
                    }
                    if (!checked) {
                        __syncwarp();
                        return;
                    }
                }
                if (active) {
                    auto sweep = [&](auto ck) {
                        constexpr bool CK = decltype(ck)::value;
#pragma unroll 2
                    for (int k = sj; k < fill; k += nsplit) {
                        const T sx = ss[wi][k][0], sy = ss[wi][k][1], sz = ss[wi][k][2];
                        const T ux = sw[wi][k][0], uy = sw[wi][k][1], uz = sw[wi][k][2], vv = sw[wi][k][3];
                        const int32_t id = CK ? sid[wi][k] : 0;
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            if (!val[q]) continue;
                            const T dx = xj[q][0] - sx, dy = xj[q][1] - sy, dz = xj[q][2] - sz;
                            if constexpr (SOFT != HOT_SOFT_PLUMMER) {
                                const T r2 = dx * dx + dy * dy + dz * dz;
                                T f, f2, psi;
                                compact_pair<SOFT>(r2, kc, f, f2, psi);
                                if constexpr (CK) {
                                    const bool ok = (r2 > T(0) || kc.e2 > T(0)) && (id != (int32_t)slot[q]);
                                    f = ok ? f : T(0);
                                    f2 = ok ? f2 : T(0);
                                    psi = ok ? psi : T(0);
                                }
                                const T du = dx * ux + dy * uy + dz * uz;
                                const T cd = f2 * du + vv * f;
                                gx[q] += f * ux + cd * dx;
                                gy[q] += f * uy + cd * dy;
                                gz[q] += f * uz + cd * dz;
                                gm[q] += du * f - vv * psi;
                                continue;
                            }
                            const T r2 = dx * dx + dy * dy + dz * dz + eps2;
                            T ri;
                            if constexpr (CK) {
                                const bool ok = (r2 > T(0)) && (id != (int32_t)slot[q]);
                                ri = ok ? hot_rsqrt(r2) : T(0);
                            } else {
                                ri = hot_rsqrt(r2);
                            }
                            const T r3 = ri * ri * ri;
                            const T du = dx * ux + dy * uy + dz * uz;
                            const T c1 = T(3) * r3 * ri * ri * du;
                            gx[q] += r3 * ux - c1 * dx + vv * r3 * dx;
                            gy[q] += r3 * uy - c1 * dy + vv * r3 * dy;
                            gz[q] += r3 * uz - c1 * dz + vv * r3 * dz;
                            gm[q] += du * r3 - vv * ri;
                        }
                    }
                    };
                    if (checked)
                        sweep(std::true_type{});
                    else
                        sweep(std::false_type{});
                }
                __syncwarp();
            };
            for (int64_t e0 = ea; e0 < eb; e0 += 32) {
                const int ne = (int)(eb - e0 < 32 ? eb - e0 : 32);
                int32_t gb = 0, gn = 0;
                bool own = false;
                if ((int)lane < ne) {
                    const int32_t gc = gcell[tval[e0 + lane]];
                    gb = cbegin[gc];
                    gn = ccount[gc];
                    own = L >= gc && L < cend[gc];
                }
                // a chunk holding a group that contains L is staged in two passes: the other
                // groups' sinks first, without the per-pair tests, then that group's with them
                const bool anyown = __any_sync(0xffffffffu, own);
                for (int pass = anyown ? 0 : 1; pass < 2; ++pass) {
                    const bool mine = !anyown || (own == (pass == 1));
                    const bool checked = (anyown && pass == 1) || !(eps2 > T(0));
                    const int incl = warp_incl_scan(mine ? gn : 0);
                    const int tot = __shfl_sync(0xffffffffu, incl, 31);
                    sex[wi][lane + 1] = incl;
                    if (lane == 0) sex[wi][0] = 0;
                    sgb[wi][lane] = gb;
                    __syncwarp();
                    for (int t0 = 0; t0 < tot; t0 += PS) {
                        const int take = tot - t0 < PS ? tot - t0 : PS;
                        for (int u = lane; u < take; u += 32) {
                            const int t = t0 + u;
                            int lo = 0, hi = ne;  // entry with sex[lo] <= t < sex[lo + 1]
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (sex[wi][mid] <= t)
                                    lo = mid;
                                else
                                    hi = mid;
                            }
                            const int64_t s = (int64_t)sgb[wi][lo] + (t - sex[wi][lo]);
                            if constexpr (sizeof(T) == 4) {
                                const float px = (xhl[8 * s + 0] - zhi[0]) + (xhl[8 * s + 4] - zlo[0]);
                                const float py = (xhl[8 * s + 1] - zhi[1]) + (xhl[8 * s + 5] - zlo[1]);
                                const float pz = (xhl[8 * s + 2] - zhi[2]) + (xhl[8 * s + 6] - zlo[2]);
                                if (PAIRED && !checked) {
                                    float *qs = &ss[wi][0][0] + 8 * (u >> 1) + (u & 1);
                                    float *qw = &sw[wi][0][0] + 8 * (u >> 1) + (u & 1);
                                    qs[0] = px;
                                    qs[2] = py;
                                    qs[4] = pz;
#pragma unroll
                                    for (int d = 0; d < 4; ++d) qw[2 * d] = w[4 * s + d];
                                    sid[wi][u] = (int32_t)s;
                                    continue;
                                }
                                ss[wi][u][0] = px;
                                ss[wi][u][1] = py;
                                ss[wi][u][2] = pz;
                            } else {
                                ss[wi][u][0] = spos[3 * s + 0] - zx;
                                ss[wi][u][1] = spos[3 * s + 1] - zy;
                                ss[wi][u][2] = spos[3 * s + 2] - zz;
                            }
#pragma unroll
                            for (int d = 0; d < 4; ++d) sw[wi][u][d] = w[4 * s + d];
                            sid[wi][u] = (int32_t)s;
                        }
                        if constexpr (PAIRED) {
                            if (!checked && (take & 1) && lane == 0) {
                                // the partner of the last sink: far away, with zero weights (its terms are 0)
                                float *qs = &ss[wi][0][0] + 8 * (take >> 1) + 1;
                                float *qw = &sw[wi][0][0] + 8 * (take >> 1) + 1;
                                qs[0] = qs[2] = qs[4] = 1e17f;
                                qw[0] = qw[2] = qw[4] = qw[6] = 0.f;
                            }
                        }
                        flush(take, checked);
                    }
                }
            }
            if (two) {
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    if (val[q]) {
                        T *o = pout + 4 * (int64_t)(slot[q] - lb);
                        o[0] = gx[q];
                        o[1] = gy[q];
                        o[2] = gz[q];
                        o[3] = gm[q];
                    }
            } else {
                if (active) {
                    red[wi][lane][0] = (double)gx[0];
                    red[wi][lane][1] = (double)gy[0];
                    red[wi][lane][2] = (double)gz[0];
                    red[wi][lane][3] = (double)gm[0];
                }
                __syncwarp();
                if (active && sj == 0) {
                    double t[4] = {0, 0, 0, 0};
                    for (int q = 0; q < nsplit; ++q)
                        for (int d = 0; d < 4; ++d) t[d] += red[wi][jj + q * nj][d];
                    T *o = pout + 4 * (int64_t)(slot[0] - lb);
                    for (int d = 0; d < 4; ++d) o[d] = (T)t[d];
                }
            }
            __syncwarp();
        }
    }
}

// dL/dx_j, dL/dm_j of the P2P source side: the partial sums of a leaf's items, added in
// item order (float64).  One warp per leaf, lanes over its particles.
template <class T>
__global__ void __launch_bounds__(AW * 32) k_adj_p2p_combine(int64_t ncell, const int32_t *__restrict__ cnchild,
                                                             const uint32_t *__restrict__ ioff,
                                                             const int64_t *__restrict__ roff,
                                                             const int32_t *__restrict__ cbegin,
                                                             const int32_t *__restrict__ ccount,
                                                             const double *__restrict__ smass, const T *__restrict__ part,
                                                             double G, double *__restrict__ gout)
{
    const unsigned lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * AW;
    for (int64_t L = (int64_t)blockIdx.x * AW + (threadIdx.x >> 5); L < ncell; L += nw) {
        if (cnchild[L] != 0) continue;
        const uint32_t i0 = ioff[L], i1 = ioff[L + 1];
        if (i0 == i1) continue;
        const int64_t lb = cbegin[L];
        const int lc = ccount[L];
        for (int j = lane; j < lc; j += 32) {
            double t[4] = {0, 0, 0, 0};
            for (uint32_t it = i0; it < i1; ++it) {
                const T *o = part + (roff[L] + (int64_t)(it - i0) * lc + j) * 4;
#pragma unroll
                for (int d = 0; d < 4; ++d) t[d] += (double)o[d];
            }
            const double m = smass[lb + j];
            gout[4 * (lb + j) + 0] = G * m * t[0];
            gout[4 * (lb + j) + 1] = G * m * t[1];
            gout[4 * (lb + j) + 2] = G * m * t[2];
            gout[4 * (lb + j) + 3] = G * t[3];
        }
    }
}

// Position of multi-index (i, j, k) in the moment order (degree ascending, then i
// descending, then j descending).
__host__ __device__ constexpr int moment_index(int i, int j, int k)
{
    const int n = i + j + k;
    return n * (n + 1) * (n + 2) / 6 + (n - i) * (n - i + 1) / 2 + (n - i - j);
}

// Leaves: transposed P2M of dL/dM onto the particles (float64), plus the sink-side and
// P2P source-side parts; written in original order.  A half-warp per leaf, a lane per
// particle; with (d = x - z) the sums
//   dL/dm = sum_a Mbar_a d^a,   dL/dx = m sum_a Mbar_a grad(d^a)
// are taken in factorised form (z innermost, then y, then x), fully unrolled so that
// the powers stay in registers.
template <int P>
__global__ void __launch_bounds__(AW * 32) k_adj_leaf(
    int64_t ncell, const int32_t *__restrict__ cnchild, const int32_t *__restrict__ cbegin,
    const int32_t *__restrict__ ccount, const double *__restrict__ ccom, const double *__restrict__ spos,
    const double *__restrict__ smass, const double *__restrict__ Mbar, const double *__restrict__ gsink,
    const double *__restrict__ gp2p, const uint32_t *__restrict__ perm, double *__restrict__ g_pos,
    double *__restrict__ g_mass)
{
    constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
    const unsigned lane = lane_id();
    const int half = (int)(lane >> 4), hl = (int)(lane & 15);
    const int64_t nh = (int64_t)gridDim.x * AW * 2;
    for (int64_t c = ((int64_t)blockIdx.x * AW + (threadIdx.x >> 5)) * 2 + half; c < ncell; c += nh) {
        if (cnchild[c] != 0) continue;
        const double *__restrict__ mb = Mbar + c * NC;
        const int64_t b = cbegin[c], n = ccount[c];
        for (int64_t s = b + hl; s < b + n; s += 16) {
            double px[P + 1], py[P + 1], pz[P + 1];
            px[0] = py[0] = pz[0] = 1.0;
            const double dx = spos[3 * s + 0] - ccom[3 * c + 0];
            const double dy = spos[3 * s + 1] - ccom[3 * c + 1];
            const double dz = spos[3 * s + 2] - ccom[3 * c + 2];
#pragma unroll
            for (int q = 1; q <= P; ++q) {
                px[q] = px[q - 1] * dx;
                py[q] = py[q - 1] * dy;
                pz[q] = pz[q - 1] * dz;
            }
            double gm = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
            for (int i = 0; i <= P; ++i) {
                double T0 = 0.0, Ty = 0.0, Tz = 0.0;
#pragma unroll
                for (int j = 0; j <= P - i; ++j) {
                    double S0 = 0.0, Sz = 0.0;
#pragma unroll
                    for (int k = 0; k <= P - i - j; ++k) {
                        const double m = __ldg(mb + moment_index(i, j, k));
                        S0 += m * pz[k];
                        if (k > 0) Sz += (double)k * m * pz[k - 1];
                    }
                    T0 += py[j] * S0;
                    Tz += py[j] * Sz;
                    if (j > 0) Ty += (double)j * py[j - 1] * S0;
                }
                gm += px[i] * T0;
                gy += px[i] * Ty;
                gz += px[i] * Tz;
                if (i > 0) gx += (double)i * px[i - 1] * T0;
            }
            const double m = smass[s];
            const int64_t o = perm[s];
            g_pos[3 * o + 0] = m * gx + gsink[3 * s + 0] + gp2p[4 * s + 0];
            g_pos[3 * o + 1] = m * gy + gsink[3 * s + 1] + gp2p[4 * s + 1];
            g_pos[3 * o + 2] = m * gz + gsink[3 * s + 2] + gp2p[4 * s + 2];
            g_mass[o] = gm + gp2p[4 * s + 3];
        }
    }
}

template <int P, class T>
int adjoint_pt(hot_ctx *c, const double *g_acc, const double *g_pot, double *g_pos, double *g_mass)
{
    constexpr int NS = ACfg<P, T>::NS;
    constexpr int NC = ACfg<P, T>::NC;
    cudaStream_t s = c->st;
    const int64_t N = c->N, nc = c->ncell, ng = c->ngroup;
    const T *rec = nullptr;
    if constexpr (sizeof(T) == 4)
        rec = c->rec32.p;
    else
        rec = c->rec64.p;

    // weights and positions in sorted order
    HOT_CK(c->adj_w.ensure(4 * sizeof(T) * (size_t)N, s));
    HOT_CK(c->adj_xhl.ensure(8 * (size_t)N, s));
    T *w = (T *)c->adj_w.p;
    HOT_COUNT_LAUNCH();
    k_adj_prep<T><<<hot_blocks(N, 256), 256, 0, s>>>(g_acc, g_pot, c->idx.p, c->spos.p, N, w, c->adj_xhl.p);

    // sink side (interaction kernel in adjoint mode) on the second stream, concurrent with
    // the source side below (they share no buffer the other writes), forked once the M2P
    // coefficient adjoints are launched: the latency-bound steps that follow (per-cell
    // sums, the descent of dL/dM, the P2P lists' transposition) then run beside it (at
    // 2^18 the adjoint 8.95 -> 8.70 ms against a fork before the lists' transposition)
    HOT_CK(c->adj_gsink.ensure(3 * (size_t)N, s));
    bool sink_launched = false;
    auto launch_sink = [&]() -> int {
        if (sink_launched) return HOT_OK;
        sink_launched = true;
        if (cudaEventRecord(c->ev_fork, s) != cudaSuccess) return HOT_ECUDA;
        if (cudaStreamWaitEvent(c->st2, c->ev_fork, 0) != cudaSuccess) return HOT_ECUDA;
        return hot_impl_adjoint_sink(c, w, c->adj_gsink.p, c->st2);
    };
    int r = HOT_OK;
    auto source_side = [&]() -> int {
        int r = HOT_OK;
        // source side of M2P: transpose the lists, coefficient adjoints per item
        const int64_t nm = c->n_m2p;
        int bits = 1;
        while ((int64_t(1) << bits) <= nc) ++bits;
        HOT_CK(c->tp_key.ensure(nm + 1, s));
        HOT_CK(c->tp_key2.ensure(nm + 1, s));
        HOT_CK(c->tp_val.ensure(nm + 1, s));
        HOT_CK(c->tp_val2.ensure(nm + 1, s));
        HOT_CK(c->tp_start.ensure(nc + 1, s));
        HOT_CK(c->tp_end.ensure(nc + 1, s));
        HOT_CK(c->it_cnt.ensure(nc + 1, s));
        HOT_CK(c->it_off.ensure(nc + 1, s));
        HOT_CK(c->adj_mbar.ensure((size_t)NC * nc, s));
        HOT_CK(c->scan_tmp.ensure(hot_scan_tmp_elems(nc + 64), s));
        HOT_CK(cudaMemsetAsync(c->adj_mbar.p, 0, sizeof(double) * NC * (size_t)nc, s));
        if (nm > 0) {
            HOT_COUNT_LAUNCH();
            k_expand_pairs<<<hot_blocks(ng * 32, 256), 256, 0, s>>>(c->off_m2p.p, c->l_m2p.p, ng, c->tp_key.p, c->tp_val.p);
            r = hot_sort_pairs(c, c->tp_key.p, c->tp_val.p, c->tp_key2.p, c->tp_val2.p, nm, bits);
            if (r) return r;
            HOT_CK(cudaMemsetAsync(c->tp_start.p, 0, sizeof(int64_t) * (nc + 1), s));
            HOT_CK(cudaMemsetAsync(c->tp_end.p, 0, sizeof(int64_t) * (nc + 1), s));
            HOT_COUNT_LAUNCH();
            k_ranges<<<hot_blocks(nm, 256), 256, 0, s>>>(c->tp_key.p, nm, c->tp_start.p, c->tp_end.p);
            HOT_COUNT_LAUNCH();
            k_item_count_adj<<<hot_blocks(nc, 256), 256, 0, s>>>(c->tp_start.p, c->tp_end.p, nc, c->it_cnt.p);
            r = hot_scan_u32_to_u32(c->it_cnt.p, c->it_off.p, nc, c->scan_tmp.p, s);
            if (r) return r;
            const int64_t max_items = nm / KG + nc + 1;
            HOT_CK(c->it_cell.ensure(max_items, s));
            HOT_CK(c->it_a.ensure(max_items, s));
            HOT_CK(c->it_b.ensure(max_items, s));
            HOT_CK(c->it_part.ensure(sizeof(T) * NS * (size_t)max_items, s));
            HOT_COUNT_LAUNCH();
            k_item_fill_adj<<<hot_blocks(nc, 256), 256, 0, s>>>(c->tp_start.p, c->tp_end.p, c->it_off.p, nc, c->it_cell.p,
                                                                c->it_a.p, c->it_b.p);
            T *part = (T *)c->it_part.p;
            unsigned *swork = (unsigned *)(c->sizes.p + 63);
            HOT_CK(cudaMemsetAsync(swork, 0, sizeof(unsigned), s));
            HOT_COUNT_LAUNCH();
            k_adj_src<P, T><<<c->nsm * 8, AW * 32, 0, s>>>(c->it_off.p + nc, c->it_cell.p, c->it_a.p, c->it_b.p,
                                                          c->tp_val.p, c->gcell.p, c->cbegin.p, c->ccount.p, rec, w,
                                                          c->adj_xhl.p, c->spos.p, nullptr, swork, part);
            r = launch_sink();
            if (r) return r;
            HOT_COUNT_LAUNCH();
            k_adj_cells<P, T><<<hot_blocks(nc, AW, c->nsm * 16), AW * 32, 0, s>>>(nc, c->it_off.p, part, rec,
                                                                                  c->prm.G, c->adj_mbar.p);
        }
        // push dL/dM down the tree, level by level
        for (int l = 1; l <= (int)c->maxlevel; ++l) {
            const int64_t a = c->level_off[l], n = c->level_off[l + 1] - a;
            if (n <= 0) continue;
            HOT_COUNT_LAUNCH();
            k_adj_l2l<P><<<hot_blocks(n, AW, c->nsm * 16), AW * 32, 0, s>>>(c->level_cells.p + a, n, c->cparent.p,
                                                                           c->ccom.p, c->adj_mbar.p);
        }

        // source side of P2P: transpose the leaf lists
        const int64_t np = c->n_p2p;
        HOT_CK(c->adj_gp2p.ensure(4 * (size_t)N, s));
        HOT_CK(cudaMemsetAsync(c->adj_gp2p.p, 0, sizeof(double) * 4 * (size_t)N, s));
        if (np > 0) {
            HOT_CK(c->tp_key.ensure(np + 1, s));
            HOT_CK(c->tp_key2.ensure(np + 1, s));
            HOT_CK(c->tp_val.ensure(np + 1, s));
            HOT_CK(c->tp_val2.ensure(np + 1, s));
            HOT_COUNT_LAUNCH();
            k_expand_pairs<<<hot_blocks(ng * 32, 256), 256, 0, s>>>(c->off_p2p.p, c->l_p2p.p, ng, c->tp_key.p, c->tp_val.p);
            r = hot_sort_pairs(c, c->tp_key.p, c->tp_val.p, c->tp_key2.p, c->tp_val2.p, np, bits);
            if (r) return r;
            HOT_CK(cudaMemsetAsync(c->tp_start.p, 0, sizeof(int64_t) * (nc + 1), s));
            HOT_CK(cudaMemsetAsync(c->tp_end.p, 0, sizeof(int64_t) * (nc + 1), s));
            HOT_COUNT_LAUNCH();
            k_ranges<<<hot_blocks(np, 256), 256, 0, s>>>(c->tp_key.p, np, c->tp_start.p, c->tp_end.p);
            // work items: a leaf and up to KG of the groups that list it
            const int64_t max_items = np / KG + nc + 1;
            // rows: sum over leaves of items x particles <= (source-particle visits) / KG + N
            const int64_t max_rows = c->n_p2p_src / KG + N + 1;
            HOT_CK(c->it_cell.ensure(max_items, s));
            HOT_CK(c->it_a.ensure(max_items, s));
            HOT_CK(c->it_b.ensure(max_items, s));
            HOT_CK(c->adj_roff.ensure(nc + 1, s));
            HOT_CK(c->adj_pp.ensure(sizeof(T) * 4 * (size_t)max_rows, s));
            HOT_COUNT_LAUNCH();
            k_item_rows<<<hot_blocks(nc, 256), 256, 0, s>>>(c->tp_start.p, c->tp_end.p, c->ccount.p, c->cnchild.p, nc,
                                                            c->it_cnt.p + 0);
            r = hot_scan_u32_to_i64(c->it_cnt.p, c->adj_roff.p, nc, c->scan_tmp.p, s);
            if (r) return r;
            HOT_COUNT_LAUNCH();
            k_item_count_adj<<<hot_blocks(nc, 256), 256, 0, s>>>(c->tp_start.p, c->tp_end.p, nc, c->it_cnt.p);
            r = hot_scan_u32_to_u32(c->it_cnt.p, c->it_off.p, nc, c->scan_tmp.p, s);
            if (r) return r;
            HOT_COUNT_LAUNCH();
            k_item_fill_adj<<<hot_blocks(nc, 256), 256, 0, s>>>(c->tp_start.p, c->tp_end.p, c->it_off.p, nc, c->it_cell.p,
                                                                c->it_a.p, c->it_b.p);
            unsigned *pwork = (unsigned *)(c->sizes.p + 62);
            HOT_CK(cudaMemsetAsync(pwork, 0, sizeof(unsigned), s));
            T *pp = (T *)c->adj_pp.p;
            HOT_COUNT_LAUNCH();
            auto p2p_src = c->prm.softening == HOT_SOFT_K1       ? k_adj_p2p_src<T, HOT_SOFT_K1>
                           : c->prm.softening == HOT_SOFT_SPLINE ? k_adj_p2p_src<T, HOT_SOFT_SPLINE>
                                                                 : k_adj_p2p_src<T, HOT_SOFT_PLUMMER>;
            p2p_src<<<c->nsm * 8, AW * 32, 0, s>>>(c->it_off.p + nc, c->it_cell.p, c->it_a.p, c->it_b.p,
                                                   c->tp_val.p, c->gcell.p, c->cbegin.p, c->ccount.p, c->cend.p,
                                                   c->ccom.p, c->spos.p, c->smass.p, c->prel.p, c->adj_xhl.p, w,
                                                   (T)(c->prm.eps * c->prm.eps), c->it_off.p, c->adj_roff.p,
                                                   pwork, pp);
            HOT_COUNT_LAUNCH();
            k_adj_p2p_combine<T><<<hot_blocks(nc, AW, c->nsm * 16), AW * 32, 0, s>>>(
                nc, c->cnchild.p, c->it_off.p, c->adj_roff.p, c->cbegin.p, c->ccount.p, c->smass.p, pp, c->prm.G,
                c->adj_gp2p.p);
        }
        return HOT_OK;
    };
    if (r == HOT_OK) r = source_side();
    if (r == HOT_OK) r = launch_sink();  // when the source side had no M2P entries
    // join (also after an error, so that no work of this call is left behind on st2)
    HOT_CK(cudaEventRecord(c->ev_join, c->st2));
    HOT_CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    if (r) return r;

    // leaves: transposed P2M and the final sums, original order
    HOT_COUNT_LAUNCH();
    k_adj_leaf<P><<<c->nsm * 8, AW * 32, 0, s>>>(nc, c->cnchild.p, c->cbegin.p, c->ccount.p, c->ccom.p, c->spos.p,
                                                c->smass.p, c->adj_mbar.p, c->adj_gsink.p, c->adj_gp2p.p, c->idx.p,
                                                g_pos, g_mass);
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}

template <int P>
int adjoint_p(hot_ctx *c, const double *g_acc, const double *g_pot, double *g_pos, double *g_mass)
{
    if (c->prm.precision == HOT_FP64) return adjoint_pt<P, double>(c, g_acc, g_pot, g_pos, g_mass);
    return adjoint_pt<P, float>(c, g_acc, g_pot, g_pos, g_mass);
}

}  // namespace

int hot_impl_adjoint(hot_ctx *c, const double *g_acc, const double *g_pot, double *g_pos, double *g_mass)
{
    // the adjoint's coefficient sums are register-resident per lane: orders up to 6, one
    // order per call (not under per-interaction order selection)
    if (c->p_mom > HOT_ADJ_PMAX || c->varq || c->prm.box > 0.0) return HOT_EINVAL;
    hot_tic(c, 5);
    int r;
    switch (c->p_mom) {
        case 0: r = adjoint_p<0>(c, g_acc, g_pot, g_pos, g_mass); break;
        case 1: r = adjoint_p<1>(c, g_acc, g_pot, g_pos, g_mass); break;
        case 2: r = adjoint_p<2>(c, g_acc, g_pot, g_pos, g_mass); break;
        case 3: r = adjoint_p<3>(c, g_acc, g_pot, g_pos, g_mass); break;
        case 4: r = adjoint_p<4>(c, g_acc, g_pot, g_pos, g_mass); break;
        case 5: r = adjoint_p<5>(c, g_acc, g_pot, g_pos, g_mass); break;
        case 6: r = adjoint_p<6>(c, g_acc, g_pot, g_pos, g_mass); break;
        default: return HOT_ESTATE;
    }
    hot_toc(c, 5);
    return r;
}
