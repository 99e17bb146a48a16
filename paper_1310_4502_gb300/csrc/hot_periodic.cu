// hot_periodic.cu -- periodic boundaries, the far images (Sec. "Boundary Conditions").
//
// The tree serves the central cube and its images within ws cubes (the traversal and the
// interaction kernels, their list entries tagged with the image).  Every farther image acts
// through one local expansion about the cube's centre c:
//
//   phi_far(x) = -G sum_b (x - c)^b / b! L_b,   a_far(x) = G sum_b L_b (x - c)^(b - e_d) / (b - e_d)!
//   L_b = sum_a (-1)^|a| / a! M_a D^(a + b) psi_far(0),   M_a = sum_j m_j (x_j - c)^a,
//
// |a| <= 8 (the order of the paper), |b| <= 9 (so that the acceleration is of order 8).
// D^g psi_far(0), |g| <= 17, are lattice sums of the periodic Green's function without the
// images within ws, under the conventions of Ewald summation (a uniform neutralising
// background, a conducting boundary at infinity):
//
//   psi(r) = sum_n erfc(alpha |r + nL|) / |r + nL| + (4 pi / V) sum_{k != 0} exp(-k^2 / 4 alpha^2)
//            / k^2 cos(k . r) - pi / (alpha^2 V),     psi_far = psi - sum_{|n|_inf <= ws} 1 / |r + nL|,
//
// computed once per (L, ws) on the host, in units of L (alpha = 1) and scaled by
// L^-(|g| + 1).  The derivatives of each radial term f(|r|) come from the McMurchie-Davidson
// recurrence: with G_m = (1/s d/ds)^m f and R^m_tuv = d_x^t d_y^u d_z^v G_m,
//   R^m_(t+1)uv = X R^(m+1)_tuv + t R^(m+1)_(t-1)uv   (likewise in y and z),
// and (1/s d/ds)^m of erfc(alpha s)/s, erf(alpha s)/s in the incomplete-gamma form
// (-1)^m (2m - 1)!! s^-(2m+1) Q(m + 1/2, alpha^2 s^2), resp. P(...): no difference of
// nearly equal terms at any order.
//
// Multi-indices are in graded order: by |g|, then by descending g_x, then by descending g_y,
// far_idx(g) = n (n + 1) (n + 2) / 6 + j (j + 1) / 2 + g_z, n = |g|, j = g_y + g_z.
#include <cmath>
#include <vector>

#include "hot_common.cuh"

namespace {

constexpr int PF = HOT_PFAR;   // order of the far images' moments
constexpr int KD = 2 * PF + 1; // order of the lattice sums

__host__ __device__ constexpr int far_nc(int n) { return (n + 1) * (n + 2) * (n + 3) / 6; }  // |g| <= n
__host__ __device__ constexpr int far_idx(int a, int b, int c)
{
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

constexpr int NM = far_nc(PF);      // moments, and acceleration coefficients per axis
constexpr int NL = far_nc(PF + 1);  // local coefficients
constexpr int ND = far_nc(KD);      // lattice sums
constexpr int NCOEF = NL + 3 * NM;  // potential and acceleration coefficients of the L2P
constexpr int FT = 128;             // particles per tile of the moments kernel
constexpr int FB = 192;             // threads of the moments kernel (NM of them work)
// Orders kept in float64 in the mixed mode: moments and potential terms up to 2, acceleration
// terms up to 1.  They carry the part of the far field that cancels against the images' sum
// in the tree (for a near-uniform cube the far potential's constant is ~60 G M / L against
// a total of ~0.05 G M / L, the far acceleration several times the total): rounded to
// float32 they would cost the potential ~1e-3 of its rms.
constexpr int NLO = far_nc(2);

__host__ __device__ inline void far_decode(int t, int &a, int &b, int &c)
{
    int n = 0;
    while (far_nc(n) <= t) ++n;
    int r = t - (n > 0 ? far_nc(n - 1) : 0);
    int j = 0;
    while ((j + 1) * (j + 2) / 2 <= r) ++j;
    c = r - j * (j + 1) / 2;
    b = j - c;
    a = n - j;
}

// ---- lattice sums (host) ----

// Regularised lower incomplete gamma P(a, x) = pre * sum_k x^k / ((a + 1) ... (a + k)),
// pre = x^a e^-x / Gamma(a + 1) given: positive terms, for the moderate x of the near images.
double gamma_p_series(double a, double x, double pre)
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 1000; ++k) {
        term *= x / (a + k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return pre * sum;
}

// D^g psi_far(0) in units of L = 1, |g| <= K, graded order.
void lattice_sums_unit(int ws, int K, double *D)
{
    const int nd = far_nc(K);
    for (int i = 0; i < nd; ++i) D[i] = 0.0;
    const double alpha = 1.0;
    const int NR = 6;  // real space |n|_inf <= 6: erfc(6) ~ 2e-17
    const int KM = 4;  // reciprocal |m|_inf <= 4: exp(-pi^2 m^2) ~ 1e-69 at |m| = 4
    const int S = K + 1;
    std::vector<double> E((size_t)S * S * S * S);
    auto at = [&](int m, int t, int u, int v) -> double & { return E[(((size_t)m * S + t) * S + u) * S + v]; };
    std::vector<double> Gm(K + 1);
    const double rpi = std::sqrt(M_PI);
    for (int nx = -NR; nx <= NR; ++nx)
        for (int ny = -NR; ny <= NR; ++ny)
            for (int nz = -NR; nz <= NR; ++nz) {
                const int ninf = std::max(std::abs(nx), std::max(std::abs(ny), std::abs(nz)));
                const double X = nx, Y = ny, Z = nz;
                if (ninf == 0) {
                    // - erf(alpha s) / s at s = 0: G_m = 2^m F^(m)(0), F(u) the series in u = s^2
                    double pw = 1.0;
                    for (int m = 0; m <= K; ++m) {
                        Gm[m] = -(2.0 * alpha / rpi) * pw / (2.0 * m + 1.0);
                        pw *= -2.0 * alpha * alpha;
                    }
                } else {
                    const double s2 = X * X + Y * Y + Z * Z, s = std::sqrt(s2), x = alpha * alpha * s2;
                    const bool near = ninf <= ws;
                    // Q(1/2, x) = erfc(sqrt x); Q(a + 1, x) = Q(a, x) + qt, qt = x^a e^-x / Gamma(a + 1),
                    // a = m + 1/2, itself a running product from x^(1/2) e^-x / Gamma(3/2)
                    double q = std::erfc(std::sqrt(x));
                    double qt = std::sqrt(x) * std::exp(-x) / (0.5 * rpi);
                    double base = 1.0 / s;  // (-1)^m (2m - 1)!! s^-(2m+1)
                    for (int m = 0; m <= K; ++m) {
                        const double a = m + 0.5;
                        Gm[m] = near ? -base * gamma_p_series(a, x, qt) : base * q;
                        q += qt;
                        qt *= x / (a + 1.0);
                        base *= -(2.0 * m + 1.0) / s2;
                    }
                }
                for (int m = 0; m <= K; ++m) at(m, 0, 0, 0) = Gm[m];
                for (int t = 1; t <= K; ++t)
                    for (int m = 0; m <= K - t; ++m)
                        at(m, t, 0, 0) = X * at(m + 1, t - 1, 0, 0) + (t >= 2 ? (t - 1) * at(m + 1, t - 2, 0, 0) : 0.0);
                for (int u = 1; u <= K; ++u)
                    for (int t = 0; t <= K - u; ++t)
                        for (int m = 0; m <= K - t - u; ++m)
                            at(m, t, u, 0) =
                                Y * at(m + 1, t, u - 1, 0) + (u >= 2 ? (u - 1) * at(m + 1, t, u - 2, 0) : 0.0);
                for (int v = 1; v <= K; ++v)
                    for (int u = 0; u <= K - v; ++u)
                        for (int t = 0; t <= K - u - v; ++t)
                            for (int m = 0; m <= K - t - u - v; ++m)
                                at(m, t, u, v) =
                                    Z * at(m + 1, t, u, v - 1) + (v >= 2 ? (v - 1) * at(m + 1, t, u, v - 2) : 0.0);
                for (int t = 0; t <= K; ++t)
                    for (int u = 0; u <= K - t; ++u)
                        for (int v = 0; v <= K - t - u; ++v) D[far_idx(t, u, v)] += at(0, t, u, v);
            }
    // reciprocal space: d^g cos(k . r) at 0 is (-1)^(|g|/2) k^g for even |g|, 0 for odd
    for (int mx = -KM; mx <= KM; ++mx)
        for (int my = -KM; my <= KM; ++my)
            for (int mz = -KM; mz <= KM; ++mz) {
                if (!mx && !my && !mz) continue;
                const double kx = 2.0 * M_PI * mx, ky = 2.0 * M_PI * my, kz = 2.0 * M_PI * mz;
                const double k2 = kx * kx + ky * ky + kz * kz;
                const double w = 4.0 * M_PI * std::exp(-k2 / (4.0 * alpha * alpha)) / k2;
                double px = 1.0;
                for (int t = 0; t <= K; ++t, px *= kx) {
                    double py = 1.0;
                    for (int u = 0; u <= K - t; ++u, py *= ky) {
                        double pz = 1.0;
                        for (int v = 0; v <= K - t - u; ++v, pz *= kz) {
                            const int n = t + u + v;
                            if (n & 1) continue;
                            D[far_idx(t, u, v)] += ((n / 2) & 1 ? -w : w) * px * py * pz;
                        }
                    }
                }
            }
    D[0] += -M_PI / (alpha * alpha);
}

// ---- far field (device) ----

// Moments about c of the particles of tiles blockIdx.x, blockIdx.x + gridDim.x, ...:
// part[block][a] = sum m (x - c)^a, |a| <= PF.  T: arithmetic of a tile's sum (float32:
// the tile sums are added in float64).  The moments of order <= 2 are float64 throughout:
// each loading thread accumulates those of its own particles (1, x, y, z, x^2, xy, xz,
// y^2, yz, z^2 in the graded order), reduced over the block at the end.
template <class T>
__global__ void __launch_bounds__(FB) k_far_moments(const double *__restrict__ spos, const double *__restrict__ smass,
                                                    int64_t N, double cx, double cy, double cz,
                                                    double *__restrict__ part)
{
    __shared__ T pw[FT][3][PF + 1];
    __shared__ T ms[FT];
    __shared__ double red[FT / 32][NLO];
    const int t = threadIdx.x;
    int a0 = 0, a1 = 0, a2 = 0;
    if (t < NM) far_decode(t, a0, a1, a2);
    double tot = 0.0;
    double lo[NLO];
#pragma unroll
    for (int k = 0; k < NLO; ++k) lo[k] = 0.0;
    const int64_t ntile = (N + FT - 1) / FT;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        __syncthreads();
        if (t < FT) {
            const int64_t i = tile * FT + t;
            const bool ok = i < N;
            const double c3[3] = {cx, cy, cz};
            double y[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                y[d] = ok ? spos[3 * i + d] - c3[d] : 0.0;
                const T yt = (T)y[d];
                T p = T(1);
#pragma unroll
                for (int k = 0; k <= PF; ++k) {
                    pw[t][d][k] = p;
                    p *= yt;
                }
            }
            const double m = ok ? smass[i] : 0.0;
            ms[t] = (T)m;
            if (sizeof(T) == 4) {
                const double mx = m * y[0], my = m * y[1], mz = m * y[2];
                lo[0] += m;
                lo[1] += mx;
                lo[2] += my;
                lo[3] += mz;
                lo[4] += mx * y[0];
                lo[5] += mx * y[1];
                lo[6] += mx * y[2];
                lo[7] += my * y[1];
                lo[8] += my * y[2];
                lo[9] += mz * y[2];
            }
        }
        __syncthreads();
        if (t < NM && (sizeof(T) == 8 || t >= NLO)) {
            T s = T(0);
#pragma unroll 4
            for (int i = 0; i < FT; ++i) s += ms[i] * pw[i][0][a0] * pw[i][1][a1] * pw[i][2][a2];
            tot += (double)s;
        }
    }
    if (sizeof(T) == 4) {
        // the float64 low orders: warp sums of the loading threads, then across their warps
        if (t < FT) {
#pragma unroll
            for (int k = 0; k < NLO; ++k) {
                double v = lo[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if ((t & 31) == 0) red[t >> 5][k] = v;
            }
        }
        __syncthreads();
        if (t < NLO) {
            tot = 0.0;
#pragma unroll
            for (int w = 0; w < FT / 32; ++w) tot += red[w][t];
        }
    }
    if (t < NM) part[(int64_t)blockIdx.x * NM + t] = tot;
}

__device__ inline double fact(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

// One block: the moments M_a (block partials summed in a fixed order), the local
// coefficients L_b from the lattice sums D, and the L2P coefficients:
// coef[b] = -G L_b / b! (|b| <= PF + 1), coef[NL + 3 b' + d] = G L_(b' + e_d) / b'! (|b'| <= PF),
// coef[NCOEF + b] = L_b.
__global__ void __launch_bounds__(256) k_far_local(const double *__restrict__ part, int nb,
                                                   const double *__restrict__ D, double G, double *__restrict__ coef)
{
    __shared__ double sM[NM];
    __shared__ double sL[NL];
    __shared__ unsigned char dec[NL][3];
    const int t = threadIdx.x;
    if (t < NL) {
        int a, b, c;
        far_decode(t, a, b, c);
        dec[t][0] = (unsigned char)a;
        dec[t][1] = (unsigned char)b;
        dec[t][2] = (unsigned char)c;
    }
    if (t < NM) {
        double m = 0.0;
        for (int k = 0; k < nb; ++k) m += part[(int64_t)k * NM + t];
        int a, b, c;
        far_decode(t, a, b, c);
        sM[t] = ((a + b + c) & 1 ? -m : m) / (fact(a) * fact(b) * fact(c));
    }
    __syncthreads();
    if (t < NL) {
        const int b0 = dec[t][0], b1 = dec[t][1], b2 = dec[t][2];
        double l = 0.0;
        for (int a = 0; a < NM; ++a) l += sM[a] * D[far_idx(dec[a][0] + b0, dec[a][1] + b1, dec[a][2] + b2)];
        sL[t] = l;
        coef[NCOEF + t] = l;
    }
    __syncthreads();
    if (t < NL) {
        const int b0 = dec[t][0], b1 = dec[t][1], b2 = dec[t][2];
        const double bf = fact(b0) * fact(b1) * fact(b2);
        coef[t] = -G * sL[t] / bf;
        if (t < NM) {
            coef[NL + 3 * t + 0] = G * sL[far_idx(b0 + 1, b1, b2)] / bf;
            coef[NL + 3 * t + 1] = G * sL[far_idx(b0, b1 + 1, b2)] / bf;
            coef[NL + 3 * t + 2] = G * sL[far_idx(b0, b1, b2 + 1)] / bf;
        }
    }
}

// L2P of the local expansion at every particle (sorted slot i, output row perm[i]), added
// to the accelerations and potentials of the tree.  Potential terms of order <= 2 and
// acceleration terms of order <= 1 in float64, the rest in T.
template <class T>
__global__ void __launch_bounds__(256) k_far_l2p(const double *__restrict__ spos, const uint32_t *__restrict__ perm,
                                                 int64_t N, double cx, double cy, double cz,
                                                 const double *__restrict__ coef, double *__restrict__ acc,
                                                 double *__restrict__ pot)
{
    __shared__ T cp[NL];
    __shared__ T ca[NM][3];
    __shared__ double cpd[NLO];
    __shared__ double cad[far_nc(1)][3];
    for (int k = threadIdx.x; k < NL; k += blockDim.x) cp[k] = (T)coef[k];
    for (int k = threadIdx.x; k < 3 * NM; k += blockDim.x) ca[k / 3][k % 3] = (T)coef[NL + k];
    for (int k = threadIdx.x; k < NLO; k += blockDim.x) cpd[k] = coef[k];
    for (int k = threadIdx.x; k < 3 * far_nc(1); k += blockDim.x) cad[k / 3][k % 3] = coef[NL + k];
    __syncthreads();
    // one particle per thread: a grid-stride loop would let the compiler hoist the 715
    // coefficient loads out of it as invariants (and spill them)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const double xd = spos[3 * i + 0] - cx, yd = spos[3 * i + 1] - cy, zd = spos[3 * i + 2] - cz;
        const double qx[3] = {1.0, xd, xd * xd}, qy[3] = {1.0, yd, yd * yd}, qz[3] = {1.0, zd, zd * zd};
        const T x = (T)xd, y = (T)yd, z = (T)zd;
        T px[PF + 2], py[PF + 2], pz[PF + 2];
        px[0] = py[0] = pz[0] = T(1);
#pragma unroll
        for (int k = 1; k <= PF + 1; ++k) {
            px[k] = px[k - 1] * x;
            py[k] = py[k - 1] * y;
            pz[k] = pz[k - 1] * z;
        }
        T ph = T(0), ax = T(0), ay = T(0), az = T(0);
        double phd = 0.0, axd = 0.0, ayd = 0.0, azd = 0.0;
#pragma unroll
        for (int n = 0; n <= PF + 1; ++n)
#pragma unroll
            for (int j = 0; j <= n; ++j)
#pragma unroll
                for (int v = 0; v <= j; ++v) {
                    const int k = far_idx(n - j, j - v, v);
                    if (n <= 2) {
                        const double mono = qx[n - j] * qy[j - v] * qz[v];
                        phd += cpd[k] * mono;
                        if (n <= 1) {
                            axd += cad[k][0] * mono;
                            ayd += cad[k][1] * mono;
                            azd += cad[k][2] * mono;
                        } else {
                            const T m = (T)mono;
                            ax += ca[k][0] * m;
                            ay += ca[k][1] * m;
                            az += ca[k][2] * m;
                        }
                    } else {
                        const T mono = px[n - j] * py[j - v] * pz[v];
                        ph += cp[k] * mono;
                        if (n <= PF) {
                            ax += ca[k][0] * mono;
                            ay += ca[k][1] * mono;
                            az += ca[k][2] * mono;
                        }
                    }
                }
        const int64_t o = perm[i];
        acc[3 * o + 0] += (double)ax + axd;
        acc[3 * o + 1] += (double)ay + ayd;
        acc[3 * o + 2] += (double)az + azd;
        if (pot) pot[o] += (double)ph + phd;
    }
}

}  // namespace

extern "C" int hot_lattice_sums(double L, int ws, int order, double *out)
{
    if (!out || !(L > 0.0) || !std::isfinite(L) || ws < 1 || ws > HOT_WS_MAX || order < 0 || order > KD)
        return HOT_EINVAL;
    std::vector<double> D(far_nc(KD));
    lattice_sums_unit(ws, order, D.data());
    for (int t = 0; t < far_nc(order); ++t) {
        int a, b, c;
        far_decode(t, a, b, c);
        out[t] = D[t] / std::pow(L, a + b + c + 1);
    }
    return HOT_OK;
}

// Far images under periodic boundaries: the local expansion added to acc [N][3] and pot [N]
// (original order) on the context's stream.
int hot_impl_far_field(hot_ctx *c, double *acc, double *pot)
{
    if (!(c->prm.box > 0.0)) return HOT_OK;
    cudaStream_t s = c->st;
    const double L = c->prm.box;
    if (c->per_D_L != L || c->per_D_ws != c->prm.ws || c->per_Dh.empty()) {
        c->per_Dh.assign(ND, 0.0);
        const int e = hot_lattice_sums(L, c->prm.ws, KD, c->per_Dh.data());
        if (e) return e;
        HOT_CK(c->per_D.ensure(ND, s));
        HOT_CK(cudaMemcpyAsync(c->per_D.p, c->per_Dh.data(), ND * sizeof(double), cudaMemcpyHostToDevice, s));
        c->per_D_L = L;
        c->per_D_ws = c->prm.ws;
    }
    const double cx = c->prm.box_lo[0] + 0.5 * L, cy = c->prm.box_lo[1] + 0.5 * L, cz = c->prm.box_lo[2] + 0.5 * L;
    const int64_t ntile = (c->N + FT - 1) / FT;
    const int nb = (int)(ntile < 2 * (int64_t)c->nsm ? ntile : 2 * (int64_t)c->nsm);
    HOT_CK(c->per_part.ensure((size_t)nb * NM, s));
    HOT_CK(c->per_coef.ensure(NCOEF + NL, s));
    const bool f64 = c->prm.precision == HOT_FP64;
    HOT_COUNT_LAUNCH();
    if (f64)
        k_far_moments<double><<<nb, FB, 0, s>>>(c->spos.p, c->smass.p, c->N, cx, cy, cz, c->per_part.p);
    else
        k_far_moments<float><<<nb, FB, 0, s>>>(c->spos.p, c->smass.p, c->N, cx, cy, cz, c->per_part.p);
    HOT_COUNT_LAUNCH();
    k_far_local<<<1, 256, 0, s>>>(c->per_part.p, nb, c->per_D.p, c->prm.G, c->per_coef.p);
    const int64_t bl = (c->N + 255) / 256;
    HOT_COUNT_LAUNCH();
    if (f64)
        k_far_l2p<double><<<(unsigned)bl, 256, 0, s>>>(c->spos.p, c->idx.p, c->N, cx, cy, cz, c->per_coef.p, acc, pot);
    else
        k_far_l2p<float><<<(unsigned)bl, 256, 0, s>>>(c->spos.p, c->idx.p, c->N, cx, cy, cz, c->per_coef.p, acc, pot);
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}
