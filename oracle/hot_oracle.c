/*
 * hot_oracle.c -- plain CPU FP64 oracle for the hashed oct-tree gravity path of
 * Warren, "2HOT: An Improved Parallel Hashed Oct-Tree N-Body Algorithm for
 * Cosmological Simulation" (SC'13, arXiv:1310.4502).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or generator with the CUDA library; the CUDA path must never
 * call it.
 *
 * Built with -O2 -ffp-contract=off: every expression is evaluated with the
 * roundings it is written with (no fused multiply-add).
 *
 * What each part follows (section / equation of the paper):
 *   direct sum ............ Eq. (eom) with a = 1 (no expansion), Plummer force
 *                           smoothing or the K1 compensating kernel (Sec. "Force
 *                           Smoothing"; the K1 density is a stated reading, below)
 *   keys .................. space-filling-curve (Morton) keys, Sec. "Domain
 *                           Decomposition"; 21 bits per dimension, x highest in
 *                           each bit triplet, a leading placeholder bit
 *   tree .................. hashed oct-tree cells = key prefixes, Sec. "Tree
 *                           Construction and Traversal"; a cell with more than
 *                           leaf_max particles is refined, level 21 always a leaf
 *   moments ............... Eq. (moment tensor) M_a(z) = sum m (y - z)^a, taken
 *                           by definition from the particles of each cell, z =
 *                           centre of mass
 *   acceptance test ....... Sec. "Multipole Error Bounds": an absolute bound on
 *                           the acceleration error of a cell-body interaction,
 *                           geometry of Fig. "mac" (b_max, Delta_max)
 *   M2P ................... the Cartesian Taylor expansion of Sec. "Multipole
 *                           Error Bounds" (phi = sum (-1)^n/n! d^nG (.) M^n),
 *                           derivatives of the softened kernel in closed form
 *   P2P ................... pairwise softened sum, Eq. (eom)
 *   sink groups / lists ... dual-tree traversal with m x n blocking, Sec.
 *                           "Improving instruction-level parallelism"
 *   periodic images ....... Sec. "Boundary Conditions": the tree's images within ws
 *                           cubes as further sources (the far field and the Ewald
 *                           reference are in periodic.py)
 *   gradient .............. analytic derivative of the direct sum (pair sum
 *                           weighted by the tidal tensor); frozen-structure tree
 *                           function for finite differences
 *
 * Parity pins for every function live in tests/test_oracle.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXP 8
#define ORC_MAXLEVEL 21

int orc_nthreads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------
 * Force smoothing (Sec. "Force Smoothing").  A source of mass m at d = x_j - x_i,
 * r = |d|, gives the sink a = G m f(r^2) d and phi = -G m psi(r); the tidal tensor
 * of the pair is da/dx_i = -G m [f I + f2 d d^T], f2 = 2 df/d(r^2).
 *   ORC_SOFT_PLUMMER: s^2 = r^2 + eps^2, f = s^-3, f2 = -3 s^-5, psi = 1/s.
 *   ORC_SOFT_K1: Dehnen's K1 compensating kernel.  The paper names it (forces above
 *     the Newtonian ones at the outer edge of the kernel compensate the weaker forces
 *     inside) without a formula; it is read here as the kernel of unit mass, support
 *     r < eps and density rho(x) = 105/(64 pi eps^3) (1 - x^2)(5 - 9 x^2), x = r/eps:
 *     the even quartic vanishing at the edge whose second moment is zero (negative
 *     density for x^2 > 5/9).  Its enclosed mass is M(x) = 175/16 x^3 - 147/8 x^5 +
 *     135/16 x^7, so for r < eps, with u = x^2,
 *       f = g(u)/eps^3, g(u) = 175/16 - 147/8 u + 135/16 u^2,
 *       f2 = 2 g'(u)/eps^5, g'(u) = -147/8 + 135/8 u,
 *       psi = (105 - 175 u + 147 u^2 - 45 u^3) / (32 eps)
 *     (psi from integrating M(x)/x^2 inwards from psi(eps) = 1/eps), and exactly
 *     Newtonian (f = r^-3, f2 = -3 r^-5, psi = 1/r) for r >= eps.  The multipole
 *     expansion then uses the unsoftened kernel, and a cell is accepted only if every
 *     sink-source pair is at least eps apart (d >= b_max + eps).
 *   ORC_SOFT_SPLINE: the cubic spline kernel the paper cites (Springel 2005), read as the
 *     kernel of unit mass, support r < eps and density 8/(pi eps^3) w(x), x = r/eps,
 *     w = 1 - 6x^2 + 6x^3 (x < 1/2), 2(1 - x)^3 (1/2 <= x < 1).  Its enclosed mass
 *     M(x) = 32/3 x^3 - 192/5 x^5 + 32 x^6 (x < 1/2),
 *            -1/15 + 64/3 x^3 - 48 x^4 + 192/5 x^5 - 32/3 x^6 (x >= 1/2), so with
 *     f = g(x)/eps^3, g = M/x^3, f2 = g'(x)/(x eps^5) and psi (integrating M/x^2 inwards
 *     from psi(eps) = 1/eps):
 *       x < 1/2:  g = 32/3 - 192/5 x^2 + 32 x^3,  g'/x = -384/5 + 96 x,
 *                 psi eps = 14/5 - 16/3 x^2 + 48/5 x^4 - 32/5 x^5;
 *       x >= 1/2: g = 64/3 - 48 x + 192/5 x^2 - 32/3 x^3 - 1/(15 x^3),
 *                 g'/x = 384/5 - 48/x - 32 x + 1/(5 x^5),
 *                 psi eps = 16/5 - 1/(15 x) - 32/3 x^2 + 16 x^3 - 48/5 x^4 + 32/15 x^5;
 *     Newtonian for r >= eps; like K1 (a kernel of compact support), unsoftened
 *     expansions and the guard d >= b_max + eps.
 * ------------------------------------------------------------------------- */
enum { ORC_SOFT_PLUMMER = 0, ORC_SOFT_K1 = 1, ORC_SOFT_SPLINE = 2 };

/* Kernels of compact support (Newtonian beyond eps). */
static int soft_compact(int kind) { return kind == ORC_SOFT_K1 || kind == ORC_SOFT_SPLINE; }
typedef struct {
    int kind;
    double eps;
} orc_soft;

/* f, f2, psi of one pair at squared separation r2; 0 for a pair that is skipped
 * (zero separation without softening). */
static int soft_eval(orc_soft sf, double r2, double *f, double *f2, double *psi)
{
    if (sf.kind == ORC_SOFT_SPLINE && r2 < sf.eps * sf.eps) {
        double e = sf.eps, e3 = e * e * e;
        double x = sqrt(r2) / e;
        double g, gx, pe;
        if (x < 0.5) {
            g = 32.0 / 3.0 + x * x * (-192.0 / 5.0 + 32.0 * x);
            gx = -384.0 / 5.0 + 96.0 * x;
            pe = 14.0 / 5.0 + x * x * (-16.0 / 3.0 + x * x * (48.0 / 5.0 - 32.0 / 5.0 * x));
        } else {
            double x3 = x * x * x;
            g = 64.0 / 3.0 + x * (-48.0 + x * (192.0 / 5.0 - 32.0 / 3.0 * x)) - 1.0 / (15.0 * x3);
            gx = 384.0 / 5.0 - 48.0 / x - 32.0 * x + 1.0 / (5.0 * x3 * x * x);
            pe = 16.0 / 5.0 - 1.0 / (15.0 * x) + x * x * (-32.0 / 3.0 + x * (16.0 + x * (-48.0 / 5.0 + 32.0 / 15.0 * x)));
        }
        *f = g / e3;
        *f2 = gx / (e3 * e * e);
        *psi = pe / e;
        return 1;
    }
    if (sf.kind == ORC_SOFT_K1 && r2 < sf.eps * sf.eps) {
        double e2 = sf.eps * sf.eps;
        double e3 = e2 * sf.eps;
        double u = r2 / e2;
        *f = (175.0 / 16.0 + u * (-147.0 / 8.0 + u * (135.0 / 16.0))) / e3;
        *f2 = 2.0 * (-147.0 / 8.0 + u * (135.0 / 8.0)) / (e3 * e2);
        *psi = (105.0 + u * (-175.0 + u * (147.0 - 45.0 * u))) / (32.0 * sf.eps);
        return 1;
    }
    double s2 = soft_compact(sf.kind) ? r2 : r2 + sf.eps * sf.eps;
    if (s2 == 0.0) return 0;
    double sinv = 1.0 / sqrt(s2);
    *psi = sinv;
    *f = sinv * sinv * sinv;
    *f2 = -3.0 * *f * sinv * sinv;
    return 1;
}

/* f, f2, psi at separation r (for the parity pins); returns 0 if skipped. */
int orc_soft_eval(int kind, double eps, double r, double *out)
{
    orc_soft sf = {kind, eps};
    return soft_eval(sf, r * r, out, out + 1, out + 2);
}

/* The kernel the multipole expansion uses: softened for Plummer, Newtonian for K1. */
static double m2p_eps2(orc_soft sf) { return soft_compact(sf.kind) ? 0.0 : sf.eps * sf.eps; }

/* ---------------------------------------------------------------------------
 * Direct sum.  a_i = G sum_{j != i} m_j f(|x_j - x_i|^2) (x_j - x_i),
 *              phi_i = -G sum_{j != i} m_j psi(|x_j - x_i|); Plummer:
 *              a_i = G sum m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2},
 *              phi_i = -G sum m_j / sqrt(|x_j - x_i|^2 + eps^2).
 * A pair whose softened distance is exactly zero is skipped.
 * ------------------------------------------------------------------------- */
static void pair_acc(const double *xi, const double *xj, double mj, double G,
                     orc_soft sf, double *a, double *phi)
{
    double dx = xj[0] - xi[0];
    double dy = xj[1] - xi[1];
    double dz = xj[2] - xi[2];
    if (soft_compact(sf.kind)) {
        double f, f2, psi;
        if (!soft_eval(sf, dx * dx + dy * dy + dz * dz, &f, &f2, &psi)) return;
        double gm = G * mj;
        a[0] += gm * f * dx;
        a[1] += gm * f * dy;
        a[2] += gm * f * dz;
        *phi -= gm * psi;
        return;
    }
    double r2 = dx * dx + dy * dy + dz * dz + sf.eps * sf.eps;
    if (r2 == 0.0) return;
    double rinv = 1.0 / sqrt(r2);
    double gm = G * mj;
    double f = gm * rinv * rinv * rinv;
    a[0] += f * dx;
    a[1] += f * dy;
    a[2] += f * dz;
    *phi -= gm * rinv;
}

/* sinks == NULL means every particle; outputs are indexed like the sink list. */
void orc_direct(int64_t N, const double *pos, const double *mass, double G, double eps, int kind,
                int64_t nsink, const int64_t *sinks, double *acc, double *pot)
{
    orc_soft sf = {kind, eps};
    if (sinks == NULL) nsink = N;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nsink; s++) {
        int64_t i = sinks ? sinks[s] : s;
        double a[3] = {0.0, 0.0, 0.0}, phi = 0.0;
        for (int64_t j = 0; j < N; j++) {
            if (j == i) continue;
            pair_acc(pos + 3 * i, pos + 3 * j, mass[j], G, sf, a, &phi);
        }
        acc[3 * s + 0] = a[0];
        acc[3 * s + 1] = a[1];
        acc[3 * s + 2] = a[2];
        if (pot) pot[s] = phi;
    }
}

/* Analytic gradient of L = sum_i w_i . a_i + sum_i v_i phi_i of the direct sum.
 * With d = x_j - x_k and the pair kernel f, f2, psi above, K(d) = f I + f2 d d^T:
 *   dL/dx_k = G sum_{j != k} [ K(d) (m_k w_j - m_j w_k) - (v_j m_k + v_k m_j) f d ]
 *   dL/dm_j = G sum_{i != j} [ w_i . (x_j - x_i) f - v_i psi ]
 * (Plummer: s^2 = |d|^2 + eps^2, K(d) = I/s^3 - 3 d d^T / s^5, f = s^-3, psi = 1/s.)
 * v may be NULL (no potential term). */
void orc_direct_grad(int64_t N, const double *pos, const double *mass, double G, double eps, int kind,
                     const double *w, const double *v, double *gpos, double *gmass)
{
    orc_soft sf = {kind, eps};
    double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < N; k++) {
        double g[3] = {0.0, 0.0, 0.0}, gm = 0.0;
        const double *xk = pos + 3 * k;
        const double *wk = w + 3 * k;
        double vk = v ? v[k] : 0.0;
        for (int64_t j = 0; j < N; j++) {
            if (j == k) continue;
            const double *xj = pos + 3 * j;
            const double *wj = w + 3 * j;
            double d[3] = {xj[0] - xk[0], xj[1] - xk[1], xj[2] - xk[2]};
            if (soft_compact(sf.kind)) {
                double f, f2, psi;
                if (!soft_eval(sf, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], &f, &f2, &psi)) continue;
                double c[3];
                for (int e = 0; e < 3; e++) c[e] = mass[k] * wj[e] - mass[j] * wk[e];
                double dc = d[0] * c[0] + d[1] * c[1] + d[2] * c[2];
                double vj = v ? v[j] : 0.0;
                double pv = vj * mass[k] + vk * mass[j];
                for (int e = 0; e < 3; e++) g[e] += G * (c[e] * f + f2 * d[e] * dc - pv * d[e] * f);
                gm += G * (-(wj[0] * d[0] + wj[1] * d[1] + wj[2] * d[2]) * f - vj * psi);
                continue;
            }
            double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
            if (s2 == 0.0) continue;
            double sinv = 1.0 / sqrt(s2);
            double s3 = sinv * sinv * sinv;
            double s5 = s3 * sinv * sinv;
            double c[3];
            for (int e = 0; e < 3; e++) c[e] = mass[k] * wj[e] - mass[j] * wk[e];
            double dc = d[0] * c[0] + d[1] * c[1] + d[2] * c[2];
            double vj = v ? v[j] : 0.0;
            double pv = vj * mass[k] + vk * mass[j];
            for (int e = 0; e < 3; e++)
                g[e] += G * (c[e] * s3 - 3.0 * d[e] * dc * s5 - pv * d[e] * s3);
            /* dL/dm_k: sink j sees source k at x_k: w_j . (x_k - x_j)/s^3 - v_j/s */
            gm += G * (-(wj[0] * d[0] + wj[1] * d[1] + wj[2] * d[2]) * s3 - vj * sinv);
        }
        gpos[3 * k + 0] = g[0];
        gpos[3 * k + 1] = g[1];
        gpos[3 * k + 2] = g[2];
        gmass[k] = gm;
    }
}

/* ---------------------------------------------------------------------------
 * Keys.  Cube frame: lo_d = min x_d, L = max_d (max x_d - min x_d) (1 if 0).
 * c_d = min(floor((x_d - lo_d) * (2^21 / L)), 2^21 - 1), one subtract then one
 * multiply.  key = 2^63 | sum_k bit_k(c_x) << (3k+2) | bit_k(c_y) << (3k+1) |
 * bit_k(c_z) << 3k.
 * ------------------------------------------------------------------------- */
void orc_bbox(int64_t N, const double *pos, double *lo, double *L)
{
    double hi[3];
    for (int d = 0; d < 3; d++) lo[d] = hi[d] = pos[d];
    for (int64_t i = 1; i < N; i++)
        for (int d = 0; d < 3; d++) {
            double x = pos[3 * i + d];
            if (x < lo[d]) lo[d] = x;
            if (x > hi[d]) hi[d] = x;
        }
    double ext = 0.0;
    for (int d = 0; d < 3; d++)
        if (hi[d] - lo[d] > ext) ext = hi[d] - lo[d];
    *L = ext > 0.0 ? ext : 1.0;
}

static uint64_t int_coord(double x, double lo, double s)
{
    double t = (x - lo) * s;
    double f = floor(t);
    uint64_t c = (f <= 0.0) ? 0 : (uint64_t)f;
    if (c > 2097151u) c = 2097151u;
    return c;
}

void orc_keys(int64_t N, const double *pos, const double *lo, double L, uint64_t *keys)
{
    double s = 2097152.0 / L;
    for (int64_t i = 0; i < N; i++) {
        uint64_t c[3];
        for (int d = 0; d < 3; d++) c[d] = int_coord(pos[3 * i + d], lo[d], s);
        uint64_t key = (uint64_t)1 << 63;
        for (int k = 0; k < 21; k++) {
            key |= ((c[0] >> k) & 1u) << (3 * k + 2);
            key |= ((c[1] >> k) & 1u) << (3 * k + 1);
            key |= ((c[2] >> k) & 1u) << (3 * k);
        }
        keys[i] = key;
    }
}

/* ---------------------------------------------------------------------------
 * Sort: stable by key (ties keep the original index order).  Sorting the pairs
 * (key, index) under the total order (key, index) gives exactly that.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint64_t key;
    int64_t idx;
} kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

void orc_sort(int64_t N, const uint64_t *keys, int64_t *perm)
{
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; i++) {
        kv[i].key = keys[i];
        kv[i].idx = i;
    }
    qsort(kv, (size_t)N, sizeof(kv_t), kv_cmp);
    for (int64_t i = 0; i < N; i++) perm[i] = kv[i].idx;
    free(kv);
}

/* ---------------------------------------------------------------------------
 * Multi-indices a = (i, j, k), |a| <= p, in the order used for moment arrays:
 * by degree n ascending; within a degree i descending, then j descending.
 * ------------------------------------------------------------------------- */
static int ncomp(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

static void midx_table(int p, int (*tab)[3])
{
    int c = 0;
    for (int n = 0; n <= p; n++)
        for (int i = n; i >= 0; i--)
            for (int j = n - i; j >= 0; j--) {
                tab[c][0] = i;
                tab[c][1] = j;
                tab[c][2] = n - i - j;
                c++;
            }
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= (double)i;
    return f;
}

/* Raw moments of particles [b, b+n) about z, by definition. */
static void moments_about(const double *spos, const double *smass, int64_t b, int64_t n,
                          const double *z, int p, const int (*tab)[3], double *M)
{
    int nc = ncomp(p);
    for (int c = 0; c < nc; c++) M[c] = 0.0;
    for (int64_t s = b; s < b + n; s++) {
        double d[3], pw[3][ORC_MAXP + 1];
        for (int e = 0; e < 3; e++) {
            d[e] = spos[3 * s + e] - z[e];
            pw[e][0] = 1.0;
            for (int q = 1; q <= p; q++) pw[e][q] = pw[e][q - 1] * d[e];
        }
        for (int c = 0; c < nc; c++)
            M[c] += smass[s] * pw[0][tab[c][0]] * pw[1][tab[c][1]] * pw[2][tab[c][2]];
    }
}

/* ---------------------------------------------------------------------------
 * Derivatives of the softened kernel F(R) = (|R|^2 + eps^2)^{-1/2}.
 * Writing u = |R|^2 + eps^2 and f(u) = u^{-1/2},
 *   d^(i,j,k) F = sum_{l1<=i/2, l2<=j/2, l3<=k/2} c(i,l1) c(j,l2) c(k,l3)
 *                 (2R_x)^{i-2l1} (2R_y)^{j-2l2} (2R_z)^{k-2l3} f^(m)(u),
 *   c(i,l) = i!/(l! (i-2l)!),  m = i+j+k-l1-l2-l3,
 *   f^(m)(u) = (-1)^m (2m-1)!!/2^m u^{-(2m+1)/2}.
 * ------------------------------------------------------------------------- */
static double cfac(int i, int l) { return factorial(i) / (factorial(l) * factorial(i - 2 * l)); }

static double dkernel(int i, int j, int k, double tw[3][ORC_MAXP + 3], const double *fm)
{
    double s = 0.0;
    for (int l1 = 0; 2 * l1 <= i; l1++)
        for (int l2 = 0; 2 * l2 <= j; l2++)
            for (int l3 = 0; 2 * l3 <= k; l3++) {
                int m = i + j + k - l1 - l2 - l3;
                s += cfac(i, l1) * cfac(j, l2) * cfac(k, l3) * tw[0][i - 2 * l1] *
                     tw[1][j - 2 * l2] * tw[2][k - 2 * l3] * fm[m];
            }
    return s;
}

/* One multipole-to-particle interaction (Cartesian expansion to order p):
 *   phi += -G sum_a (-1)^|a| / a! d^a F(R) M_a
 *   acc += +G sum_a (-1)^|a| / a! grad d^a F(R) M_a,      R = x - z.        */
static void m2p_eval(int p, const int (*tab)[3], const double *M, const double *R, double G,
                     double eps2, double *a, double *phi)
{
    double u = R[0] * R[0] + R[1] * R[1] + R[2] * R[2] + eps2;
    double rs = 1.0 / sqrt(u);
    double fm[ORC_MAXP + 3];
    double rpow = rs; /* u^{-(2m+1)/2} */
    double dfact = 1.0; /* (2m-1)!! */
    for (int m = 0; m <= p + 1; m++) {
        if (m > 0) {
            rpow *= rs * rs;
            dfact *= (double)(2 * m - 1);
        }
        double sign = (m % 2) ? -1.0 : 1.0;
        fm[m] = sign * dfact / ldexp(1.0, m) * rpow;
    }
    double tw[3][ORC_MAXP + 3];
    for (int e = 0; e < 3; e++) {
        tw[e][0] = 1.0;
        for (int q = 1; q <= p + 1; q++) tw[e][q] = tw[e][q - 1] * (2.0 * R[e]);
    }
    int nc = ncomp(p);
    double sp = 0.0, sa[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < nc; c++) {
        int i = tab[c][0], j = tab[c][1], k = tab[c][2];
        double w = (((i + j + k) % 2) ? -1.0 : 1.0) /
                   (factorial(i) * factorial(j) * factorial(k)) * M[c];
        sp += w * dkernel(i, j, k, tw, fm);
        sa[0] += w * dkernel(i + 1, j, k, tw, fm);
        sa[1] += w * dkernel(i, j + 1, k, tw, fm);
        sa[2] += w * dkernel(i, j, k + 1, tw, fm);
    }
    *phi -= G * sp;
    a[0] += G * sa[0];
    a[1] += G * sa[1];
    a[2] += G * sa[2];
}

/* Exported for unit tests: one M2P of moments M (order p) at offset R. */
void orc_m2p(int p, const double *M, const double *R, double G, double eps, double *acc,
             double *pot)
{
    int tab[200][3];
    midx_table(p, tab);
    acc[0] = acc[1] = acc[2] = 0.0;
    *pot = 0.0;
    m2p_eval(p, (const int(*)[3])tab, M, R, G, eps * eps, acc, pot);
}

/* The same expansion (moments M about z) at n points x: acc [n][3], pot [n] added to. */
void orc_m2p_points(int p, const double *M, const double *z, int64_t n, const double *x, double G,
                    double eps, double *acc, double *pot)
{
    int tab[200][3];
    midx_table(p, tab);
    for (int64_t i = 0; i < n; i++) {
        double R[3] = {x[3 * i] - z[0], x[3 * i + 1] - z[1], x[3 * i + 2] - z[2]};
        double a[3] = {0.0, 0.0, 0.0}, ph = 0.0;
        m2p_eval(p, (const int(*)[3])tab, M, R, G, eps * eps, a, &ph);
        for (int d = 0; d < 3; d++) acc[3 * i + d] += a[d];
        pot[i] += ph;
    }
}

/* Exported for unit tests: raw moments of a particle set about z. */
void orc_moments(int64_t n, const double *pos, const double *mass, const double *z, int p,
                 double *M)
{
    int tab[200][3];
    midx_table(p, tab);
    moments_about(pos, mass, 0, n, z, p, (const int(*)[3])tab, M);
}

/* Acceptance bound (absolute acceleration error of one cell-body interaction):
 *   E(d) = G/d^2 * 1/(1 - b/d)^2 * [(p+2) B_{p+1}/d^{p+1} - (p+1) B_{p+2}/d^{p+2}],
 * with B_n = sum m |x - z|^n and b = b_max, valid for d > b. */
double orc_mac_bound(double d, double b, double Bp1, double Bp2, int p, double G)
{
    double q = 1.0 - b / d;
    double dp1 = 1.0;
    for (int i = 0; i < p + 1; i++) dp1 *= d;
    double dp2 = dp1 * d;
    return G / (d * d) / (q * q) * ((double)(p + 2) * Bp1 / dp1 - (double)(p + 1) * Bp2 / dp2);
}

/* ---------------------------------------------------------------------------
 * Tree.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t *v;
    int64_t n, cap;
} ivec;

static void ivec_push(ivec *a, int32_t x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 64;
        a->v = (int32_t *)realloc(a->v, sizeof(int32_t) * (size_t)a->cap);
    }
    a->v[a->n++] = x;
}

typedef struct orc_tree {
    int64_t N;
    int leaf_max, group_max;
    double lo[3], L;
    uint64_t *key;   /* particle keys, original order */
    int64_t *perm;   /* perm[s] = original index of sorted slot s */
    int64_t *iperm;  /* iperm[i] = sorted slot of particle i */
    uint64_t *skey;  /* sorted keys */
    double *spos, *smass;
    /* cells, depth-first pre-order, children in ascending octant */
    int64_t ncell, ccap;
    uint64_t *ckey;
    int32_t *clevel, *cparent, *cnchild;
    int32_t (*cchild)[8];
    int64_t *cbegin, *ccount;
    /* groups */
    int64_t ngroup;
    int32_t *gcell;
    double *gcen, *gdmax;
    /* moments (order p) */
    int p;
    double *cmass, *ccom, *cmom, *cbmax, *cB1, *cB2;
    /* lists per group */
    ivec *lm2p, *lp2p, *lborder;
    double tol, Gmac;
    /* force smoothing the lists are built for (Plummer unless set) */
    int soft;
    double soft_eps;
    /* per-interaction order selection: with varq, each accepted cell is evaluated at
     * the lowest order q in [p_lo, p] whose bound meets the tolerance (orders in lm2pq);
     * cBn[(p+3) c + n] = sum m |x - z|^n, n = 0..p+2 */
    int varq, p_lo;
    double *cBn;
    ivec *lm2pq;
    /* periodic images (Sec. "Boundary Conditions"): with per_L > 0 every group also
     * traverses the tree shifted by n per_L, |n|_inf <= per_ws; the image of every list
     * entry in lm2pi / lp2pi (index ((nx+ws) w + ny+ws) w + nz+ws, w = 2 ws + 1) */
    double per_L;
    int per_ws;
    ivec *lm2pi, *lp2pi;
} orc_tree;

static int64_t new_cell(orc_tree *t)
{
    if (t->ncell == t->ccap) {
        int64_t c = t->ccap ? 2 * t->ccap : 1024;
        t->ckey = (uint64_t *)realloc(t->ckey, sizeof(uint64_t) * (size_t)c);
        t->clevel = (int32_t *)realloc(t->clevel, sizeof(int32_t) * (size_t)c);
        t->cparent = (int32_t *)realloc(t->cparent, sizeof(int32_t) * (size_t)c);
        t->cnchild = (int32_t *)realloc(t->cnchild, sizeof(int32_t) * (size_t)c);
        t->cchild = (int32_t(*)[8])realloc(t->cchild, sizeof(int32_t) * 8 * (size_t)c);
        t->cbegin = (int64_t *)realloc(t->cbegin, sizeof(int64_t) * (size_t)c);
        t->ccount = (int64_t *)realloc(t->ccount, sizeof(int64_t) * (size_t)c);
        t->ccap = c;
    }
    return t->ncell++;
}

/* A cell at level < 21 holding more than leaf_max particles is refined into its
 * non-empty octants; the octant of a particle at the next level is the key digit
 * (key >> 3*(20-level)) & 7. */
static void build_rec(orc_tree *t, int64_t begin, int64_t count, uint64_t key, int level,
                      int32_t parent)
{
    int64_t c = new_cell(t);
    t->ckey[c] = key;
    t->clevel[c] = level;
    t->cparent[c] = parent;
    t->cbegin[c] = begin;
    t->ccount[c] = count;
    t->cnchild[c] = 0;
    for (int o = 0; o < 8; o++) t->cchild[c][o] = -1;
    if (level < ORC_MAXLEVEL && count > t->leaf_max) {
        int shift = 3 * (20 - level);
        int64_t b = begin, end = begin + count;
        for (int o = 0; o < 8; o++) {
            int64_t e = b;
            while (e < end && (int)((t->skey[e] >> shift) & 7u) == o) e++;
            if (e > b) {
                int32_t ch = (int32_t)t->ncell;
                build_rec(t, b, e - b, (key << 3) | (uint64_t)o, level + 1, (int32_t)c);
                t->cchild[c][t->cnchild[c]++] = ch;
            }
            b = e;
        }
    }
}

static int is_leaf(const orc_tree *t, int64_t c) { return t->cnchild[c] == 0; }

orc_tree *orc_tree_new(int64_t N, const double *pos, const double *mass, int leaf_max,
                       int group_max)
{
    if (N < 1 || leaf_max < 1 || group_max < 1) return NULL;
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->N = N;
    t->leaf_max = leaf_max;
    t->group_max = group_max;
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    t->perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    t->iperm = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    t->skey = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    t->spos = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    t->smass = (double *)malloc(sizeof(double) * (size_t)N);
    orc_bbox(N, pos, t->lo, &t->L);
    orc_keys(N, pos, t->lo, t->L, t->key);
    orc_sort(N, t->key, t->perm);
    for (int64_t s = 0; s < N; s++) {
        int64_t i = t->perm[s];
        t->iperm[i] = s;
        t->skey[s] = t->key[i];
        for (int d = 0; d < 3; d++) t->spos[3 * s + d] = pos[3 * i + d];
        t->smass[s] = mass[i];
    }
    build_rec(t, 0, N, 1u, 0, -1);
    /* Sink groups: the topmost cells that are leaves or hold <= group_max particles. */
    t->gcell = (int32_t *)malloc(sizeof(int32_t) * (size_t)t->ncell);
    t->ngroup = 0;
    for (int64_t c = 0; c < t->ncell; c++) {
        int small = is_leaf(t, c) || t->ccount[c] <= group_max;
        int top = t->cparent[c] < 0 || t->ccount[t->cparent[c]] > group_max;
        if (small && top) t->gcell[t->ngroup++] = (int32_t)c;
    }
    /* Group centre = centre of the particles' bounding box; Delta_max = max |x - g|. */
    t->gcen = (double *)malloc(sizeof(double) * 3 * (size_t)t->ngroup);
    t->gdmax = (double *)malloc(sizeof(double) * (size_t)t->ngroup);
    for (int64_t g = 0; g < t->ngroup; g++) {
        int64_t c = t->gcell[g], b = t->cbegin[c], n = t->ccount[c];
        double lo[3], hi[3];
        for (int d = 0; d < 3; d++) lo[d] = hi[d] = t->spos[3 * b + d];
        for (int64_t s = b + 1; s < b + n; s++)
            for (int d = 0; d < 3; d++) {
                double x = t->spos[3 * s + d];
                if (x < lo[d]) lo[d] = x;
                if (x > hi[d]) hi[d] = x;
            }
        for (int d = 0; d < 3; d++) t->gcen[3 * g + d] = (lo[d] + hi[d]) * 0.5;
        double r2max = 0.0;
        for (int64_t s = b; s < b + n; s++) {
            double dx = t->spos[3 * s + 0] - t->gcen[3 * g + 0];
            double dy = t->spos[3 * s + 1] - t->gcen[3 * g + 1];
            double dz = t->spos[3 * s + 2] - t->gcen[3 * g + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > r2max) r2max = r2;
        }
        t->gdmax[g] = sqrt(r2max);
    }
    return t;
}

static void free_lists(orc_tree *t)
{
    if (!t->lm2p) return;
    for (int64_t g = 0; g < t->ngroup; g++) {
        free(t->lm2p[g].v);
        free(t->lp2p[g].v);
        free(t->lborder[g].v);
    }
    free(t->lm2p);
    free(t->lp2p);
    free(t->lborder);
    t->lm2p = t->lp2p = t->lborder = NULL;
    if (t->lm2pq) {
        for (int64_t g = 0; g < t->ngroup; g++) free(t->lm2pq[g].v);
        free(t->lm2pq);
        t->lm2pq = NULL;
    }
    if (t->lm2pi) {
        for (int64_t g = 0; g < t->ngroup; g++) {
            free(t->lm2pi[g].v);
            free(t->lp2pi[g].v);
        }
        free(t->lm2pi);
        free(t->lp2pi);
        t->lm2pi = t->lp2pi = NULL;
    }
}

/* Images of the periodic tree: their number, the central one, and the shift of one. */
static int per_nimg(const orc_tree *t)
{
    int w = 2 * t->per_ws + 1;
    return t->per_L > 0.0 ? w * w * w : 1;
}
static int per_central(const orc_tree *t) { return (per_nimg(t) - 1) / 2; }
static void per_shift(const orc_tree *t, int img, double sh[3])
{
    if (!(t->per_L > 0.0)) {
        sh[0] = sh[1] = sh[2] = 0.0;
        return;
    }
    int w = 2 * t->per_ws + 1;
    sh[0] = (double)(img / (w * w) - t->per_ws) * t->per_L;
    sh[1] = (double)((img / w) % w - t->per_ws) * t->per_L;
    sh[2] = (double)(img % w - t->per_ws) * t->per_L;
}

/* Periodic images for the lists and forces: side L > 0 of the periodic cube and the
 * number ws of neighbouring cubes on every side whose images the tree serves (the rest
 * is the far field's); L = 0 restores open boundaries.  Set before the traversal. */
int orc_tree_periodic(orc_tree *t, double L, int ws)
{
    if (!(L >= 0.0) || ws < 0 || ws > 4) return -1;
    t->per_L = L;
    t->per_ws = ws;
    return 0;
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    free_lists(t);
    free(t->key); free(t->perm); free(t->iperm); free(t->skey); free(t->spos); free(t->smass);
    free(t->ckey); free(t->clevel); free(t->cparent); free(t->cnchild); free(t->cchild);
    free(t->cbegin); free(t->ccount);
    free(t->gcell); free(t->gcen); free(t->gdmax);
    free(t->cmass); free(t->ccom); free(t->cmom); free(t->cbmax); free(t->cB1); free(t->cB2); free(t->cBn);
    free(t);
}

/* info: [N, ncell, ngroup, nleaf, max level, p] */
void orc_tree_info(const orc_tree *t, int64_t *info)
{
    int64_t nleaf = 0, maxl = 0;
    for (int64_t c = 0; c < t->ncell; c++) {
        if (is_leaf(t, c)) nleaf++;
        if (t->clevel[c] > maxl) maxl = t->clevel[c];
    }
    info[0] = t->N;
    info[1] = t->ncell;
    info[2] = t->ngroup;
    info[3] = nleaf;
    info[4] = maxl;
    info[5] = t->p;
}

void orc_tree_frame(const orc_tree *t, double *lo, double *L)
{
    for (int d = 0; d < 3; d++) lo[d] = t->lo[d];
    *L = t->L;
}

void orc_tree_keys(const orc_tree *t, uint64_t *keys, int64_t *perm)
{
    memcpy(keys, t->key, sizeof(uint64_t) * (size_t)t->N);
    memcpy(perm, t->perm, sizeof(int64_t) * (size_t)t->N);
}

void orc_tree_cells(const orc_tree *t, uint64_t *key, int32_t *level, int64_t *begin,
                    int64_t *count, int32_t *parent, int32_t *nchild)
{
    for (int64_t c = 0; c < t->ncell; c++) {
        key[c] = t->ckey[c];
        level[c] = t->clevel[c];
        begin[c] = t->cbegin[c];
        count[c] = t->ccount[c];
        parent[c] = t->cparent[c];
        nchild[c] = t->cnchild[c];
    }
}

void orc_tree_groups(const orc_tree *t, int32_t *cell, double *centre, double *dmax)
{
    for (int64_t g = 0; g < t->ngroup; g++) {
        cell[g] = t->gcell[g];
        for (int d = 0; d < 3; d++) centre[3 * g + d] = t->gcen[3 * g + d];
        dmax[g] = t->gdmax[g];
    }
}

/* Moments of every cell by definition from its own particles (no translation):
 * m = sum m_j, z = sum m_j x_j / m, M_a = sum m_j (x_j - z)^a (|a| <= p),
 * b_max = max |x_j - z|, B_{p+1} = sum m_j |x_j - z|^{p+1}, B_{p+2} likewise. */
int orc_tree_moments(orc_tree *t, int p)
{
    if (p < 0 || p > ORC_MAXP) return -1;
    int nc = ncomp(p);
    int tab[200][3];
    midx_table(p, tab);
    t->p = p;
    free(t->cmass); free(t->ccom); free(t->cmom); free(t->cbmax); free(t->cB1); free(t->cB2); free(t->cBn);
    t->varq = 0;
    t->cBn = (double *)malloc(sizeof(double) * (size_t)(p + 3) * (size_t)t->ncell);
    t->cmass = (double *)malloc(sizeof(double) * (size_t)t->ncell);
    t->ccom = (double *)malloc(sizeof(double) * 3 * (size_t)t->ncell);
    t->cmom = (double *)malloc(sizeof(double) * (size_t)nc * (size_t)t->ncell);
    t->cbmax = (double *)malloc(sizeof(double) * (size_t)t->ncell);
    t->cB1 = (double *)malloc(sizeof(double) * (size_t)t->ncell);
    t->cB2 = (double *)malloc(sizeof(double) * (size_t)t->ncell);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < t->ncell; c++) {
        int64_t b = t->cbegin[c], n = t->ccount[c];
        double m = 0.0, mx[3] = {0.0, 0.0, 0.0};
        for (int64_t s = b; s < b + n; s++) {
            m += t->smass[s];
            for (int d = 0; d < 3; d++) mx[d] += t->smass[s] * t->spos[3 * s + d];
        }
        double *z = t->ccom + 3 * c;
        for (int d = 0; d < 3; d++) z[d] = mx[d] / m;
        t->cmass[c] = m;
        moments_about(t->spos, t->smass, b, n, z, p, (const int(*)[3])tab, t->cmom + (size_t)nc * c);
        double bmax = 0.0, B1 = 0.0, B2 = 0.0;
        for (int64_t s = b; s < b + n; s++) {
            double dx = t->spos[3 * s + 0] - z[0];
            double dy = t->spos[3 * s + 1] - z[1];
            double dz = t->spos[3 * s + 2] - z[2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r > bmax) bmax = r;
            double rp = 1.0;
            for (int i = 0; i < p + 1; i++) rp *= r;
            B1 += t->smass[s] * rp;
            B2 += t->smass[s] * rp * r;
        }
        t->cbmax[c] = bmax;
        t->cB1[c] = B1;
        t->cB2[c] = B2;
        double *Bn = t->cBn + (size_t)(p + 3) * c;
        for (int q = 0; q < p + 3; q++) Bn[q] = 0.0;
        for (int64_t s = b; s < b + n; s++) {
            double dx = t->spos[3 * s + 0] - z[0];
            double dy = t->spos[3 * s + 1] - z[1];
            double dz = t->spos[3 * s + 2] - z[2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double rq = 1.0;
            for (int q = 0; q < p + 3; q++) {
                Bn[q] += t->smass[s] * rq;
                rq *= r;
            }
        }
    }
    return 0;
}

/* Per-interaction order selection (Sec. "Multipole Error Bounds": the bounds decide
 * between orders of expansion and refinement): after orc_tree_moments(p), orders
 * p_lo..p; every accepted cell is then evaluated at the lowest order whose bound meets
 * the tolerance.  p_lo < 0 restores the fixed order p. */
int orc_tree_order_range(orc_tree *t, int p_lo)
{
    if (!t->cmom || p_lo > t->p) return -1;
    t->varq = p_lo >= 0;
    t->p_lo = p_lo >= 0 ? p_lo : t->p;
    return 0;
}

void orc_tree_get_moments(const orc_tree *t, double *mass, double *com, double *mom,
                          double *bmax, double *B1, double *B2)
{
    int nc = ncomp(t->p);
    memcpy(mass, t->cmass, sizeof(double) * (size_t)t->ncell);
    memcpy(com, t->ccom, sizeof(double) * 3 * (size_t)t->ncell);
    memcpy(mom, t->cmom, sizeof(double) * (size_t)nc * (size_t)t->ncell);
    memcpy(bmax, t->cbmax, sizeof(double) * (size_t)t->ncell);
    memcpy(B1, t->cB1, sizeof(double) * (size_t)t->ncell);
    memcpy(B2, t->cB2, sizeof(double) * (size_t)t->ncell);
}

/* Is cell c the group's cell or one of its ancestors?  Keys carry a leading
 * placeholder bit, so an ancestor's key is the group key shifted right. */
static int ancestor_or_self(const orc_tree *t, int64_t c, int64_t gc)
{
    int dl = t->clevel[gc] - t->clevel[c];
    if (dl < 0) return 0;
    return (t->ckey[gc] >> (3 * dl)) == t->ckey[c];
}

/* Is cell c inside the group's cell (a proper descendant)?  Its particles are all sinks
 * of the group, within Delta_max of g, so its centre of mass is too: d <= 0, never
 * accepted.  Taken by this rule rather than by the rounded d, which can come out a unit in
 * the last place above 0 for a one-particle leaf at the group's farthest point (and would
 * then make that sink meet itself through the expansion). */
static int inside_group(const orc_tree *t, int64_t c, int64_t gc)
{
    int dl = t->clevel[c] - t->clevel[gc];
    if (dl <= 0) return 0;
    return (t->ckey[c] >> (3 * dl)) == t->ckey[gc];
}

/* Traversal for one group, depth first from cell c, children in ascending octant:
 *   ancestor-or-self of the group -> descend (a leaf here is the group itself -> P2P)
 *   inside the group's cell -> descend, a leaf -> P2P (d <= 0)
 *   otherwise d = |z_c - g| - Delta_max;
 *     d > b_max and E(d) <= tol -> M2P
 *     else leaf                 -> P2P
 *     else                      -> descend
 * Decisions within 1e-9 (relative) of a threshold are recorded as borderline. */
static void push_m2p(orc_tree *t, int64_t g, int64_t c, int img)
{
    ivec_push(&t->lm2p[g], (int32_t)c);
    if (t->lm2pi) ivec_push(&t->lm2pi[g], img);
}
static void push_p2p(orc_tree *t, int64_t g, int64_t c, int img)
{
    ivec_push(&t->lp2p[g], (int32_t)c);
    if (t->lp2pi) ivec_push(&t->lp2pi[g], img);
}

static void trav_rec(orc_tree *t, int64_t g, int64_t c, int img)
{
    int64_t gc = t->gcell[g];
    if (img == per_central(t) && (ancestor_or_self(t, c, gc) || inside_group(t, c, gc))) {
        if (is_leaf(t, c))
            push_p2p(t, g, c, img);
        else
            for (int k = 0; k < t->cnchild[c]; k++) trav_rec(t, g, t->cchild[c][k], img);
        return;
    }
    const double *z0 = t->ccom + 3 * c;
    double z[3] = {z0[0], z0[1], z0[2]};
    if (t->per_L > 0.0) {
        double sh[3];
        per_shift(t, img, sh);
        for (int d = 0; d < 3; d++) z[d] += sh[d];
    }
    double dx = z[0] - t->gcen[3 * g + 0];
    double dy = z[1] - t->gcen[3 * g + 1];
    double dz = z[2] - t->gcen[3 * g + 2];
    double dist = sqrt(dx * dx + dy * dy + dz * dz);
    double d = dist - t->gdmax[g];
    double b = t->cbmax[c];
    int accept = 0;
    /* K1: accepted only if no sink comes within eps of a source of the cell */
    int guard = !soft_compact(t->soft) || d >= b + t->soft_eps;
    if (soft_compact(t->soft) && b + t->soft_eps > 0.0 && fabs(d - (b + t->soft_eps)) <= 1e-9 * (b + t->soft_eps))
        ivec_push(&t->lborder[g], (int32_t)c);
    if (t->varq) {
        /* the lowest order in [p_lo, p] whose bound meets the tolerance */
        int qa = -1;
        if (d > b && guard) {
            const double *Bn = t->cBn + (size_t)(t->p + 3) * c;
            for (int q = t->p_lo; q <= t->p && qa < 0; q++) {
                double E = orc_mac_bound(d, b, Bn[q + 1], Bn[q + 2], q, t->Gmac);
                if (fabs(E - t->tol) <= 1e-9 * t->tol) ivec_push(&t->lborder[g], (int32_t)c);
                if (E <= t->tol) qa = q;
            }
        }
        if (b > 0.0 && fabs(d - b) <= 1e-9 * b) ivec_push(&t->lborder[g], (int32_t)c);
        if (qa >= 0) {
            push_m2p(t, g, c, img);
            ivec_push(&t->lm2pq[g], (int32_t)qa);
        } else if (is_leaf(t, c)) {
            push_p2p(t, g, c, img);
        } else {
            for (int k = 0; k < t->cnchild[c]; k++) trav_rec(t, g, t->cchild[c][k], img);
        }
        return;
    }
    if (d > b) {
        double E = orc_mac_bound(d, b, t->cB1[c], t->cB2[c], t->p, t->Gmac);
        accept = guard && E <= t->tol;
        if (fabs(E - t->tol) <= 1e-9 * t->tol) ivec_push(&t->lborder[g], (int32_t)c);
    }
    if (b > 0.0 && fabs(d - b) <= 1e-9 * b) ivec_push(&t->lborder[g], (int32_t)c);
    if (accept)
        push_m2p(t, g, c, img);
    else if (is_leaf(t, c))
        push_p2p(t, g, c, img);
    else
        for (int k = 0; k < t->cnchild[c]; k++) trav_rec(t, g, t->cchild[c][k], img);
}

/* All lists of group g: the central tree and, when periodic, every image. */
static void trav_group(orc_tree *t, int64_t g)
{
    for (int img = 0; img < per_nimg(t); img++) trav_rec(t, g, 0, img);
}

static void alloc_lists(orc_tree *t)
{
    t->lm2p = (ivec *)calloc((size_t)t->ngroup, sizeof(ivec));
    t->lp2p = (ivec *)calloc((size_t)t->ngroup, sizeof(ivec));
    t->lborder = (ivec *)calloc((size_t)t->ngroup, sizeof(ivec));
    if (t->varq) t->lm2pq = (ivec *)calloc((size_t)t->ngroup, sizeof(ivec));
    if (t->per_L > 0.0) {
        t->lm2pi = (ivec *)calloc((size_t)t->ngroup, sizeof(ivec));
        t->lp2pi = (ivec *)calloc((size_t)t->ngroup, sizeof(ivec));
    }
}

/* Force smoothing of the lists and forces: kind ORC_SOFT_PLUMMER (default) or
 * ORC_SOFT_K1 or ORC_SOFT_SPLINE with support eps.  Set before the traversal. */
int orc_tree_softening(orc_tree *t, int kind, double eps)
{
    if ((kind != ORC_SOFT_PLUMMER && !soft_compact(kind)) || !(eps >= 0.0)) return -1;
    t->soft = kind;
    t->soft_eps = eps;
    return 0;
}

/* The smoothing of a force call: the tree's kind with the given eps; K1 needs the eps
 * its lists were built with (-2 otherwise). */
static int force_soft(const orc_tree *t, double eps, orc_soft *sf)
{
    sf->kind = t->soft;
    sf->eps = eps;
    return (soft_compact(t->soft) && eps != t->soft_eps) ? -2 : 0;
}

int orc_tree_traverse(orc_tree *t, double tol, double G)
{
    if (!t->cmom || tol <= 0.0) return -1;
    free_lists(t);
    t->tol = tol;
    t->Gmac = G;
    alloc_lists(t);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t g = 0; g < t->ngroup; g++) trav_group(t, g);
    return 0;
}

/* sizes[3*g + {0,1,2}] = M2P cells, P2P leaves, borderline cells of group g */
void orc_tree_list_sizes(const orc_tree *t, int64_t *sizes)
{
    for (int64_t g = 0; g < t->ngroup; g++) {
        sizes[3 * g + 0] = t->lm2p[g].n;
        sizes[3 * g + 1] = t->lp2p[g].n;
        sizes[3 * g + 2] = t->lborder[g].n;
    }
}

/* Order of every M2P entry, concatenated like the M2P lists (p everywhere with a fixed
 * order). */
void orc_tree_list_orders(const orc_tree *t, int32_t *orders)
{
    int64_t a = 0;
    for (int64_t g = 0; g < t->ngroup; g++)
        for (int64_t e = 0; e < t->lm2p[g].n; e++) orders[a++] = t->lm2pq ? t->lm2pq[g].v[e] : t->p;
}

/* Image of every M2P and P2P entry, concatenated like the lists (0 without periodicity). */
void orc_tree_list_images(const orc_tree *t, int32_t *m2p_img, int32_t *p2p_img)
{
    int64_t a = 0, b = 0;
    for (int64_t g = 0; g < t->ngroup; g++) {
        for (int64_t e = 0; e < t->lm2p[g].n; e++) m2p_img[a++] = t->lm2pi ? t->lm2pi[g].v[e] : 0;
        for (int64_t e = 0; e < t->lp2p[g].n; e++) p2p_img[b++] = t->lp2pi ? t->lp2pi[g].v[e] : 0;
    }
}

/* Concatenated lists in group order. */
void orc_tree_lists(const orc_tree *t, int32_t *m2p, int32_t *p2p, int32_t *border)
{
    int64_t a = 0, b = 0, c = 0;
    for (int64_t g = 0; g < t->ngroup; g++) {
        memcpy(m2p + a, t->lm2p[g].v, sizeof(int32_t) * (size_t)t->lm2p[g].n);
        memcpy(p2p + b, t->lp2p[g].v, sizeof(int32_t) * (size_t)t->lp2p[g].n);
        memcpy(border + c, t->lborder[g].v, sizeof(int32_t) * (size_t)t->lborder[g].n);
        a += t->lm2p[g].n;
        b += t->lp2p[g].n;
        c += t->lborder[g].n;
    }
}

/* Expansion order of M2P entry e of group g (the moments' order p unless selected per
 * interaction; lower orders use the leading components, which are ordered by degree). */
static int m2p_order(const orc_tree *t, int64_t g, int64_t e) { return t->lm2pq ? t->lm2pq[g].v[e] : t->p; }

/* Force on the sinks of one group from its lists, given per-cell moments and
 * (frozen) expansion centres.  Outputs are written at the sinks' original indices. */
static void group_force(const orc_tree *t, int64_t g, const double *spos, const double *smass,
                        const double *mom, const int (*tab)[3], double G, orc_soft sf,
                        double *acc, double *pot)
{
    int nc = ncomp(t->p);
    double eps2 = m2p_eps2(sf);
    int64_t gc = t->gcell[g];
    for (int64_t s = t->cbegin[gc]; s < t->cbegin[gc] + t->ccount[gc]; s++) {
        double a[3] = {0.0, 0.0, 0.0}, phi = 0.0;
        const double *x = spos + 3 * s;
        for (int64_t e = 0; e < t->lm2p[g].n; e++) {
            int64_t c = t->lm2p[g].v[e];
            double R[3], sh[3];
            per_shift(t, t->lm2pi ? t->lm2pi[g].v[e] : 0, sh);
            for (int d = 0; d < 3; d++) R[d] = x[d] - (t->ccom[3 * c + d] + sh[d]);
            m2p_eval(m2p_order(t, g, e), tab, mom + (size_t)nc * c, R, G, eps2, a, &phi);
        }
        for (int64_t e = 0; e < t->lp2p[g].n; e++) {
            int64_t c = t->lp2p[g].v[e];
            const int img = t->lp2pi ? t->lp2pi[g].v[e] : per_central(t);
            double sh[3];
            per_shift(t, img, sh);
            for (int64_t j = t->cbegin[c]; j < t->cbegin[c] + t->ccount[c]; j++) {
                if (j == s && img == per_central(t)) continue;
                if (t->per_L > 0.0) {
                    const double xj[3] = {spos[3 * j] + sh[0], spos[3 * j + 1] + sh[1], spos[3 * j + 2] + sh[2]};
                    pair_acc(x, xj, smass[j], G, sf, a, &phi);
                } else {
                    pair_acc(x, spos + 3 * j, smass[j], G, sf, a, &phi);
                }
            }
        }
        int64_t i = t->perm[s];
        for (int d = 0; d < 3; d++) acc[3 * i + d] = a[d];
        if (pot) pot[i] = phi;
    }
}

/* Tree force for the sinks of the listed groups (all groups if gsel == NULL).
 * acc [N][3], pot [N] in original particle order; untouched for other sinks. */
int orc_tree_force(const orc_tree *t, double G, double eps, int64_t nsel, const int64_t *gsel,
                   double *acc, double *pot)
{
    if (!t->lm2p) return -1;
    int tab[200][3];
    midx_table(t->p, tab);
    orc_soft sf;
    if (force_soft(t, eps, &sf)) return -2;
    if (!gsel) nsel = t->ngroup;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nsel; q++) {
        int64_t g = gsel ? gsel[q] : q;
        group_force(t, g, t->spos, t->smass, t->cmom, (const int(*)[3])tab, G, sf, acc, pot);
    }
    return 0;
}

/* Traversal of selected groups only (for timing samples).  Lists of other
 * groups are left empty. */
int orc_tree_traverse_groups(orc_tree *t, double tol, double G, int64_t nsel, const int64_t *gsel)
{
    if (!t->cmom || tol <= 0.0) return -1;
    free_lists(t);
    t->tol = tol;
    t->Gmac = G;
    alloc_lists(t);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nsel; q++) trav_group(t, gsel[q]);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Frozen-structure tree function, for finite differences of the adjoint.
 * The sorted order, the cells' particle ranges, the lists and the expansion
 * centres z_c are those of the tree; the moments are recomputed about the
 * frozen z_c from the given (perturbed) positions and masses.
 *   L = sum_i w_i . a_i + sum_i v_i phi_i      (v may be NULL)
 * With k >= 0, only the terms that depend on particle k (original index) are
 * summed: sink k's own force, and for every other sink the one list entry
 * (cell or leaf) that contains k.  Every other term of L is independent of
 * particle k, so finite differences of this partial sum equal those of L.
 * ------------------------------------------------------------------------- */
double orc_frozen_loss(const orc_tree *t, const double *pos, const double *mass, double G,
                       double eps, const double *w, const double *v, int64_t k)
{
    if (!t->lm2p || t->per_L > 0.0) return NAN;  /* open boundaries only */
    int64_t N = t->N;
    int p = t->p, nc = ncomp(p);
    int tab[200][3];
    midx_table(p, tab);
    orc_soft sf;
    if (force_soft(t, eps, &sf)) return NAN;
    double eps2 = m2p_eps2(sf);
    double *spos = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *smass = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t s = 0; s < N; s++) {
        int64_t i = t->perm[s];
        for (int d = 0; d < 3; d++) spos[3 * s + d] = pos[3 * i + d];
        smass[s] = mass[i];
    }
    int64_t sk = k >= 0 ? t->iperm[k] : -1;
    /* Moments about the frozen centres.  With k >= 0 only cells containing k
     * can differ from the stored ones; the others are reused as stored. */
    double *mom = (double *)malloc(sizeof(double) * (size_t)nc * (size_t)t->ncell);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < t->ncell; c++) {
        int inside = sk >= t->cbegin[c] && sk < t->cbegin[c] + t->ccount[c];
        if (k < 0 || inside)
            moments_about(spos, smass, t->cbegin[c], t->ccount[c], t->ccom + 3 * c, p,
                          (const int(*)[3])tab, mom + (size_t)nc * c);
        else
            memcpy(mom + (size_t)nc * c, t->cmom + (size_t)nc * c, sizeof(double) * (size_t)nc);
    }
    double L = 0.0;
    if (k < 0) {
        double *acc = (double *)malloc(sizeof(double) * 3 * (size_t)N);
        double *pot = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t g = 0; g < t->ngroup; g++)
            group_force(t, g, spos, smass, mom, (const int(*)[3])tab, G, sf, acc, pot);
        for (int64_t i = 0; i < N; i++) {
            L += w[3 * i] * acc[3 * i] + w[3 * i + 1] * acc[3 * i + 1] + w[3 * i + 2] * acc[3 * i + 2];
            if (v) L += v[i] * pot[i];
        }
        free(acc);
        free(pot);
    } else {
        /* sink k's own force: its group's full lists */
        int64_t gk = -1;
        for (int64_t g = 0; g < t->ngroup && gk < 0; g++) {
            int64_t gc = t->gcell[g];
            if (sk >= t->cbegin[gc] && sk < t->cbegin[gc] + t->ccount[gc]) gk = g;
        }
        {
            double a[3] = {0.0, 0.0, 0.0}, phi = 0.0;
            const double *x = spos + 3 * sk;
            for (int64_t e = 0; e < t->lm2p[gk].n; e++) {
                int64_t c = t->lm2p[gk].v[e];
                double R[3];
                for (int d = 0; d < 3; d++) R[d] = x[d] - t->ccom[3 * c + d];
                m2p_eval(m2p_order(t, gk, e), (const int(*)[3])tab, mom + (size_t)nc * c, R, G, eps2, a, &phi);
            }
            for (int64_t e = 0; e < t->lp2p[gk].n; e++) {
                int64_t c = t->lp2p[gk].v[e];
                for (int64_t j = t->cbegin[c]; j < t->cbegin[c] + t->ccount[c]; j++)
                    if (j != sk) pair_acc(x, spos + 3 * j, smass[j], G, sf, a, &phi);
            }
            L += w[3 * k] * a[0] + w[3 * k + 1] * a[1] + w[3 * k + 2] * a[2];
            if (v) L += v[k] * phi;
        }
        /* every other sink: the entries of its group's lists that contain k */
        double Lo = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : Lo)
        for (int64_t g = 0; g < t->ngroup; g++) {
            int64_t gc = t->gcell[g];
            for (int64_t e = 0; e < t->lm2p[g].n; e++) {
                int64_t c = t->lm2p[g].v[e];
                if (!(sk >= t->cbegin[c] && sk < t->cbegin[c] + t->ccount[c])) continue;
                for (int64_t s = t->cbegin[gc]; s < t->cbegin[gc] + t->ccount[gc]; s++) {
                    if (s == sk) continue;
                    double a[3] = {0.0, 0.0, 0.0}, phi = 0.0, R[3];
                    for (int d = 0; d < 3; d++) R[d] = spos[3 * s + d] - t->ccom[3 * c + d];
                    m2p_eval(m2p_order(t, g, e), (const int(*)[3])tab, mom + (size_t)nc * c, R, G, eps2, a, &phi);
                    int64_t i = t->perm[s];
                    Lo += w[3 * i] * a[0] + w[3 * i + 1] * a[1] + w[3 * i + 2] * a[2];
                    if (v) Lo += v[i] * phi;
                }
            }
            for (int64_t e = 0; e < t->lp2p[g].n; e++) {
                int64_t c = t->lp2p[g].v[e];
                if (!(sk >= t->cbegin[c] && sk < t->cbegin[c] + t->ccount[c])) continue;
                for (int64_t s = t->cbegin[gc]; s < t->cbegin[gc] + t->ccount[gc]; s++) {
                    if (s == sk) continue;
                    double a[3] = {0.0, 0.0, 0.0}, phi = 0.0;
                    pair_acc(spos + 3 * s, spos + 3 * sk, smass[sk], G, sf, a, &phi);
                    int64_t i = t->perm[s];
                    Lo += w[3 * i] * a[0] + w[3 * i + 1] * a[1] + w[3 * i + 2] * a[2];
                    if (v) Lo += v[i] * phi;
                }
            }
        }
        L += Lo;
    }
    free(spos);
    free(smass);
    free(mom);
    return L;
}

/* Frozen-structure force: the tree's sorted order, cell ranges, lists and expansion
 * centres, with every cell's moments recomputed about its frozen centre from the given
 * positions and masses (original order).  acc [N][3], pot [N] or NULL, original order.
 * At the tree's own positions this is the tree force. */
int orc_frozen_force(const orc_tree *t, const double *pos, const double *mass, double G, double eps,
                     double *acc, double *pot)
{
    if (!t->lm2p) return -1;
    int64_t N = t->N;
    int p = t->p, nc = ncomp(p);
    int tab[200][3];
    midx_table(p, tab);
    orc_soft sf;
    if (force_soft(t, eps, &sf)) return -2;
    double *spos = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *smass = (double *)malloc(sizeof(double) * (size_t)N);
    double *ph = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t s = 0; s < N; s++) {
        int64_t i = t->perm[s];
        for (int d = 0; d < 3; d++) spos[3 * s + d] = pos[3 * i + d];
        smass[s] = mass[i];
    }
    double *mom = (double *)malloc(sizeof(double) * (size_t)nc * (size_t)t->ncell);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < t->ncell; c++)
        moments_about(spos, smass, t->cbegin[c], t->ccount[c], t->ccom + 3 * c, p, (const int(*)[3])tab,
                      mom + (size_t)nc * c);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t g = 0; g < t->ngroup; g++)
        group_force(t, g, spos, smass, mom, (const int(*)[3])tab, G, sf, acc, ph);
    if (pot) memcpy(pot, ph, sizeof(double) * (size_t)N);
    free(spos);
    free(smass);
    free(ph);
    free(mom);
    return 0;
}
