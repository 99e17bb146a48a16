// hot_traverse.cu -- group-wise tree traversal into interaction lists (Warren 2013,
// Sec. "Improving instruction-level parallelism": a sink cell's n particles share the
// list of m source cells; Sec. "Multipole Error Bounds" and Fig. "mac": the acceptance
// test bounds the absolute acceleration error of each cell-body interaction).
//
// One warp per sink group.  The warp tests 32 cells of the current frontier at a time;
// accepted cells go to the M2P list, rejected leaves to the P2P list, and the children
// of rejected inner cells form the next frontier (kept in per-warp global scratch).  One
// pass writes each group's lists into per-group slots sized from the previous call's
// largest counts, and a compaction copies them into CSR order; a group that does not fit
// its slots makes that call fall back to a count pass, a scan and an identical fill
// pass.  Every decision depends only on the (cell, group) pair, so the lists equal those
// of a depth-first traversal as sets; within a list the order is by level, then by
// parent, then octant.
#include "hot_common.cuh"

namespace {

constexpr int TW = 8;  // warps per block

// Ascending 16-bit sort key of a descending cost: the cost's binary exponent and the 11
// bits below its leading one (monotone, 1/2048 relative resolution: enough to order the
// work largest first; the sort then needs two passes instead of four).
__device__ __forceinline__ uint64_t cost_key16(uint64_t cost)
{
    if (cost == 0) return 0xffffull;
    const uint64_t c = cost < 0xffffffffull ? cost : 0xffffffffull;
    const int e = 63 - __clzll((long long)c);  // 0..31
    const uint32_t m = e >= 11 ? (uint32_t)(c >> (e - 11)) & 0x7ffu : (uint32_t)(c << (11 - e)) & 0x7ffu;
    return 0xffffull - (((uint64_t)e << 11) | m);
}

// Absolute acceleration error bound of one accepted cell at distance d (d > b):
// E(d) = G/d^2 (1 - b/d)^-2 [(p+2) B_{p+1}/d^{p+1} - (p+1) B_{p+2}/d^{p+2}]
__device__ __forceinline__ double mac_bound(double d, double b, double B1, double B2, int p, double G)
{
    double q = __dsub_rn(1.0, __ddiv_rn(b, d));
    double dp1 = 1.0;
    for (int i = 0; i < p + 1; ++i) dp1 = __dmul_rn(dp1, d);
    double dp2 = __dmul_rn(dp1, d);
    double t1 = __ddiv_rn(__dmul_rn((double)(p + 2), B1), dp1);
    double t2 = __ddiv_rn(__dmul_rn((double)(p + 1), B2), dp2);
    return __dmul_rn(__ddiv_rn(__ddiv_rn(G, __dmul_rn(d, d)), __dmul_rn(q, q)), __dsub_rn(t1, t2));
}

// ln E(d) - ln tol and its derivative in ln d, for the radius solver (any rounding: the
// traversal re-takes decisions near the threshold with mac_bound itself).  With
// T(d) d^{p+2} = (p+2) B_{p+1} d - (p+1) B_{p+2} > 0 on (b, inf):
//   d (ln E)'(d) = -2 - 2b/(d - b) - (p+1)(p+2)(B_{p+1} d - B_{p+2}) / ((p+2) B_{p+1} d - (p+1) B_{p+2})
__device__ __forceinline__ void mac_log_newton(double d, double b, double B1, double B2, int p, double G,
                                               double ltol, double &f, double &df)
{
    const double q = 1.0 - b / d;
    const double tn = (p + 2) * B1 * d - (p + 1) * B2;  // T(d) d^{p+2}
    // ln E = ln G - 2 ln d - 2 ln q + ln tn - (p+2) ln d
    f = log(G) - (p + 4) * log(d) - 2.0 * log(q) + log(tn) - ltol;
    df = -2.0 - 2.0 * b / (d - b) - (double)((p + 1) * (p + 2)) * (B1 * d - B2) / tn;
}

// Acceptance radius of every cell for the tolerance: E is strictly decreasing on
// (b_max, inf), so "d > b_max and E(d) <= tol" is "d >= r_c" with E(r_c) = tol.  A
// bracket [lo, hi] with E(lo) > tol >= E(hi) is found around the far-field estimate
// d0 = (G (p+2) B_{p+1} / tol)^(1/(p+3)) (the leading term of E), by doubling up or
// halving down from it (one or two evaluations of E on most cells, where doubling up
// from b_max took log2(r_c / b_max)), then Newton steps in ln d on ln E - ln tol (which
// is nearly linear in ln d; the first ones in float32), falling back to bisection whenever
// a step leaves the bracket, until a step or the bracket is below 1e-11 relative (r_c = 0
// when b_max = 0, where E vanishes).  That accuracy moves (d_max + r_c)^2 by at most 2e-11
// relative, far inside the 1e-9 band in which the traversal re-takes decisions with the
// bound itself.
// guard > 0 (K1 smoothing, guard = eps) also requires d >= b_max + guard, so that every
// source of an accepted cell is at least eps from every sink: r_c = max(r_c, b_max + guard)
// (guard = 0 leaves r_c, which is above b_max, unchanged).
__device__ double mac_radius_solve(double b, double B1, double B2, int p, double G, double tol)
{
    double rc = 0.0;
    if (b > 0.0) {
        double d0 = pow(G * (p + 2) * B1 / tol, 1.0 / (p + 3));
        if (!(d0 > 1.0001 * b)) d0 = 2.0 * b;  // also for a non-finite estimate
        double lo = b, hi = d0;
        int k = 0;
        if (mac_bound(d0, b, B1, B2, p, G) <= tol) {
            // halve down towards b while the bound still holds
            while (k < 1100) {
                const double t = 0.5 * hi;
                if (!(t > b) || !(mac_bound(t, b, B1, B2, p, G) <= tol)) {
                    lo = t > b ? t : b;
                    break;
                }
                hi = t;
                ++k;
            }
        } else {
            lo = d0;
            hi = 2.0 * d0;
            while (!(mac_bound(hi, b, B1, B2, p, G) <= tol) && k < 1100) {
                lo = hi;
                hi *= 2.0;
                ++k;
            }
        }
        if (k >= 1100) {
            rc = INFINITY;
        } else {
            const double ltol = log(tol);
            double d = hi;
            // float32 Newton steps first, on the same function written with rho = B_{p+2} /
            // B_{p+1} and C = ln G + ln B_{p+1} - ln tol (so that no float32 quantity
            // under- or overflows): f = C - (p+3) ln d - 2 ln(1 - b/d) + ln((p+2) - (p+1)
            // rho/d), inside the bracket, until a step is below 1e-6 relative; the float64
            // steps below then take one or two iterations where they took about six from
            // the bracket end
            if (B1 > 0.0) {
                const float Cf = (float)(log(G) + log(B1) - ltol);
                const float bf = (float)b, rf = (float)(B2 / B1), lof = (float)lo, hif = (float)hi;
                const float c1 = (float)(p + 1), c2 = (float)(p + 2), c3 = (float)(p + 3);
                float x = (float)d;
                for (int it = 0; it < 12; ++it) {
                    const float q = 1.f - bf / x;
                    const float u = c2 - c1 * rf / x;
                    if (!(q > 0.f) || !(u > 0.f)) break;
                    const float f = Cf - c3 * logf(x) - 2.f * logf(q) + logf(u);
                    const float df = -2.f - 2.f * bf / (x - bf) - c1 * c2 * (x - rf) / (c2 * x - c1 * rf);
                    const float xn = x * expf(-f / df);
                    if (!(xn > lof && xn < hif)) break;  // left to the float64 steps
                    const bool done = fabsf(xn - x) <= 1e-6f * x;
                    x = xn;
                    if (done) break;
                }
                if ((double)x > lo && (double)x < hi) d = (double)x;
            }
            for (int it = 0; it < 60; ++it) {
                double f, df;
                mac_log_newton(d, b, B1, B2, p, G, ltol, f, df);
                double dn = d * exp(-f / df);
                if (fabs(dn - d) <= 1e-11 * d) {  // converged (possibly onto a bracket end)
                    d = dn;
                    break;
                }
                if (!(dn > lo && dn < hi)) dn = 0.5 * (lo + hi);
                if (!(dn > lo && dn < hi)) break;
                if (mac_bound(dn, b, B1, B2, p, G) <= tol)
                    hi = dn;
                else
                    lo = dn;
                d = dn;
                if (hi - lo <= 1e-11 * hi) {
                    d = hi;
                    break;
                }
            }
            rc = d;
        }
    }
    return rc;
}

// Per-interaction order selection: the radius of order q of cell c, one thread per (cell,
// order) pair (the solves are long float64 sequences: one thread per cell looping over
// the orders left most of the GPU idle), into rcq[nq c + q - q_lo].
__global__ void k_mac_radius_orders(const double *__restrict__ cbmax, int64_t ncell, int p, double G, double tol,
                                    const double *__restrict__ cBn, int q_lo, double *__restrict__ rcq,
                                    float *__restrict__ rcqf)
{
    const int nq = p - q_lo + 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell * nq) return;
    const int64_t c = i / nq;
    const int q = q_lo + (int)(i - c * nq);
    const double *Bn = cBn + (int64_t)(p + 3) * c;
    const double r = mac_radius_solve(cbmax[c], Bn[q + 1], Bn[q + 2], q, G, tol);
    rcq[i] = r;
    rcqf[i] = (float)r;
}

// With per-interaction order selection (cBn != nullptr: B_n of every cell, n = 0..p+2) the
// radius of every order q_lo..p is in rcq (k_mac_radius_orders) and a cell is accepted at
// the smallest one (some order meets the tolerance).
__global__ void k_mac_radius(const double *__restrict__ ccom, const double *__restrict__ cbmax,
                             const double *__restrict__ cB1, const double *__restrict__ cB2, int64_t ncell, int p,
                             double G, double tol, double guard, const double *__restrict__ cBn, int q_lo,
                             double *__restrict__ rcq, float *__restrict__ rcqf, TCell *__restrict__ tc,
                             TCellF *__restrict__ tcf)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double b = cbmax[c];
    double rc;
    if (cBn) {
        const int nq = p - q_lo + 1;
        rc = INFINITY;
        for (int q = q_lo; q <= p; ++q) rc = fmin(rc, rcq[(int64_t)nq * c + (q - q_lo)]);
    } else {
        rc = mac_radius_solve(b, cB1[c], cB2[c], p, G, tol);
    }
    rc = fmax(rc, b + guard);
    TCell t;
    t.x = ccom[3 * c + 0];
    t.y = ccom[3 * c + 1];
    t.z = ccom[3 * c + 2];
    t.rc = rc;
    tc[c] = t;
    TCellF f;
    f.hx = (float)t.x;
    f.hy = (float)t.y;
    f.hz = (float)t.z;
    f.lx = (float)(t.x - (double)f.hx);
    f.ly = (float)(t.y - (double)f.hy);
    f.lz = (float)(t.z - (double)f.hz);
    f.rc = (float)rc;
    f.pad = 0.f;
    tcf[c] = f;
}

// MODE 0: count the entries of every group's lists (and the interaction totals);
// MODE 1: fill the CSR lists at the scanned offsets;
// MODE 2: one pass for both -- the entries go to fixed-capacity per-group slots (capm,
// capp entries), the counts and totals as in MODE 0, and the largest counts to maxc[2];
// a group whose lists do not fit sets *slot_over and keeps counting.  MODE 0 also
// records the largest counts.  Both add the P2P source-particle visits (the particles
// of every listed leaf, summed over groups) to maxc[3] and write each group's cost key.
// PER: periodic boundaries (per_L > 0), the open-boundary instantiation carrying none of
// the image loop's state.
template <int MODE, bool PER>
__global__ void __launch_bounds__(TW * 32) k_traverse(
    int64_t ngroup, const int32_t *__restrict__ gcell, const double *__restrict__ gcen,
    const double *__restrict__ gdmax, const TCell *__restrict__ tcell, const TCellF *__restrict__ tcf,
    const int32_t *__restrict__ cend,
    const int32_t *__restrict__ child8, const int32_t *__restrict__ cnchild,
    const int32_t *__restrict__ ccount, const double *__restrict__ ccom, const double *__restrict__ cbmax,
    const double *__restrict__ cB1, const double *__restrict__ cB2, int p, double G, double tol, double guard,
    const double *__restrict__ cBn, int q_lo, const double *__restrict__ rcq, const float *__restrict__ rcqf,
    double per_L, int per_ws,
    int32_t *__restrict__ scratch, int cap, unsigned *__restrict__ work, uint32_t *__restrict__ cnt_m2p,
    uint32_t *__restrict__ cnt_p2p, const int64_t *__restrict__ off_m2p, const int64_t *__restrict__ off_p2p,
    int32_t *__restrict__ l_m2p, int32_t *__restrict__ l_p2p, unsigned long long *__restrict__ stats,
    int64_t capm, int64_t capp, unsigned long long *__restrict__ maxc, unsigned *__restrict__ slot_over,
    uint64_t *__restrict__ gkey, unsigned *__restrict__ status)
{
    constexpr bool FILL = MODE == 1, SLOTS = MODE == 2;
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t *bufA = scratch + gw * 2 * (int64_t)cap;
    int32_t *bufB = bufA + cap;
    for (;;) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(work, 1u);
        const int64_t g = __shfl_sync(0xffffffffu, g0, 0);
        if (g >= ngroup) break;
        const int32_t gc = gcell[g];
        const int32_t gend = cend[gc];
        const double gx0 = gcen[3 * g + 0], gy0 = gcen[3 * g + 1], gz0 = gcen[3 * g + 2];
        const double dmax = gdmax[g];
        const float dmaxf = (float)dmax;
        int64_t om = 0, op = 0;
        if (FILL) {
            om = off_m2p[g];
            op = off_p2p[g];
        } else if (SLOTS) {
            om = g * capm;
            op = g * capp;
        }
        uint32_t nm = 0, np = 0;
        uint64_t p2p_parts = 0;
        bool overflow = false;
        // periodic boundaries: the central tree and its images within per_ws, the image's
        // sources being the tree shifted by s, i.e. the group centre moved by -s; every
        // entry is tagged with its image
        const bool per = PER && per_L > 0.0;
        const int pw = 2 * per_ws + 1;
        const int nimg = per ? pw * pw * pw : 1;
        for (int img = 0; img < nimg && !overflow; ++img) {
        const bool central = 2 * img == nimg - 1;
        const uint32_t tag = per ? (uint32_t)img << HOT_IMG_SHIFT : 0u;
        const double gx = per ? gx0 - (double)(img / (pw * pw) - per_ws) * per_L : gx0;
        const double gy = per ? gy0 - (double)((img / pw) % pw - per_ws) * per_L : gy0;
        const double gz = per ? gz0 - (double)(img % pw - per_ws) * per_L : gz0;
        const float ghx = (float)gx, ghy = (float)gy, ghz = (float)gz;
        const float glx = (float)(gx - (double)ghx), gly = (float)(gy - (double)ghy), glz = (float)(gz - (double)ghz);
        int32_t *A = bufA, *B = bufB;
        if (lane == 0) A[0] = 0;
        __syncwarp();
        int na = 1;
        while (na > 0 && !overflow) {
            int nb = 0;
            for (int base = 0; base < na; base += 32) {
                const int i = base + (int)lane;
                const int32_t c = i < na ? A[i] : -1;
                int32_t ent = c;  // the M2P entry: the cell, with its order under order selection
                int kind = 0;  // 1 M2P, 2 P2P, 3 open
                if (c >= 0) {
                    const bool leaf = cnchild[c] == 0;
                    // pre-order: c is the group's cell or an ancestor iff gc lies in c's subtree,
                    // inside the group's cell iff it lies in gc's subtree (its particles are sinks
                    // of the group: d <= 0, never accepted, whatever the rounding of d); in the
                    // central tree only, in an image every cell is a source
                    const bool anc = central && ((c <= gc && gc < cend[c]) || (gc < c && c < gend));
                    if (anc) {
                        kind = leaf ? 2 : 3;
                    } else {
                        // float32 pre-test on hi/lo offsets (relative error below 1e-6): decisions
                        // outside a 1e-5 band are those of the float64 test; inside it, that test
                        const TCellF f = tcf[c];
                        const float ox = (f.hx - ghx) + (f.lx - glx);
                        const float oy = (f.hy - ghy) + (f.ly - gly);
                        const float oz = (f.hz - ghz) + (f.lz - glz);
                        const float d2f = ox * ox + oy * oy + oz * oz;
                        const float thf = dmaxf + f.rc;
                        const float th2f = thf * thf;
                        bool acc;
                        if (d2f > th2f * 1.00001f) {
                            acc = true;
                        } else if (d2f < th2f * 0.99999f || !(f.rc < INFINITY)) {
                            acc = false;
                        } else {
                        const TCell t = tcell[c];
                        const double dx = t.x - gx, dy = t.y - gy, dz = t.z - gz;
                        const double dist2 = dx * dx + dy * dy + dz * dz;
                        const double thr = dmax + t.rc;
                        const double thr2 = thr * thr;
                        if (dist2 > thr2 * (1.0 + 1e-9)) {
                            acc = true;
                        } else if (dist2 < thr2 * (1.0 - 1e-9) || !(t.rc < INFINITY)) {
                            acc = false;
                        } else {
                            // within 1e-9 of the threshold: the acceptance test as stated
                            const double ex = __dsub_rn(t.x, gx), ey = __dsub_rn(t.y, gy), ez = __dsub_rn(t.z, gz);
                            const double dist = __dsqrt_rn(
                                __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
                            const double d = __dsub_rn(dist, dmax);
                            const double b = cbmax[c];
                            if (cBn) {
                                // some order of the range meets the tolerance
                                const double *Bn = cBn + (int64_t)(p + 3) * c;
                                acc = false;
                                if (d > b && d >= __dadd_rn(b, guard))
                                    for (int q = q_lo; q <= p && !acc; ++q)
                                        acc = mac_bound(d, b, Bn[q + 1], Bn[q + 2], q, G) <= tol;
                            } else {
                                acc = d > b && d >= __dadd_rn(b, guard) && mac_bound(d, b, cB1[c], cB2[c], p, G) <= tol;
                            }
                        }
                        }
                        kind = acc ? 1 : (leaf ? 2 : 3);
                        int qf = -1;  // the order when the float32 test decides it
                        if (cBn && acc) {
                            // float32 first, on the squared distances as for the acceptance: the
                            // lowest order whose radius the distance clearly reaches, every lower one
                            // clearly not; a radius within 1e-5 leaves it to the float64 choice
                            const int nq = p - q_lo + 1;
                            for (int q = q_lo; q <= p; ++q) {
                                const float rq = rcqf[(int64_t)nq * c + (q - q_lo)];
                                if (!(rq < INFINITY)) continue;
                                const float th = dmaxf + rq;
                                const float t2 = th * th;
                                if (d2f > t2 * 1.00001f) {
                                    qf = q;
                                    break;
                                }
                                if (!(d2f < t2 * 0.99999f)) break;
                            }
                        }
                        if (qf >= 0) {
                            ent = (int32_t)((uint32_t)c | ((uint32_t)qf << HOT_ORDER_SHIFT));
                        } else if (cBn && acc) {
                            // the lowest order whose radius the distance reaches; within 1e-9 of a
                            // radius, that order's bound as stated (d rounded as the oracle does)
                            const TCell t = tcell[c];
                            const double ex = __dsub_rn(t.x, gx), ey = __dsub_rn(t.y, gy), ez = __dsub_rn(t.z, gz);
                            const double dist = __dsqrt_rn(
                                __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
                            const double d = __dsub_rn(dist, dmax);
                            const double b = cbmax[c];
                            const double *Bn = cBn + (int64_t)(p + 3) * c;
                            const int nq = p - q_lo + 1;
                            int qa = p;
                            for (int q = q_lo; q <= p; ++q) {
                                const double rq = rcq[(int64_t)nq * c + (q - q_lo)];
                                bool ok;
                                if (!(rq < INFINITY))
                                    ok = false;
                                else if (d > rq * (1.0 + 1e-9))
                                    ok = true;
                                else if (d < rq * (1.0 - 1e-9))
                                    ok = false;
                                else
                                    ok = d > b && mac_bound(d, b, Bn[q + 1], Bn[q + 2], q, G) <= tol;
                                if (ok) {
                                    qa = q;
                                    break;
                                }
                            }
                            ent = (int32_t)((uint32_t)c | ((uint32_t)qa << HOT_ORDER_SHIFT));
                        }
                    }
                }
                const unsigned mm = __ballot_sync(0xffffffffu, kind == 1);
                const unsigned pm = __ballot_sync(0xffffffffu, kind == 2);
                if (FILL) {
                    if (kind == 1) l_m2p[om + nm + __popc(mm & lt)] = (int32_t)((uint32_t)ent | tag);
                    if (kind == 2) l_p2p[op + np + __popc(pm & lt)] = (int32_t)((uint32_t)c | tag);
                } else {
                    if (SLOTS) {
                        const int64_t im = nm + __popc(mm & lt), ip = np + __popc(pm & lt);
                        if (kind == 1 && im < capm) l_m2p[om + im] = (int32_t)((uint32_t)ent | tag);
                        if (kind == 2 && ip < capp) l_p2p[op + ip] = (int32_t)((uint32_t)c | tag);
                    }
                    if (kind == 2) p2p_parts += (uint64_t)ccount[c];
                }
                nm += __popc(mm);
                np += __popc(pm);
                const int nch = kind == 3 ? cnchild[c] : 0;
                const int incl = warp_incl_scan(nch);
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                if (nb + tot > cap) {
                    overflow = true;
                    break;
                }
                if (kind == 3) {
                    int k = nb + incl - nch;
#pragma unroll
                    for (int o = 0; o < 8; ++o) {
                        const int32_t ch = child8[8 * (int64_t)c + o];
                        if (ch >= 0) B[k++] = ch;
                    }
                }
                nb += tot;
            }
            __syncwarp();
            int32_t *t = A;
            A = B;
            B = t;
            na = nb;
        }
        }  // images
        if (overflow) {
            if (lane == 0) hot_flag(status, HOT_ST_FRONTIER);
            nm = np = 0;
        }
        if (!FILL) {
            p2p_parts = warp_sum(p2p_parts);
            if (lane == 0) {
                cnt_m2p[g] = nm;
                cnt_p2p[g] = np;
                const uint64_t ns = (uint64_t)ccount[gc];
                atomicAdd(&stats[0], (unsigned long long)(ns * nm));
                atomicAdd(&stats[1], (unsigned long long)(ns * p2p_parts));
                atomicMax(&maxc[0], (unsigned long long)nm);
                atomicMax(&maxc[1], (unsigned long long)np);
                atomicAdd(&maxc[3], (unsigned long long)p2p_parts);  // source-particle visits
                // interaction cost of one 32-sink slice of the group (one M2P evaluation ~ 10
                // P2P source visits), as an ascending sort key for largest-first processing
                const uint64_t cost = 10ull * nm + p2p_parts;
                gkey[g] = cost_key16(cost);
                if (SLOTS && ((int64_t)nm > capm || (int64_t)np > capp)) atomicOr(slot_over, 1u);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Background subtraction (Sec. "Background Subtraction").  The acceptance estimate of a
// contrast expansion about a cube's centre (half-diagonal b, Q_n the size of its order-n
// multipole):
//   E(d) = G / (1 - b/d)^2 [(p+2) Q_{p+1} / d^{p+3} + (p+3) Q_{p+2} / d^{p+4}],  d > b,
// strictly decreasing on (b, inf), so it too is pre-solved per cube into a radius.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double bg_bound(double d, double b, double Q1, double Q2, int p, double G)
{
    const double q = __dsub_rn(1.0, __ddiv_rn(b, d));
    double dp = d;  // d^{p+3} by repeated multiplication
    for (int i = 0; i < p + 2; ++i) dp = __dmul_rn(dp, d);
    const double t1 = __ddiv_rn(__dmul_rn((double)(p + 2), Q1), dp);
    const double t2 = __ddiv_rn(__dmul_rn((double)(p + 3), Q2), __dmul_rn(dp, d));
    return __dmul_rn(__ddiv_rn(G, __dmul_rn(q, q)), __dadd_rn(t1, t2));
}

// The radius of E(d) = tol: a bracket around the larger of the two terms' far-field
// radii, then Newton steps in ln d with bisection as the safeguard (as for the plain
// bound); b when E vanishes (a contrast with no omitted multipole: accepted as soon as
// d > b).
__device__ double bg_radius_solve(double b, double Q1, double Q2, int p, double G, double tol)
{
    if (!(Q1 > 0.0 || Q2 > 0.0)) return b;
    double d0 = fmax(pow(G * (p + 2) * Q1 / tol, 1.0 / (p + 3)), pow(G * (p + 3) * Q2 / tol, 1.0 / (p + 4)));
    if (!(d0 > 1.0001 * b)) d0 = 2.0 * b;
    double lo = b, hi = d0;
    int k = 0;
    if (bg_bound(d0, b, Q1, Q2, p, G) <= tol) {
        while (k < 1100) {
            const double t = 0.5 * hi;
            if (!(t > b) || !(bg_bound(t, b, Q1, Q2, p, G) <= tol)) {
                lo = t > b ? t : b;
                break;
            }
            hi = t;
            ++k;
        }
    } else {
        lo = d0;
        hi = 2.0 * d0;
        while (!(bg_bound(hi, b, Q1, Q2, p, G) <= tol) && k < 1100) {
            lo = hi;
            hi *= 2.0;
            ++k;
        }
    }
    if (k >= 1100) return INFINITY;
    const double ltol = log(tol);
    double d = hi;
    for (int it = 0; it < 80; ++it) {
        // ln E and its derivative in ln d
        const double a1 = (p + 2) * Q1 * pow(d, -(double)(p + 3)), a2 = (p + 3) * Q2 * pow(d, -(double)(p + 4));
        const double f = log(G) - 2.0 * log(1.0 - b / d) + log(a1 + a2) - ltol;
        const double df = -2.0 * b / (d - b) - ((p + 3) * a1 + (p + 4) * a2) / (a1 + a2);
        double dn = d * exp(-f / df);
        if (fabs(dn - d) <= 1e-13 * d) {
            d = dn;
            break;
        }
        if (!(dn > lo && dn < hi)) dn = 0.5 * (lo + hi);
        if (!(dn > lo && dn < hi)) break;
        if (bg_bound(dn, b, Q1, Q2, p, G) <= tol)
            hi = dn;
        else
            lo = dn;
        d = dn;
        if (hi - lo <= 1e-13 * hi) {
            d = hi;
            break;
        }
    }
    return d;
}

__global__ void k_bg_radius(const double *__restrict__ cen, const double *__restrict__ half,
                            const double *__restrict__ bq, int64_t ncube, int p, double G, double tol,
                            TCell *__restrict__ tc, TCellF *__restrict__ tcf)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ncube) return;
    const double b = 0.5 * sqrt(3.0) * (2.0 * half[q]);
    TCell t;
    t.x = cen[3 * q + 0];
    t.y = cen[3 * q + 1];
    t.z = cen[3 * q + 2];
    t.rc = bg_radius_solve(b, bq[2 * q], bq[2 * q + 1], p, G, tol);
    tc[q] = t;
    TCellF f;
    f.hx = (float)t.x;
    f.hy = (float)t.y;
    f.hz = (float)t.z;
    f.lx = (float)(t.x - (double)f.hx);
    f.ly = (float)(t.y - (double)f.hy);
    f.lz = (float)(t.z - (double)f.hz);
    f.rc = (float)t.rc;
    f.pad = 0.f;
    tcf[q] = f;
}

// The float32 pre-test of a radius test on hi/lo offsets (relative error below 1e-6, as in
// k_traverse): 1 accept, 0 reject, -1 within 1e-5 of the threshold (take the float64 test).
struct GroupF {
    float hx, hy, hz, lx, ly, lz, dmax;
};
__device__ __forceinline__ int pretest(const TCellF &f, const GroupF &g)
{
    const float ox = (f.hx - g.hx) + (f.lx - g.lx);
    const float oy = (f.hy - g.hy) + (f.ly - g.ly);
    const float oz = (f.hz - g.hz) + (f.lz - g.lz);
    const float d2f = ox * ox + oy * oy + oz * oz;
    const float thf = g.dmax + f.rc;
    const float th2f = thf * thf;
    if (!(f.rc < INFINITY)) return 0;
    if (d2f > th2f * 1.00001f) return 1;
    if (d2f < th2f * 0.99999f) return 0;
    return -1;
}

// Acceptance of a contrast expansion (cube q) for a group at (gx, gy, gz), Delta_max dmax:
// d = |c - g| - dmax >= r_c, decided as stated within 1e-9 of the threshold.
__device__ __forceinline__ bool bg_accept(const TCell &t, double half, const double *__restrict__ bq, int64_t q,
                                          double gx, double gy, double gz, double dmax, int p, double G, double tol)
{
    if (!(t.rc < INFINITY)) return false;
    const double dx = t.x - gx, dy = t.y - gy, dz = t.z - gz;
    const double dist2 = dx * dx + dy * dy + dz * dz;
    const double thr = dmax + t.rc;
    const double thr2 = thr * thr;
    if (dist2 > thr2 * (1.0 + 1e-9)) return true;
    if (dist2 < thr2 * (1.0 - 1e-9)) return false;
    const double ex = __dsub_rn(t.x, gx), ey = __dsub_rn(t.y, gy), ez = __dsub_rn(t.z, gz);
    const double dist = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
    const double d = __dsub_rn(dist, dmax);
    const double b = 0.5 * sqrt(3.0) * (2.0 * half);
    return d > b && bg_bound(d, b, bq[2 * q], bq[2 * q + 1], p, G) <= tol;
}

// The plain acceptance test of a cell's matter expansion (as in k_traverse, float64 only).
__device__ __forceinline__ bool plain_accept(const TCell &t, double b, double B1, double B2, double gx, double gy,
                                             double gz, double dmax, int p, double G, double tol)
{
    if (!(t.rc < INFINITY)) return false;
    const double dx = t.x - gx, dy = t.y - gy, dz = t.z - gz;
    const double dist2 = dx * dx + dy * dy + dz * dz;
    const double thr = dmax + t.rc;
    const double thr2 = thr * thr;
    if (dist2 > thr2 * (1.0 + 1e-9)) return true;
    if (dist2 < thr2 * (1.0 - 1e-9)) return false;
    const double ex = __dsub_rn(t.x, gx), ey = __dsub_rn(t.y, gy), ez = __dsub_rn(t.z, gz);
    const double dist = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
    const double d = __dsub_rn(dist, dmax);
    return d > b && mac_bound(d, b, B1, B2, p, G) <= tol;
}

// Group-wise traversal under background subtraction, one warp per group, breadth-first as
// k_traverse.  S, the group's surrounding cube, is its cell's ancestor `up` levels up.
//   * the group's cell and its ancestors are opened (a leaf among them goes to P2P);
//   * a cell inside S: the plain method (matter expansion about the centre of mass, the
//     plain test; else P2P for a leaf, else opened);
//   * a cell outside S: its contrast expansion if accepted (M2P entry ncell + c); else a
//     leaf goes to P2P and its cube's background to the cube list (entry c); else opened;
//   * every opened cell outside S (ancestors above S included): each empty octant e is a
//     contrast expansion if accepted (M2P entry 2 ncell + e), else an analytic cube (cube
//     list entry ncell + e).
// MODE 0 counts (and writes S, the totals and the cost keys), MODE 1 fills at the offsets.
template <int MODE>
__global__ void __launch_bounds__(TW * 32) k_traverse_bg(
    int64_t ngroup, int64_t ncell, const int32_t *__restrict__ gcell, const double *__restrict__ gcen,
    const double *__restrict__ gdmax, const int32_t *__restrict__ cparent, const TCell *__restrict__ tcell,
    const TCellF *__restrict__ tcf, const TCell *__restrict__ tbg, const TCellF *__restrict__ tbgf,
    const double *__restrict__ bhalf, const double *__restrict__ bq,
    const uint32_t *__restrict__ eoff, const int32_t *__restrict__ cend, const int32_t *__restrict__ child8,
    const int32_t *__restrict__ cnchild, const int32_t *__restrict__ ccount, const double *__restrict__ cbmax,
    const double *__restrict__ cB1, const double *__restrict__ cB2, int p, double G, double tol, int up,
    int32_t *__restrict__ scratch, int cap, unsigned *__restrict__ work, uint32_t *__restrict__ cnt_m2p,
    uint32_t *__restrict__ cnt_p2p, uint32_t *__restrict__ cnt_box, const int64_t *__restrict__ off_m2p,
    const int64_t *__restrict__ off_p2p, const int64_t *__restrict__ off_box, int32_t *__restrict__ l_m2p,
    int32_t *__restrict__ l_p2p, int32_t *__restrict__ l_box, int32_t *__restrict__ gS,
    unsigned long long *__restrict__ stats, uint64_t *__restrict__ gkey, unsigned *__restrict__ status)
{
    constexpr bool FILL = MODE == 1;
    const unsigned lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t *A = scratch + gw * 2 * (int64_t)cap;
    int32_t *B = A + cap;
    for (;;) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(work, 1u);
        const int64_t g = __shfl_sync(0xffffffffu, g0, 0);
        if (g >= ngroup) break;
        const int32_t gc = gcell[g];
        const int32_t gend = cend[gc];
        const double gx = gcen[3 * g + 0], gy = gcen[3 * g + 1], gz = gcen[3 * g + 2];
        const double dmax = gdmax[g];
        GroupF gf;
        gf.hx = (float)gx;
        gf.hy = (float)gy;
        gf.hz = (float)gz;
        gf.lx = (float)(gx - (double)gf.hx);
        gf.ly = (float)(gy - (double)gf.hy);
        gf.lz = (float)(gz - (double)gf.hz);
        gf.dmax = (float)dmax;
        auto plain_ok = [&](int32_t c) {
            const int r = pretest(tcf[c], gf);
            return r >= 0 ? r == 1 : plain_accept(tcell[c], cbmax[c], cB1[c], cB2[c], gx, gy, gz, dmax, p, G, tol);
        };
        auto bg_ok = [&](int64_t q) {
            const int r = pretest(tbgf[q], gf);
            return r >= 0 ? r == 1 : bg_accept(tbg[q], bhalf[q], bq, q, gx, gy, gz, dmax, p, G, tol);
        };
        int32_t S = gc;
        for (int k = 0; k < up && S > 0; ++k) S = cparent[S];
        const int32_t Send = cend[S];
        const int64_t om = FILL ? off_m2p[g] : 0, op = FILL ? off_p2p[g] : 0, ob = FILL ? off_box[g] : 0;
        uint32_t nm = 0, np = 0, nb = 0, ncon = 0, nemp = 0;
        uint64_t parts = 0;
        bool overflow = false;
        if (lane == 0) A[0] = 0;
        __syncwarp();
        int na = 1;
        while (na > 0 && !overflow) {
            int nbf = 0;
            for (int base = 0; base < na; base += 32) {
                const int i = base + (int)lane;
                const int32_t c = i < na ? A[i] : -1;
                int32_t em = -1, eb = -1;  // this cell's M2P and cube entries
                bool pp = false, open = false, empt = false;
                if (c >= 0) {
                    const bool leaf = cnchild[c] == 0;
                    const bool anc = c <= gc && gc < cend[c];
                    const bool inS = S <= c && c < Send;
                    if (anc) {
                        pp = leaf;
                        open = !leaf;
                        empt = !leaf && !inS;
                    } else if (gc < c && c < gend) {
                        // inside the group's cell: d <= 0, never expanded (inside S)
                        pp = leaf;
                        open = !leaf;
                    } else if (inS) {
                        if (plain_ok(c))
                            em = c;
                        else if (leaf)
                            pp = true;
                        else
                            open = true;
                    } else {
                        if (bg_ok(c)) {
                            em = (int32_t)(ncell + c);
                        } else if (leaf) {
                            pp = true;
                            eb = c;
                        } else {
                            open = true;
                            empt = true;
                        }
                    }
                }
                // empty octants of an opened cell outside S: accepted ones (bit set in am)
                // or analytic cubes
                unsigned am = 0, ab = 0;
                uint32_t e0 = 0;
                if (empt) {
                    e0 = eoff[c];
                    uint32_t e = e0;
                    for (int o = 0; o < 8; ++o) {
                        if (child8[8 * (int64_t)c + o] >= 0) continue;
                        const int64_t qb = ncell + e;
                        if (bg_ok(qb))
                            am |= 1u << (e - e0);
                        else
                            ab |= 1u << (e - e0);
                        ++e;
                    }
                }
                const uint32_t lm = (em >= 0 ? 1u : 0u) + (uint32_t)__popc(am);
                const uint32_t lp = pp ? 1u : 0u;
                const uint32_t lb = (eb >= 0 ? 1u : 0u) + (uint32_t)__popc(ab);
                const uint32_t im = warp_incl_scan(lm), ip = warp_incl_scan(lp), ib = warp_incl_scan(lb);
                if (FILL) {
                    int64_t km = om + nm + im - lm, kb = ob + nb + ib - lb;
                    if (em >= 0) l_m2p[km++] = em;
                    for (unsigned bm = am; bm; bm &= bm - 1u) l_m2p[km++] = (int32_t)(2 * ncell + e0 + __ffs(bm) - 1);
                    if (pp) l_p2p[op + np + ip - lp] = c;
                    if (eb >= 0) l_box[kb++] = eb;
                    for (unsigned bb = ab; bb; bb &= bb - 1u) l_box[kb++] = (int32_t)(ncell + e0 + __ffs(bb) - 1);
                } else if (pp) {
                    parts += (uint64_t)ccount[c];
                }
                ncon += __popc(__ballot_sync(0xffffffffu, em >= ncell));
                nemp += warp_sum((uint32_t)__popc(am));
                nm += __shfl_sync(0xffffffffu, im, 31);
                np += __shfl_sync(0xffffffffu, ip, 31);
                nb += __shfl_sync(0xffffffffu, ib, 31);
                const int nch = open ? cnchild[c] : 0;
                const int incl = warp_incl_scan(nch);
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                if (nbf + tot > cap) {
                    overflow = true;
                    break;
                }
                if (open) {
                    int k = nbf + incl - nch;
#pragma unroll
                    for (int o = 0; o < 8; ++o) {
                        const int32_t ch = child8[8 * (int64_t)c + o];
                        if (ch >= 0) B[k++] = ch;
                    }
                }
                nbf += tot;
            }
            __syncwarp();
            int32_t *t = A;
            A = B;
            B = t;
            na = nbf;
        }
        if (overflow) {
            if (lane == 0) hot_flag(status, HOT_ST_FRONTIER);
            nm = np = nb = ncon = nemp = 0;
        }
        if (!FILL) {
            parts = warp_sum(parts);
            if (lane == 0) {
                cnt_m2p[g] = nm;
                cnt_p2p[g] = np;
                cnt_box[g] = nb;
                gS[g] = S;
                const uint64_t ns = (uint64_t)ccount[gc];
                atomicAdd(&stats[0], (unsigned long long)(ns * nm));
                atomicAdd(&stats[1], (unsigned long long)(ns * parts));
                atomicAdd(&stats[2], (unsigned long long)(ns * (nb + 1)));
                atomicAdd(&stats[3], (unsigned long long)(ns * ncon));
                atomicAdd(&stats[4], (unsigned long long)(ns * nemp));
                atomicAdd(&stats[5], (unsigned long long)parts);
                const uint64_t cost = 10ull * nm + parts;
                gkey[g] = cost_key16(cost);
            }
        }
        __syncwarp();
    }
}

__global__ void k_iota(uint32_t *__restrict__ v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

// Number of 32-sink slices of every group, in the sorted group order.
__global__ void k_slice_count(const uint32_t *__restrict__ gorder, const int32_t *__restrict__ gcell,
                              const int32_t *__restrict__ ccount, int64_t ng, uint32_t *__restrict__ cnt)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < ng) cnt[j] = (uint32_t)((ccount[gcell[gorder[j]]] + 31) / 32);
}

// Work items: the slices of every group, groups in the sorted order, each item the group
// index (high word) and its first sink within the group (low word).
__global__ void k_slice_fill(const uint32_t *__restrict__ gorder, const uint32_t *__restrict__ off, int64_t ng,
                             uint64_t *__restrict__ items)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ng) return;
    const uint64_t g = gorder[j];
    for (uint32_t q = off[j]; q < off[j + 1]; ++q) items[q] = (g << 32) | (uint64_t)((q - off[j]) * 32u);
}

// Copy every group's slot entries to its CSR range (one warp per group, in order).
__global__ void k_compact_lists(int64_t ngroup, int64_t capm, int64_t capp, const int32_t *__restrict__ sm,
                                const int32_t *__restrict__ sp, const int64_t *__restrict__ off_m2p,
                                const int64_t *__restrict__ off_p2p, int32_t *__restrict__ l_m2p,
                                int32_t *__restrict__ l_p2p)
{
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= ngroup) return;
    const unsigned lane = lane_id();
    const int64_t m0 = off_m2p[g], nm = off_m2p[g + 1] - m0;
    const int64_t p0 = off_p2p[g], np = off_p2p[g + 1] - p0;
    for (int64_t k = lane; k < nm; k += 32) l_m2p[m0 + k] = sm[g * capm + k];
    for (int64_t k = lane; k < np; k += 32) l_p2p[p0 + k] = sp[g * capp + k];
}

}  // namespace

namespace {

// Work order of the interactions: groups by descending slice cost (stable, so ties keep
// index order), each expanded into its 32-sink slices, so that no single large group is
// one warp's work.
int work_items(hot_ctx *c)
{
    cudaStream_t s = c->st;
    const int64_t ng = c->ngroup;
    HOT_COUNT_LAUNCH();
    k_iota<<<hot_blocks(ng, 256), 256, 0, s>>>(c->gorder.p, ng);
    int rs = hot_sort_pairs(c, c->gkey.p, c->gorder.p, c->gkey2.p, c->gorder2.p, ng, 16);
    if (rs) return rs;
    HOT_CK(c->slice_cnt.ensure(ng + 1, s));
    HOT_CK(c->slice_off.ensure(ng + 1, s));
    HOT_CK(c->items.ensure(ng + c->N / 32 + 1, s));
    HOT_COUNT_LAUNCH();
    k_slice_count<<<hot_blocks(ng, 256), 256, 0, s>>>(c->gorder.p, c->gcell.p, c->ccount.p, ng, c->slice_cnt.p);
    rs = hot_scan_u32_to_u32(c->slice_cnt.p, c->slice_off.p, ng, c->scan_tmp.p, s);
    if (rs) return rs;
    HOT_COUNT_LAUNCH();
    k_slice_fill<<<hot_blocks(ng, 256), 256, 0, s>>>(c->gorder.p, c->slice_off.p, ng, c->items.p);
    return HOT_OK;
}

// Lists under background subtraction: count, scan, fill (three lists per group), then the
// work items as for the plain method.
int traverse_bg(hot_ctx *c, double tol)
{
    cudaStream_t s = c->st;
    const int64_t ng = c->ngroup, nc = c->ncell, ncube = nc + c->n_empty;
    HOT_CK(c->cnt_m2p.ensure(ng + 1, s));
    HOT_CK(c->cnt_p2p.ensure(ng + 1, s));
    HOT_CK(c->cnt_box.ensure(ng + 1, s));
    HOT_CK(c->off_m2p.ensure(ng + 1, s));
    HOT_CK(c->off_p2p.ensure(ng + 1, s));
    HOT_CK(c->off_box.ensure(ng + 1, s));
    HOT_CK(c->bg_gS.ensure(ng + 1, s));
    HOT_CK(c->scan_tmp.ensure(hot_scan_tmp_elems(ng + c->ncell + c->N + 64), s));
    HOT_CK(c->tcell.ensure(nc, s));
    HOT_CK(c->tcellf.ensure(nc, s));
    HOT_CK(c->bg_tc.ensure(ncube, s));
    HOT_CK(c->bg_tcf.ensure(ncube, s));
    HOT_CK(c->gkey.ensure(ng + 1, s));
    HOT_CK(c->gkey2.ensure(ng + 1, s));
    HOT_CK(c->gorder.ensure(ng + 1, s));
    HOT_CK(c->gorder2.ensure(ng + 1, s));
    const int blocks = c->nsm * 4;
    const int64_t nwarps = (int64_t)blocks * TW;
    unsigned *work = (unsigned *)(c->sizes.p + 50);
    unsigned long long *stats = (unsigned long long *)(c->sizes.p + 52);  // 6 counters, 52..57
    HOT_COUNT_LAUNCH();
    k_mac_radius<<<hot_blocks(nc, 128), 128, 0, s>>>(c->ccom.p, c->cbmax.p, c->cB1.p, c->cB2.p, nc, c->p_mom,
                                                      c->prm.G, tol, 0.0, nullptr, c->q_lo, nullptr, nullptr,
                                                      c->tcell.p, c->tcellf.p);
    HOT_COUNT_LAUNCH();
    k_bg_radius<<<hot_blocks(ncube, 128), 128, 0, s>>>(c->bg_cen.p, c->bg_half.p, c->bg_q.p, ncube, c->p_mom,
                                                       c->prm.G, tol, c->bg_tc.p, c->bg_tcf.p);
    int64_t host[9];
    for (int attempt = 0;; ++attempt) {
        HOT_CK(c->trav_scratch.ensure((size_t)nwarps * 2 * c->trav_cap, s));
        HOT_CK(cudaMemsetAsync(c->sizes.p + 50, 0, 8 * sizeof(int64_t), s));
        HOT_COUNT_LAUNCH();
        k_traverse_bg<0><<<blocks, TW * 32, 0, s>>>(
            ng, nc, c->gcell.p, c->gcen.p, c->gdmax.p, c->cparent.p, c->tcell.p, c->tcellf.p, c->bg_tc.p, c->bg_tcf.p,
            c->bg_half.p, c->bg_q.p,
            c->bg_eoff.p, c->cend.p, c->child8.p, c->cnchild.p, c->ccount.p, c->cbmax.p, c->cB1.p, c->cB2.p,
            c->p_mom, c->prm.G, tol, c->prm.bg_up, c->trav_scratch.p, c->trav_cap, work, c->cnt_m2p.p,
            c->cnt_p2p.p, c->cnt_box.p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, c->bg_gS.p, stats,
            c->gkey.p, c->d_status);
        int r = hot_scan_u32_to_i64(c->cnt_m2p.p, c->off_m2p.p, ng, c->scan_tmp.p, s);
        if (r) return r;
        r = hot_scan_u32_to_i64(c->cnt_p2p.p, c->off_p2p.p, ng, c->scan_tmp.p, s);
        if (r) return r;
        r = hot_scan_u32_to_i64(c->cnt_box.p, c->off_box.p, ng, c->scan_tmp.p, s);
        if (r) return r;
        HOT_CK(cudaMemcpyAsync(host + 0, c->off_m2p.p + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HOT_CK(cudaMemcpyAsync(host + 1, c->off_p2p.p + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HOT_CK(cudaMemcpyAsync(host + 2, c->off_box.p + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HOT_CK(cudaMemcpyAsync(host + 3, stats, 6 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HOT_CK(cudaStreamSynchronize(s));
        unsigned st = 0;
        HOT_CK(cudaMemcpy(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
        if (st & HOT_ST_FRONTIER) {
            HOT_CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s));
            if (attempt >= 3) return HOT_EOVERFLOW;
            c->trav_cap *= 4;
            continue;
        }
        int e = hot_sync_status(c);
        if (e) return e;
        break;
    }
    c->n_m2p = host[0];
    c->n_p2p = host[1];
    c->n_box = host[2];
    c->n_m2p_int = host[3];
    c->n_pairs = host[4];
    c->n_box_eval = host[5];
    c->n_m2p_con = host[6];
    c->n_m2p_emp = host[7];
    c->n_p2p_src = host[8];
    HOT_CK(c->l_m2p.ensure(c->n_m2p + 1, s));
    HOT_CK(c->l_p2p.ensure(c->n_p2p + 1, s));
    HOT_CK(c->l_box.ensure(c->n_box + 1, s));
    HOT_CK(cudaMemsetAsync(work, 0, sizeof(int64_t), s));
    HOT_COUNT_LAUNCH();
    k_traverse_bg<1><<<blocks, TW * 32, 0, s>>>(
        ng, nc, c->gcell.p, c->gcen.p, c->gdmax.p, c->cparent.p, c->tcell.p, c->tcellf.p, c->bg_tc.p, c->bg_tcf.p,
            c->bg_half.p, c->bg_q.p,
        c->bg_eoff.p, c->cend.p, c->child8.p, c->cnchild.p, c->ccount.p, c->cbmax.p, c->cB1.p, c->cB2.p, c->p_mom,
        c->prm.G, tol, c->prm.bg_up, c->trav_scratch.p, c->trav_cap, work, nullptr, nullptr, nullptr, c->off_m2p.p,
        c->off_p2p.p, c->off_box.p, c->l_m2p.p, c->l_p2p.p, c->l_box.p, nullptr, nullptr, nullptr, c->d_status);
    return work_items(c);
}

}  // namespace

int hot_impl_traverse(hot_ctx *c, double tol)
{
    cudaStream_t s = c->st;
    const int64_t ng = c->ngroup;
    hot_tic(c, 3);
    if (c->prm.background) {
        const int r = traverse_bg(c, tol);
        if (r) return r;
        hot_toc(c, 3);
        if (cudaGetLastError() != cudaSuccess) return HOT_ECUDA;
        c->tol_lists = tol;
        c->stage = 3;
        return HOT_OK;
    }
    HOT_CK(c->cnt_m2p.ensure(ng + 1, s));
    HOT_CK(c->cnt_p2p.ensure(ng + 1, s));
    HOT_CK(c->off_m2p.ensure(ng + 1, s));
    HOT_CK(c->off_p2p.ensure(ng + 1, s));
    HOT_CK(c->scan_tmp.ensure(hot_scan_tmp_elems(ng + c->ncell + c->N + 64), s));
    const int blocks = c->nsm * 4;
    const int64_t nwarps = (int64_t)blocks * TW;
    unsigned *work = (unsigned *)(c->sizes.p + 50);
    unsigned long long *stats = (unsigned long long *)(c->sizes.p + 52);
    unsigned long long *maxc = (unsigned long long *)(c->sizes.p + 58);
    unsigned *slot_over = (unsigned *)(c->sizes.p + 60);
    HOT_CK(c->tcell.ensure(c->ncell, s));
    HOT_CK(c->tcellf.ensure(c->ncell, s));
    HOT_CK(c->gkey.ensure(ng + 1, s));
    HOT_CK(c->gkey2.ensure(ng + 1, s));
    HOT_CK(c->gorder.ensure(ng + 1, s));
    HOT_CK(c->gorder2.ensure(ng + 1, s));
    // acceptance guard of the compact kernels (K1, spline): no source of an accepted cell
    // within eps of a sink
    const double guard = c->prm.softening != HOT_SOFT_PLUMMER ? c->prm.eps : 0.0;
    // per-interaction order selection: radii of every order, orders in the M2P entries
    const double *cBn = c->varq ? c->cBn.p : nullptr;
    // periodic boundaries: images of the tree, tagged in the entries
    const double per_L = c->prm.box > 0.0 ? c->prm.box : 0.0;
    if (per_L > 0.0 && c->ncell > (int64_t)HOT_IMG_CELL_MASK) return HOT_EINVAL;
    if (c->varq) {
        if (c->ncell > (int64_t)HOT_CELL_MASK) return HOT_EINVAL;
        HOT_CK(c->rcq.ensure((size_t)(c->p_mom - c->q_lo + 1) * c->ncell, s));
        HOT_CK(c->rcqf.ensure((size_t)(c->p_mom - c->q_lo + 1) * c->ncell, s));
    }
    if (cBn) {
        const int64_t nrq = (int64_t)(c->p_mom - c->q_lo + 1) * c->ncell;
        HOT_COUNT_LAUNCH();
        k_mac_radius_orders<<<hot_blocks(nrq, 128), 128, 0, s>>>(c->cbmax.p, c->ncell, c->p_mom, c->prm.G, tol, cBn,
                                                                 c->q_lo, c->rcq.p, c->rcqf.p);
    }
    HOT_COUNT_LAUNCH();
    k_mac_radius<<<hot_blocks(c->ncell, 128), 128, 0, s>>>(c->ccom.p, c->cbmax.p, c->cB1.p, c->cB2.p, c->ncell,
                                                            c->p_mom, c->prm.G, tol, guard, cBn, c->q_lo, c->rcq.p,
                                                            c->rcqf.p, c->tcell.p, c->tcellf.p);
    // One pass into per-group slots when their capacities (the largest counts of the
    // previous traversal plus headroom) fit the budget; otherwise count, scan, fill.
    const int64_t capm = c->slot_capm, capp = c->slot_capp;
    const bool slots = (double)ng * (double)(capm + capp) * sizeof(int32_t) <= HOT_SLOT_BUDGET;
    if (slots) {
        HOT_CK(c->slot_m2p.ensure((size_t)ng * capm, s));
        HOT_CK(c->slot_p2p.ensure((size_t)ng * capp, s));
    }
    int64_t host[8];
#define HOT_TRAV_LAUNCH(M, ...)                                            \
    do {                                                                   \
        if (per_L > 0.0)                                                   \
            k_traverse<M, true><<<blocks, TW * 32, 0, s>>>(__VA_ARGS__);   \
        else                                                               \
            k_traverse<M, false><<<blocks, TW * 32, 0, s>>>(__VA_ARGS__);  \
    } while (0)
    for (int attempt = 0;; ++attempt) {
        HOT_CK(c->trav_scratch.ensure((size_t)nwarps * 2 * c->trav_cap, s));
        HOT_CK(cudaMemsetAsync(c->sizes.p + 50, 0, 6 * sizeof(int64_t), s));
        HOT_CK(cudaMemsetAsync(c->sizes.p + 58, 0, 4 * sizeof(int64_t), s));
        HOT_COUNT_LAUNCH();
        if (slots)
            HOT_TRAV_LAUNCH(2,
                ng, c->gcell.p, c->gcen.p, c->gdmax.p, c->tcell.p, c->tcellf.p, c->cend.p, c->child8.p, c->cnchild.p,
                c->ccount.p, c->ccom.p, c->cbmax.p, c->cB1.p, c->cB2.p, c->p_mom, c->prm.G, tol, guard, cBn, c->q_lo, c->rcq.p, c->rcqf.p, per_L, c->prm.ws, c->trav_scratch.p,
                c->trav_cap, work, c->cnt_m2p.p, c->cnt_p2p.p, nullptr, nullptr, c->slot_m2p.p, c->slot_p2p.p, stats,
                capm, capp, maxc, slot_over, c->gkey.p, c->d_status);
        else
            HOT_TRAV_LAUNCH(0,
                ng, c->gcell.p, c->gcen.p, c->gdmax.p, c->tcell.p, c->tcellf.p, c->cend.p, c->child8.p, c->cnchild.p,
                c->ccount.p, c->ccom.p, c->cbmax.p, c->cB1.p, c->cB2.p, c->p_mom, c->prm.G, tol, guard, cBn, c->q_lo, c->rcq.p, c->rcqf.p, per_L, c->prm.ws, c->trav_scratch.p,
                c->trav_cap, work, c->cnt_m2p.p, c->cnt_p2p.p, nullptr, nullptr, nullptr, nullptr, stats, 0, 0, maxc,
                slot_over, c->gkey.p, c->d_status);
        int r = hot_scan_u32_to_i64(c->cnt_m2p.p, c->off_m2p.p, ng, c->scan_tmp.p, s);
        if (r) return r;
        r = hot_scan_u32_to_i64(c->cnt_p2p.p, c->off_p2p.p, ng, c->scan_tmp.p, s);
        if (r) return r;
        HOT_CK(cudaMemcpyAsync(host + 0, c->off_m2p.p + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HOT_CK(cudaMemcpyAsync(host + 1, c->off_p2p.p + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HOT_CK(cudaMemcpyAsync(host + 2, stats, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HOT_CK(cudaMemcpyAsync(host + 4, c->sizes.p + 58, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HOT_CK(cudaStreamSynchronize(s));
        unsigned st = 0;
        HOT_CK(cudaMemcpy(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
        if (st & HOT_ST_FRONTIER) {
            HOT_CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s));
            if (attempt >= 3) return HOT_EOVERFLOW;
            c->trav_cap *= 4;
            continue;
        }
        int e = hot_sync_status(c);
        if (e) return e;
        break;
    }
    c->n_m2p = host[0];
    c->n_p2p = host[1];
    c->n_m2p_int = host[2];
    c->n_pairs = host[3];
    c->n_p2p_src = host[7];
    const bool fits = slots && (host[6] & 0xffffffffll) == 0;
    auto round_cap = [](int64_t n) { return ((n + n / 4 + 256) + 255) / 256 * 256; };
    c->slot_capm = round_cap(host[4]);
    c->slot_capp = round_cap(host[5]);
    HOT_CK(c->l_m2p.ensure(c->n_m2p + 1, s));
    HOT_CK(c->l_p2p.ensure(c->n_p2p + 1, s));
    if (fits) {
        HOT_COUNT_LAUNCH();
        k_compact_lists<<<hot_blocks(ng * 32, 256), 256, 0, s>>>(ng, capm, capp, c->slot_m2p.p, c->slot_p2p.p,
                                                                  c->off_m2p.p, c->off_p2p.p, c->l_m2p.p,
                                                                  c->l_p2p.p);
    } else {
        HOT_CK(cudaMemsetAsync(work, 0, sizeof(int64_t), s));
        HOT_COUNT_LAUNCH();
        HOT_TRAV_LAUNCH(1,
            ng, c->gcell.p, c->gcen.p, c->gdmax.p, c->tcell.p, c->tcellf.p, c->cend.p, c->child8.p, c->cnchild.p, c->ccount.p,
            c->ccom.p, c->cbmax.p, c->cB1.p, c->cB2.p, c->p_mom, c->prm.G, tol, guard, cBn, c->q_lo, c->rcq.p, c->rcqf.p, per_L, c->prm.ws, c->trav_scratch.p, c->trav_cap,
            work, nullptr, nullptr, c->off_m2p.p, c->off_p2p.p, c->l_m2p.p, c->l_p2p.p, stats + 2, 0, 0, maxc,
            slot_over, nullptr, c->d_status);
    }
    int rs = work_items(c);
    if (rs) return rs;
    hot_toc(c, 3);
    if (cudaGetLastError() != cudaSuccess) return HOT_ECUDA;
    c->tol_lists = tol;
    c->stage = 3;
    return HOT_OK;
}
