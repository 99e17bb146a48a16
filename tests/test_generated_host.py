"""The generated expansion routines of the CUDA path, compiled for the host, against the oracle.

generated.cuh holds plain arithmetic (no intrinsics besides the reciprocal square root,
which the shim below supplies), so the same source the device compiles can be built with
g++ and checked without a GPU:
* m2p_record + m2p_eval (float and double) against the oracle's M2P (Eq. for the
  multipole expansion of the softened potential, its gradient for the acceleration);
* m2p_tangent: the directional derivative of the acceleration against a central
  difference of the oracle's M2P;
* m2p_cbar + m2p_record_adjoint: dL/dM of L = u.a + v phi, which is linear in M, against
  L evaluated by the oracle on unit moment vectors;
* the moment translation (in the kernel's three one-dimensional passes): the translated
  moments against the oracle's moments taken directly about the new centre; the adjoint's
  transposed translation tables against <y, T x> = <T^T y, x>.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1310_4502_gb300", "csrc")

SHIM = r"""
#include <cmath>
#define __device__
#define __forceinline__ inline
#define __constant__
#define __restrict__
struct alignas(16) float4 { float x, y, z, w; };
struct alignas(16) double2 { double x, y; };
inline float hot_rsqrt(float u) { return 1.0f / std::sqrt(u); }
inline double hot_rsqrt(double u) { return 1.0 / std::sqrt(u); }
#include "generated.cuh"

template <int P, typename T>
void ev(const double *M, const double *z, double is, double G, double eps, const double *R, double *out)
{
    alignas(16) T rec[400];
    m2p_record<P, T>(M, z, is, G, eps, rec);
    T phi = 0, ax = 0, ay = 0, az = 0;
    m2p_eval<P, T>(rec, (T)R[0], (T)R[1], (T)R[2], phi, ax, ay, az);
    out[0] = ax; out[1] = ay; out[2] = az; out[3] = phi;
}
template <int P>
void tg(const double *M, double is, double G, double eps, const double *R, const double *u, double v, double *out)
{
    alignas(16) double rec[400];
    const double z[3] = {0, 0, 0};
    m2p_record<P, double>(M, z, is, G, eps, rec);
    double phi = 0, ax = 0, ay = 0, az = 0, dx = 0, dy = 0, dz = 0;
    m2p_tangent<P, double>(rec, R[0], R[1], R[2], u[0], u[1], u[2], phi, ax, ay, az, dx, dy, dz);
    out[0] = ax; out[1] = ay; out[2] = az; out[3] = phi; out[4] = dx; out[5] = dy; out[6] = dz;
    double cb[200] = {0}, mb[200] = {0};
    m2p_cbar<P, double>(rec[0], rec[1], R[0], R[1], R[2], u[0], u[1], u[2], v, cb);
    m2p_record_adjoint<P>(cb, is, G, mb);
    for (int i = 0; i < HOT_NCOMP[P]; ++i) out[8 + i] = mb[i];
}
#define DISPATCH(F, ...) switch (p) { case 0: F<0>(__VA_ARGS__); break; case 1: F<1>(__VA_ARGS__); break; \
    case 2: F<2>(__VA_ARGS__); break; case 3: F<3>(__VA_ARGS__); break; case 4: F<4>(__VA_ARGS__); break; \
    case 5: F<5>(__VA_ARGS__); break; case 6: F<6>(__VA_ARGS__); break; }
#define DISPATCH8(F, ...) switch (p) { case 7: F<7>(__VA_ARGS__); break; case 8: F<8>(__VA_ARGS__); break; \
    default: DISPATCH(F, __VA_ARGS__) }
template <int P> void ev32(const double *M, const double *z, double is, double G, double e, const double *R, double *o)
{ ev<P, float>(M, z, is, G, e, R, o); }
template <int P> void ev64(const double *M, const double *z, double is, double G, double e, const double *R, double *o)
{ ev<P, double>(M, z, is, G, e, R, o); }
extern "C" {
void g_eval(int p, int dbl, const double *M, const double *z, double is, double G, double eps, const double *R,
            double *out)
{
    if (dbl) { DISPATCH8(ev64, M, z, is, G, eps, R, out) } else { DISPATCH8(ev32, M, z, is, G, eps, R, out) }
}
void g_tangent(int p, const double *M, double is, double G, double eps, const double *R, const double *u,
               double v, double *out)
{
    DISPATCH(tg, M, is, G, eps, R, u, v, out)
}
static double dpow(const double *d, int g)
{
    double v = 1.0;
    for (int e = 0; e < 3; ++e)
        for (int t = 0; t < hot_midx[g][e]; ++t) v *= d[e];
    return v;
}
void g_radj(int p, const double *cb, double is, double G, double *serial, double *table)
{
    for (int a = 0; a < HOT_NCOMP[p]; ++a) serial[a] = 0.0;
    DISPATCH(m2p_record_adjoint, cb, is, G, serial)
    double ip[16];
    ip[0] = 1.0;
    for (int e = 1; e < 16; ++e) ip[e] = ip[e - 1] * is;
    for (int a = 0; a < HOT_NCOMP[p]; ++a) {
        double t = 0.0;
        for (int j = radj_start[RADJ_SBASE[p] + a]; j < radj_start[RADJ_SBASE[p] + a + 1]; ++j)
            t += radj_f[j] * ip[radj_e[j]] * cb[radj_q[j]];
        table[a] = G * t;
    }
}
static int mom_index(int i, int j, int k)
{
    const int n = i + j + k;
    return n * (n + 1) * (n + 2) / 6 + (n - i) * (n - i + 1) / 2 + (n - i - j);
}
static double binom(int n, int r)
{
    double v = 1.0;
    for (int t = 1; t <= r; ++t) v = v * (double)(n - r + t) / (double)t;
    return v;
}
// the moment translation as the moments kernel applies it: three one-dimensional passes
void g_m2m(int p, const double *Mc, const double *d, double *Mp)
{
    const int nc = HOT_NCOMP[p];
    double a[84], b[84];
    for (int q = 0; q < nc; ++q) a[q] = Mc[q];
    for (int e = 0; e < 3; ++e) {
        for (int q = 0; q < nc; ++q) {
            int x[3] = {hot_midx[q][0], hot_midx[q][1], hot_midx[q][2]};
            double t = 0.0, pw = 1.0;
            const int top = x[e];
            // sum over x_e' <= x_e of C(x_e, x_e') d_e^(x_e - x_e') a(.., x_e', ..)
            for (int r = top; r >= 0; --r) {
                int y[3] = {x[0], x[1], x[2]};
                y[e] = r;
                t += binom(top, r) * pw * a[mom_index(y[0], y[1], y[2])];
                pw *= d[e];
            }
            b[q] = t;
        }
        for (int q = 0; q < nc; ++q) a[q] = b[q];
    }
    for (int q = 0; q < nc; ++q) Mp[q] = a[q];
}
void g_m2mt(int p, const double *Mbp, const double *d, double *Mbc)
{
    for (int b = 0; b < HOT_NCOMP[p]; ++b) {
        double t = 0.0;
        for (int j = m2mt_start[b]; j < m2mt_start[b + 1] && m2mt_alpha[j] < HOT_NCOMP[p]; ++j)
            t += m2mt_coef[j] * dpow(d, m2mt_gamma[j]) * Mbp[m2mt_alpha[j]];
        Mbc[b] = t;
    }
}
}
"""


@pytest.fixture(scope="module")
def gen(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("gen")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    so = d / "shim.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)],
                   check=True)
    L = C.CDLL(str(so))
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    L.g_eval.argtypes = [C.c_int, C.c_int, dp, dp, C.c_double, C.c_double, C.c_double, dp, dp]
    L.g_tangent.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double, dp, dp, C.c_double, dp]
    L.g_m2m.argtypes = [C.c_int, dp, dp, dp]
    L.g_radj.argtypes = [C.c_int, dp, C.c_double, C.c_double, dp, dp]
    L.g_m2mt.argtypes = [C.c_int, dp, dp, dp]
    for f in (L.g_eval, L.g_tangent, L.g_m2m, L.g_m2mt, L.g_radj):
        f.restype = None
    return L


def _cluster(rng, n=24):
    z0 = rng.uniform(-2, 2, 3)
    pos = z0 + 0.3 * rng.standard_normal((n, 3))
    mass = rng.uniform(0.5, 1.5, n)
    com = (mass[:, None] * pos).sum(0) / mass.sum()
    bmax = np.max(np.linalg.norm(pos - com, axis=1))
    inv_s = 2.0 ** -np.ceil(np.log2(bmax))
    return pos, mass, com, inv_s, bmax


def _sink(rng, com, bmax):
    u = rng.standard_normal(3)
    return (rng.uniform(2.5, 6.0) * bmax) * u / np.linalg.norm(u)


@pytest.mark.parametrize("p", range(9))
def test_record_and_eval_match_oracle_m2p(gen, p):
    rng = np.random.default_rng(100 + p)
    for case in range(6):
        pos, mass, com, inv_s, bmax = _cluster(rng)
        M = oracle.moments(pos, mass, com, p)
        eps = [0.0, 0.05][case % 2]
        R = _sink(rng, com, bmax)
        ra, rphi = oracle.m2p(p, M, R, 1.0, eps)
        for dbl, tol in ((1, 1e-13), (0, 3e-6)):
            out = np.zeros(4)
            gen.g_eval(p, dbl, M, com, inv_s, 1.0, eps, R, out)
            assert np.linalg.norm(out[:3] - ra) / np.linalg.norm(ra) < tol, (p, dbl)
            assert abs(out[3] - rphi) / abs(rphi) < tol, (p, dbl)


@pytest.mark.parametrize("p", range(7))
def test_tangent_and_moment_adjoint(gen, p):
    rng = np.random.default_rng(200 + p)
    nc = oracle.ncomp(p)
    for case in range(4):
        pos, mass, com, inv_s, bmax = _cluster(rng)
        M = oracle.moments(pos, mass, com, p)
        eps = [0.0, 0.05][case % 2]
        R = _sink(rng, com, bmax)
        u = rng.standard_normal(3)
        v = float(rng.standard_normal())
        out = np.zeros(8 + 84)
        gen.g_tangent(p, M, inv_s, 1.0, eps, R, u, v, out)
        ra, rphi = oracle.m2p(p, M, R, 1.0, eps)
        assert np.linalg.norm(out[:3] - ra) / np.linalg.norm(ra) < 1e-13
        # directional derivative of the acceleration: fourth-order central difference
        h = 1e-3 * np.linalg.norm(R)
        f = [oracle.m2p(p, M, R + s * h * u, 1.0, eps)[0] for s in (1, -1, 2, -2)]
        fd = (8 * (f[0] - f[1]) - (f[2] - f[3])) / (12 * h)
        assert np.linalg.norm(out[4:7] - fd) / np.linalg.norm(fd) < 1e-8
        # L = u.a + v phi is linear in M: its gradient is L on unit moment vectors
        ref = np.zeros(nc)
        for i in range(nc):
            e = np.zeros(nc)
            e[i] = 1.0
            a_i, phi_i = oracle.m2p(p, e, R, 1.0, eps)
            ref[i] = u @ a_i + v * phi_i
        assert np.max(np.abs(out[8:8 + nc] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("p", range(7))
def test_m2m_tables_translate_moments(gen, p):
    rng = np.random.default_rng(300 + p)
    nc = oracle.ncomp(p)
    for _ in range(4):
        pos, mass, com, _, _ = _cluster(rng)
        zp = com + rng.uniform(-0.5, 0.5, 3)
        Mc = oracle.moments(pos, mass, com, p)
        Mp = np.zeros(nc)
        gen.g_m2m(p, Mc, com - zp, Mp)
        ref = oracle.moments(pos, mass, zp, p)
        assert np.max(np.abs(Mp - ref)) <= 1e-12 * np.max(np.abs(ref))
        # transposed tables
        x = rng.standard_normal(nc)
        y = rng.standard_normal(nc)
        d = rng.uniform(-0.5, 0.5, 3)
        Tx = np.zeros(nc)
        Tty = np.zeros(nc)
        gen.g_m2m(p, x, d, Tx)
        gen.g_m2mt(p, y, d, Tty)
        assert y @ Tx == pytest.approx(Tty @ x, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("p", range(7))
def test_record_adjoint_gather_table_equals_generated_map(gen, p):
    """The per-moment gather table the cell kernel uses is the same linear map as the
    straight-line record adjoint (itself pinned against the oracle above)."""
    rng = np.random.default_rng(400 + p)
    nc = oracle.ncomp(p)
    cb = rng.standard_normal(200)
    a = np.zeros(nc)
    b = np.zeros(nc)
    gen.g_radj(p, cb, 0.25, 1.7, a, b)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
