"""The uniform-box field routine of the CUDA path (csrc/hot_box.cuh, for background
subtraction), compiled for the host, against the oracle's (oracle/background.py): the two
evaluate the same closed form in code written separately, and the oracle's is pinned
against quadrature and Poisson's equation (tests/test_background_oracle.py).  No GPU."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import background as BG

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1310_4502_gb300", "csrc")

SHIM = r"""
#include <cmath>
#include <cstdint>
#define __device__
#define __forceinline__ inline
template <class T> inline T hb_log(T v) { return std::log(v); }
template <class T> inline T hb_atan(T v) { return std::atan(v); }
template <class T> inline T hb_sqrt(T v) { return std::sqrt(v); }
template <class T> inline T hb_div(T a, T b) { return a / b; }
#include "hot_box.cuh"
extern "C" void field(int64_t n, const double *p, const double *lo, const double *hi, double Grho, double *acc,
                      double *pot)
{
    const double L[3] = {lo[0], lo[1], lo[2]}, H[3] = {hi[0], hi[1], hi[2]};
    for (int64_t i = 0; i < n; ++i) {
        double ax = 0, ay = 0, az = 0, ph = 0;
        box_field<double>(p[3 * i], p[3 * i + 1], p[3 * i + 2], L, H, Grho, ax, ay, az, ph);
        acc[3 * i] = ax; acc[3 * i + 1] = ay; acc[3 * i + 2] = az; pot[i] = ph;
    }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("box")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    so = d / "shim.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)], check=True)
    L = C.CDLL(str(so))
    L.field.argtypes = [C.c_int64] + [C.c_void_p] * 3 + [C.c_double] + [C.c_void_p] * 2
    return L


def field(L, p, lo, hi, Grho):
    p = np.ascontiguousarray(p, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    acc = np.zeros((len(p), 3))
    pot = np.zeros(len(p))
    L.field(len(p), p.ctypes.data, lo.ctypes.data, hi.ctypes.data, Grho, acc.ctypes.data, pot.ctypes.data)
    return acc, pot


def test_box_field_matches_the_oracle(lib):
    rng = np.random.default_rng(12)
    lo, hi = np.array([-0.5, -0.3, -0.2]), np.array([0.5, 0.4, 0.9])
    # inside, around, a few sizes away; plus points on faces, edges and corners
    pts = np.vstack([rng.uniform(lo, hi, (200, 3)), rng.uniform(lo - 1, hi + 1, (200, 3)),
                     rng.uniform(lo - 4, hi + 4, (100, 3)),
                     [[0.5, 0.1, 0.3], [0.0, -0.3, 0.0], [0.5, 0.4, 0.2], [-0.5, -0.3, -0.2], [0.5, 0.4, 0.9],
                      [1.0, -0.3, 0.9], [-0.5, 2.0, 0.0]]])
    a, p = field(lib, pts, lo, hi, 1.3)
    ra, rp = BG.box_field(pts, lo, hi, rho=1.3)
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
    scale = np.abs(ra).max()
    np.testing.assert_allclose(a, ra, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(p, rp, rtol=1e-12, atol=1e-13 * np.abs(rp).max())
