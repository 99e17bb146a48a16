"""Periodic boundaries, host side (no GPU): the library's lattice sums (Sec. "Boundary
Conditions") against the oracle's and against the identities they obey."""
import math

import numpy as np
import pytest

from oracle import periodic as PR
from paper_1310_4502_gb300 import hot


def gidx(g):
    """Graded index of a multi-index (by |g|, then descending g_x, then descending g_y)."""
    n = sum(g)
    j = g[1] + g[2]
    return n * (n + 1) * (n + 2) // 6 + j * (j + 1) // 2 + g[2]


def order_scale(R):
    """Largest |D| of every order, the odd orders (zero by cubic symmetry) taking their
    even neighbours'."""
    mx = {}
    for g, v in R.items():
        mx[sum(g)] = max(mx.get(sum(g), 0.0), abs(v))
    return {n: max(mx.get(k, 0.0) for k in (n - 1, n, n + 1)) for n in mx}


@pytest.mark.parametrize("L,ws,order", [(1.0, 2, 17), (2.5, 1, 9), (0.3, 2, 11), (7.0, 1, 17)])
def test_lattice_sums_match_the_oracle(L, ws, order):
    """Two independent evaluations of the same Ewald-split lattice sums (the library: the
    McMurchie-Davidson recurrence in units of L; the oracle: closed-form radial
    derivatives in absolute units) agree to 1e-13 of the order's scale up to order 5,
    5e-11 up to order 9 and 1e-8 above: both lose digits to the cancellation of the split
    terms at high order (the oracle's values change by ~2e-9 at order 11 under a change of
    L alone; the library's order 10 and 14 sums are within 4e-10 of 40-digit values)."""
    D = hot.lattice_sums(L, ws, order)
    assert D.shape == ((order + 1) * (order + 2) * (order + 3) // 6,)
    R = PR.lattice_coefficients(L, order, ws)
    sc = order_scale(R)
    for g, v in R.items():
        bound = 1e-13 if sum(g) <= 5 else (5e-11 if sum(g) <= 9 else 1e-8)
        assert abs(D[gidx(g)] - v) <= bound * sc[sum(g)], (g, D[gidx(g)], v)


def test_lattice_sums_laplace_and_symmetry():
    """psi_far is harmonic near 0 except for the neutralising background:
    sum_d D^(2 e_d) = 4 pi / V and sum_d D^(g + 2 e_d) = 0 for |g| >= 1; the cube's
    symmetry makes every odd order vanish and permuted indices equal."""
    L, K = 1.7, 17
    D = hot.lattice_sums(L, 2, K)
    sc = order_scale(PR.lattice_coefficients(L, K, 2))
    lap0 = D[gidx((2, 0, 0))] + D[gidx((0, 2, 0))] + D[gidx((0, 0, 2))]
    assert abs(lap0 - 4 * math.pi / L ** 3) < 1e-12 * sc[2]
    for n in range(1, K - 1):
        for a in range(n + 1):
            for b in range(n - a + 1):
                g = (a, b, n - a - b)
                lap = sum(D[gidx(tuple(g[e] + 2 * (e == d) for e in range(3)))] for d in range(3))
                assert abs(lap) < 1e-8 * sc[n + 2], (g, lap)
                if n % 2:
                    assert abs(D[gidx(g)]) < 1e-8 * sc[n], g
                for perm in ((b, a, n - a - b), (n - a - b, b, a), (a, n - a - b, b)):
                    assert abs(D[gidx(perm)] - D[gidx(g)]) < 1e-8 * sc[n]


def test_lattice_sums_scale_as_L_to_minus_order_plus_one():
    D1 = hot.lattice_sums(1.0, 2, 9)
    D2 = hot.lattice_sums(3.0, 2, 9)
    n = np.concatenate([[k] * ((k + 1) * (k + 2) // 2) for k in range(10)])
    np.testing.assert_allclose(D2 * 3.0 ** (n + 1), D1, rtol=1e-13, atol=1e-13 * np.abs(D1).max())


@pytest.mark.parametrize("L,ws,order", [(0.0, 2, 4), (-1.0, 2, 4), (float("nan"), 2, 4), (float("inf"), 2, 4),
                                        (1.0, 0, 4), (1.0, 3, 4), (1.0, 2, -1), (1.0, 2, 18)])
def test_lattice_sums_reject_bad_arguments(L, ws, order):
    with pytest.raises(hot.HotError) as e:
        hot.lattice_sums(L, ws, order)
    assert e.value.code == hot.HOT_EINVAL


def test_lattice_sums_ws1_minus_ws2_is_the_shell_sum():
    """psi_far(ws = 1) - psi_far(ws = 2) is the plain sum of 1/|r + nL| over the 98 images
    with |n|_inf = 2: its derivatives at 0 (a finite sum, no Ewald splitting) pin the
    library's split of near and far images."""
    L, K = 1.3, 9
    d = hot.lattice_sums(L, 1, K) - hot.lattice_sums(L, 2, K)
    r = np.arange(-2, 3)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    n = n[np.max(np.abs(n), axis=1) == 2]
    R = n * L
    u = np.sum(R * R, axis=1)

    def dfact(k):
        out = 1
        while k > 1:
            out *= k
            k -= 2
        return out
    # F(u) = u^(-1/2): F^(m)(u) = (-1/2)^m (2m - 1)!! u^(-(m + 1/2))
    F = np.array([(-0.5) ** m * dfact(2 * m - 1) * u ** (-(m + 0.5)) for m in range(K + 1)])
    ref = PR._radial_derivs(F, R, K)
    sc = order_scale(ref)
    for g, v in ref.items():
        assert abs(d[gidx(g)] - v) <= 1e-11 * max(sc[sum(g)], 1e-300) + 1e-14, (g, d[gidx(g)], v)


def test_far_field_with_the_library_sums_matches_the_oracle():
    """The oracle's far-field expansion fed with the library's lattice sums instead of its
    own: forces agree to 1e-11 of their rms (the sums differ only at high orders, where
    the weights (L/2)^n / n! are small)."""
    rng = np.random.default_rng(9)
    x = rng.uniform(0, 1, (300, 3))
    m = rng.uniform(0.5, 1.5, 300) / 300
    D = hot.lattice_sums(1.0, 2, 17)
    Do = PR.lattice_coefficients(1.0, 17, 2)
    a1, p1 = PR.far_field(x, m, 1.0, (0.0, 0.0, 0.0), D=Do)
    a2, p2 = PR.far_field(x, m, 1.0, (0.0, 0.0, 0.0), D={g: D[gidx(g)] for g in Do})
    assert np.max(np.abs(a1 - a2)) < 1e-11 * np.sqrt(np.mean(a1 ** 2))
    assert np.max(np.abs(p1 - p2)) < 1e-11 * np.sqrt(np.mean(p1 ** 2))
