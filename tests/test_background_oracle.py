"""Pins of the oracle's background subtraction (Sec. "Background Subtraction"): the field of
a uniform box against quadrature, Poisson's equation, its closed-form centre value and
additivity; the moments of a uniform cube; the tree code on the density contrast against
its exact value (the direct sum minus the root cube's field) at tol -> 0 and as tol falls.
No GPU."""
import math

import numpy as np
import pytest

import oracle
from oracle import background as BG


def quad_box(x, lo, hi, nodes=60):
    """Gauss-Legendre product quadrature of int (x' - x)/r^3 dV and -int dV/r over a box,
    for a point outside it (smooth integrand)."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    ax = [lo[d] + (hi[d] - lo[d]) * (t + 1) / 2 for d in range(3)]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :] * np.prod(hi - lo) / 8
    D = np.stack([X - x[0], Y - x[1], Z - x[2]], -1)
    r = np.linalg.norm(D, axis=-1)
    return np.array([np.sum(W * D[..., k] / r ** 3) for k in range(3)]), -np.sum(W / r)


LO, HI = np.array([-0.5, -0.3, -0.2]), np.array([0.5, 0.4, 0.9])


@pytest.mark.parametrize("x", [(1.3, 0.2, 0.1), (-2.0, 3.0, 1.0), (0.6, 0.5, 1.0), (0.0, -0.5, 0.3)])
def test_box_field_matches_quadrature_outside(x):
    x = np.array(x)
    a, p = BG.box_field(x[None], LO, HI, rho=1.7, G=0.9)
    aq, pq = quad_box(x, LO, HI)
    np.testing.assert_allclose(a[0], 1.7 * 0.9 * aq, rtol=0, atol=1e-12 * np.abs(aq).max())
    assert abs(p[0] - 1.7 * 0.9 * pq) < 1e-12 * abs(pq)


def test_box_field_centre_value_and_symmetry():
    """At the centre of a unit cube, int dV / r = 3 ln((sqrt 3 + 1)/(sqrt 3 - 1)) - pi/2 and
    the field vanishes; the field is odd under reflection through the centre."""
    a, p = BG.box_field(np.zeros((1, 3)), -0.5 * np.ones(3), 0.5 * np.ones(3))
    exact = 3 * math.log((math.sqrt(3) + 1) / (math.sqrt(3) - 1)) - math.pi / 2
    assert abs(-p[0] - exact) < 1e-14 and np.abs(a).max() < 1e-15
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (20, 3))
    a1, p1 = BG.box_field(x, -0.5 * np.ones(3), 0.5 * np.ones(3))
    a2, p2 = BG.box_field(-x, -0.5 * np.ones(3), 0.5 * np.ones(3))
    np.testing.assert_allclose(a1, -a2, atol=1e-14)
    np.testing.assert_allclose(p1, p2, rtol=1e-14)


@pytest.mark.parametrize("x,inside", [((0.1, 0.05, 0.3), True), ((-0.4, 0.35, -0.1), True),
                                      ((1.2, 0.3, 0.1), False), ((0.3, -0.8, 1.5), False)])
def test_box_field_poisson_and_gradient(x, inside):
    """div a = -4 pi G rho inside the box and 0 outside; a = -grad phi (central
    differences)."""
    x = np.array(x)
    h = 1e-4
    div, grad = 0.0, np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        ap, pp = BG.box_field((x + e)[None], LO, HI)
        am, pm = BG.box_field((x - e)[None], LO, HI)
        div += (ap[0, k] - am[0, k]) / (2 * h)
        grad[k] = (pp[0] - pm[0]) / (2 * h)
    a, _ = BG.box_field(x[None], LO, HI)
    assert abs(div - (-4 * math.pi if inside else 0.0)) < 1e-5
    assert np.abs(a[0] + grad).max() < 1e-6


def test_box_field_is_additive_and_far_field_is_a_point_mass():
    rng = np.random.default_rng(4)
    x = rng.uniform(-1.5, 1.5, (30, 3))
    mid = 0.1
    a, p = BG.box_field(x, LO, HI)
    a1, p1 = BG.box_field(x, LO, np.array([mid, HI[1], HI[2]]))
    a2, p2 = BG.box_field(x, np.array([mid, LO[1], LO[2]]), HI)
    np.testing.assert_allclose(a1 + a2, a, atol=1e-12)
    np.testing.assert_allclose(p1 + p2, p, rtol=1e-12)
    # a cube has no quadrupole: at 10 sides its field is a point mass's to O((s/d)^4)
    d = np.array([7.0, -5.0, 4.0])
    ac, pc = BG.box_field(d[None], -0.5 * np.ones(3), 0.5 * np.ones(3))
    r = np.linalg.norm(d)
    np.testing.assert_allclose(ac[0], -d / r ** 3, rtol=2e-4)
    assert abs(pc[0] + 1 / r) < 2e-4 / r


def test_cube_moments_and_radial_moments():
    """Moments of a uniform cube about its centre against exact quadrature (polynomials);
    the radial moments int |x|^n dV: even n against the multinomial closed form, odd n
    converged in the number of nodes."""
    s, rho, p = 0.7, 2.5, 6
    t, w = np.polynomial.legendre.leggauss(8)
    X, Y, Z = np.meshgrid(*(0.5 * s * t,) * 3, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :] * (0.5 * s) ** 3
    M = BG.cube_moments(s, p, rho)
    for k, a in enumerate(oracle.multi_indices(p)):
        assert abs(M[k] - rho * np.sum(W * X ** a[0] * Y ** a[1] * Z ** a[2])) < 1e-15 * rho * s ** 3
    for n in (2, 4, 6, 8):
        m = n // 2
        exact = 0.0
        for i in range(m + 1):
            for j in range(m + 1 - i):
                k = m - i - j
                c = math.factorial(m) / (math.factorial(i) * math.factorial(j) * math.factorial(k))
                exact += c * np.prod([0.5 ** (2 * e) / (2 * e + 1) for e in (i, j, k)])
        assert abs(BG.cube_radial_moment(n) - exact) < 1e-13 * exact
    for n in (5, 7):
        assert abs(BG.cube_radial_moment(n, 48) - BG.cube_radial_moment(n, 96)) < 1e-12


def _lattice(n, amp, seed):
    """Perturbed lattice in the unit cube, with massless particles at the corners so that
    the tree's root cube (the key frame) is the cube the matter fills."""
    rng = np.random.default_rng(seed)
    g = (np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) / n
    x = g + amp / n * rng.standard_normal(g.shape)
    c = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float) * (1 - 1e-12)
    m = np.full(len(x), 1.0 / len(x))
    return np.vstack([x, c]), np.concatenate([m, np.zeros(8)])


def test_background_tree_is_exact_when_nothing_is_expanded():
    """At tol -> 0 every interaction is a particle pair or an analytic cube: the result is
    the direct sum minus the root cube's field, whatever the surrounding cube."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (400, 3))
    m = rng.uniform(0.5, 1.5, 400) / 400
    for up in (0, 2):
        bt = oracle.background.BackgroundTree(x, m, p=4, leaf_max=16, group_max=32, up=up)
        ra, rp = bt.exact()
        a, p, cnt = bt.force(1e-300)
        assert cnt["m2p_contrast"] == 0 and cnt["m2p_empty"] == 0
        assert np.max(np.linalg.norm(a - ra, axis=1) / np.linalg.norm(ra, axis=1)) < 1e-11
        assert np.max(np.abs(p - rp)) < 1e-11 * np.max(np.abs(rp))


def test_background_tree_converges_and_gives_the_contrast_field():
    """On a perturbed lattice the contrast field is a small part of the full field, and the
    tree code reaches it with an rms absolute error below tol, falling with tol."""
    x, m = _lattice(9, 0.05, 5)
    bt = oracle.background.BackgroundTree(x, m, p=4, leaf_max=8, group_max=16)
    ra, _ = bt.exact()
    fa, _ = oracle.direct(x, m)
    live = m > 0
    assert np.sqrt(np.mean(np.sum(ra[live] ** 2, 1))) < 0.05 * np.sqrt(np.mean(np.sum(fa[live] ** 2, 1)))
    errs = []
    for tol in (1e-3, 1e-4, 1e-5):
        a, _, cnt = bt.force(tol)
        assert cnt["m2p_contrast"] > 0
        e = np.sqrt(np.mean(np.sum((a[live] - ra[live]) ** 2, 1)))
        assert e < tol, (tol, e)
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]
