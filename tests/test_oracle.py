"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an invariant, a special case that reduces to a textbook result or a library
routine, or brute force by an independent route.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1310_4502_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_err(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


# --------------------------------------------------------------------------
# Direct sum (Eq. eom with a = 1, Plummer smoothing)
# --------------------------------------------------------------------------

def test_direct_two_body_closed_form():
    eps, G = 0.3, 2.5
    pos = np.array([[0.1, -0.2, 0.3], [1.1, 0.6, -0.1]])
    mass = np.array([0.7, 1.9])
    acc, pot = oracle.direct(pos, mass, G, eps)
    d = pos[1] - pos[0]
    s = math.sqrt(d @ d + eps * eps)
    np.testing.assert_allclose(acc[0], G * mass[1] * d / s ** 3, rtol=1e-14)
    np.testing.assert_allclose(acc[1], -G * mass[0] * d / s ** 3, rtol=1e-14)
    np.testing.assert_allclose(pot, [-G * mass[1] / s, -G * mass[0] / s], rtol=1e-14)


def test_direct_third_law_and_translation():
    rng = np.random.default_rng(3)
    pos = rng.standard_normal((500, 3))
    mass = rng.uniform(0.5, 2.0, 500)
    acc, _ = oracle.direct(pos, mass, 1.0, 0.05)
    net = (mass[:, None] * acc).sum(0)
    scale = np.abs(mass[:, None] * acc).sum()
    assert np.all(np.abs(net) < 1e-13 * scale)
    acc2, _ = oracle.direct(pos + np.array([3.0, -7.0, 11.0]), mass, 1.0, 0.05)
    assert np.max(rel_err(acc2, acc)) < 1e-10


def _fibonacci_shell(n):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = math.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def test_direct_shell_theorem():
    """Newton's shell theorem: zero force inside a uniform shell, GM/r^2 outside,
    constant potential -GM/R inside.  Massless probes measure the field."""
    n = 20000
    shell = _fibonacci_shell(n)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((40, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    inner = u[:20] * rng.uniform(0.0, 0.6, 20)[:, None]
    outer = u[20:] * rng.uniform(1.5, 4.0, 20)[:, None]
    pos = np.concatenate([shell, inner, outer])
    mass = np.concatenate([np.full(n, 1.0 / n), np.zeros(40)])
    acc, pot = oracle.direct(pos, mass, 1.0, 0.0)
    assert np.max(np.abs(acc[n:n + 20])) < 1e-5
    np.testing.assert_allclose(pot[n:n + 20], -1.0, rtol=1e-5)
    r = np.linalg.norm(outer, axis=1)
    expect = -outer / r[:, None] ** 3
    assert np.max(rel_err(acc[n + 20:], expect)) < 1e-5
    np.testing.assert_allclose(pot[n + 20:], -1.0 / r, rtol=1e-5)


def test_direct_plummer_profile():
    """Spherical symmetry: the mean radial acceleration at radius r is -G M(<r)/r^2.
    Compared with the realised enclosed mass (removes sampling noise of the
    monopole); tolerance = 4 sigma of the bin mean + the O(eps^2/r^2) softening bias."""
    n = 16384
    x = W.plummer(n, seed=11)
    m = np.full(n, 1.0 / n)
    eps = 0.01
    acc, _ = oracle.direct(x, m, 1.0, eps)
    r = np.linalg.norm(x, axis=1)
    ar = np.sum(acc * x, 1) / r
    order = np.argsort(r)
    menc = np.empty(n)
    menc[order] = np.arange(n) / n
    expect = -menc / r ** 2
    edges = [0.2, 0.4, 0.7, 1.0, 1.5, 2.5, 4.0, 8.0]
    for lo, hi in zip(edges[:-1], edges[1:]):
        s = (r >= lo) & (r < hi)
        d = (ar[s] - expect[s]) / np.abs(expect[s])
        sigma = d.std() / math.sqrt(s.sum())
        assert abs(d.mean()) < 4 * sigma + 1.5 * eps * eps / lo ** 2, (lo, hi, d.mean(), sigma)
    # and the generator follows the truncated Plummer law M(<r) = r^3/(r^2+1)^{3/2} / X(20)
    xm = W.plummer_xmax(20.0)
    for rr in (0.5, 1.0, 2.0, 5.0):
        frac = np.mean(r < rr)
        want = rr ** 3 / (rr * rr + 1) ** 1.5 / xm
        assert abs(frac - want) < 4 * math.sqrt(want * (1 - want) / n)


# --------------------------------------------------------------------------
# Keys and sort
# --------------------------------------------------------------------------

def test_keys_golden():
    g = json.load(open(os.path.join(GOLDEN, "morton_keys.json")))
    pts = np.array([p["x"] for p in g["points"]])
    lo, L = oracle.bbox(pts)
    np.testing.assert_array_equal(lo, g["frame"]["lo"])
    assert L == g["frame"]["L"]
    k = oracle.keys(pts, lo, L)
    assert [int(v) for v in k] == [int(p["key"]) for p in g["points"]]


def _octant_digits(c, level):
    """Octant digit of each level, from integer coordinates by integer division."""
    out = []
    for lev in range(1, level + 1):
        sh = 21 - lev
        out.append(((c[:, 0] >> sh) & 1) * 4 + ((c[:, 1] >> sh) & 1) * 2 + ((c[:, 2] >> sh) & 1))
    return np.stack(out, 1)


def test_keys_are_octant_digit_strings():
    """Key order must be the lexicographic order of the per-level octant digits
    (the z-order descent of an oct-tree), and decoding the 63 bits must give back
    the integer coordinates."""
    rng = np.random.default_rng(7)
    pos = rng.uniform(-3.0, 5.0, (3000, 3)) * np.array([1.0, 0.5, 0.25])
    lo, L = oracle.bbox(pos)
    k = oracle.keys(pos, lo, L)
    c = np.minimum(np.floor((pos - lo) * (2.0 ** 21 / L)).astype(np.int64), 2 ** 21 - 1)
    dig = _octant_digits(c, 21)
    for i in range(3000):
        kk = int(k[i])
        assert kk >> 63 == 1
        dd = [(kk >> (3 * (21 - lev))) & 7 for lev in range(1, 22)]
        assert dd == list(dig[i])
    lex = np.lexsort(dig.T[::-1])
    np.testing.assert_array_equal(np.sort(k), k[lex])


def test_sort_stable_against_library():
    rng = np.random.default_rng(9)
    k = rng.integers(0, 40, 5000).astype(np.uint64) | np.uint64(1 << 63)
    perm = oracle.sort(k)
    np.testing.assert_array_equal(perm, np.argsort(k, kind="stable"))


# --------------------------------------------------------------------------
# Tree topology: brute force by counting particles per integer cell
# --------------------------------------------------------------------------

def _brute_cells(pos, leaf_max):
    lo, L = oracle.bbox(pos)
    c = np.minimum(np.floor((pos - lo) * (2.0 ** 21 / L)).astype(np.int64), 2 ** 21 - 1)
    counts = {}
    for lev in range(0, 22):
        sh = 21 - lev
        cc = c >> sh
        for t in map(tuple, cc):
            counts[(lev,) + t] = counts.get((lev,) + t, 0) + 1
    cells = set()
    for key, n in counts.items():
        lev = key[0]
        if lev == 0:
            cells.add((key, n))
            continue
        parent = (lev - 1, key[1] >> 1, key[2] >> 1, key[3] >> 1)
        if counts[parent] > leaf_max and lev - 1 < 21:
            cells.add((key, n))
    return cells


@pytest.mark.parametrize("leaf_max", [1, 3, 16])
def test_tree_topology_brute_force(leaf_max):
    rng = np.random.default_rng(leaf_max)
    n = 400
    pos = np.concatenate([rng.standard_normal((n // 2, 3)) * 0.01,
                          rng.uniform(-1, 1, (n - n // 2, 3))])
    pos[5] = pos[6]  # coincident pair: forces a level-21 leaf when leaf_max == 1
    t = oracle.Tree(pos, np.ones(n), leaf_max=leaf_max, group_max=64)
    cl = t.cells()
    got = set()
    for key, lev, cnt in zip(cl["key"], cl["level"], cl["count"]):
        kk, lev = int(key), int(lev)
        xyz = [0, 0, 0]
        for l in range(lev):
            d = (kk >> (3 * (lev - 1 - l))) & 7
            xyz[0] = xyz[0] * 2 + (d >> 2)
            xyz[1] = xyz[1] * 2 + ((d >> 1) & 1)
            xyz[2] = xyz[2] * 2 + (d & 1)
        assert kk >> (3 * lev) == 1
        got.add(((int(lev), *xyz), int(cnt)))
    assert got == _brute_cells(pos, leaf_max)
    # pre-order: a parent precedes its children, children in ascending key
    par = cl["parent"]
    assert par[0] == -1 and np.all(par[1:] < np.arange(1, len(par)))
    assert np.all(np.diff(cl["begin"]) >= 0)


@pytest.mark.parametrize("leaf_max,group_max", [(16, 64), (64, 128)])
def test_groups_partition_and_extent(leaf_max, group_max):
    w = W.make("plummer4096")
    t = oracle.Tree(w.pos, w.mass, leaf_max, group_max)
    cl = t.cells()
    g = t.groups()
    cov = np.zeros(w.n, dtype=int)
    k, perm = t.keys()
    sp = w.pos[perm]
    for c, cen, dm in zip(g["cell"], g["centre"], g["dmax"]):
        b, n = cl["begin"][c], cl["count"][c]
        cov[b:b + n] += 1
        assert n <= group_max or cl["nchild"][c] == 0
        assert cl["parent"][c] < 0 or cl["count"][cl["parent"][c]] > group_max
        x = sp[b:b + n]
        np.testing.assert_allclose(cen, 0.5 * (x.min(0) + x.max(0)), rtol=0, atol=1e-15)
        assert abs(dm - np.linalg.norm(x - cen, axis=1).max()) <= 1e-15 * max(dm, 1e-300)
    assert np.all(cov == 1)


# --------------------------------------------------------------------------
# Moments (Eq. moment tensor) and M2P (Cartesian expansion)
# --------------------------------------------------------------------------

def test_moments_hand_computed():
    # particles m=1 at (1,0,0), m=2 at (0,1,0), m=3 at (0,0,2), about z = 0, p = 2
    pos = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 2.0]])
    mass = np.array([1.0, 2.0, 3.0])
    M = oracle.moments(pos, mass, np.zeros(3), 2)
    idx = oracle.multi_indices(2)
    want = {(0, 0, 0): 6, (1, 0, 0): 1, (0, 1, 0): 2, (0, 0, 1): 6, (2, 0, 0): 1,
            (1, 1, 0): 0, (1, 0, 1): 0, (0, 2, 0): 2, (0, 1, 1): 0, (0, 0, 2): 12}
    assert [M[idx.index(a)] for a in want] == list(want.values())


def test_tree_moments_invariants():
    w = W.make("plummer4096")
    t = oracle.Tree(w.pos, w.mass)
    t.moments(4)
    mo = t.get_moments()
    cl = t.cells()
    idx = oracle.multi_indices(4)
    np.testing.assert_allclose(mo["mom"][:, 0], mo["mass"], rtol=1e-15)
    dip = mo["mom"][:, 1:4]
    scale = mo["mass"] * np.maximum(mo["bmax"], 1e-300)
    assert np.all(np.abs(dip) <= 1e-12 * scale[:, None])
    # binomial translation of moments (the M2M relation) reproduces direct moments
    k, perm = t.keys()
    sp, sm = w.pos[perm], w.mass[perm]
    rng = np.random.default_rng(1)
    for c in rng.choice(len(cl["key"]), 20, replace=False):
        b, n = cl["begin"][c], cl["count"][c]
        z0 = mo["com"][c]
        z1 = z0 + rng.standard_normal(3) * 0.1
        direct = oracle.moments(sp[b:b + n], sm[b:b + n], z1, 4)
        s = z0 - z1
        shifted = np.zeros_like(direct)
        for ia, a in enumerate(idx):
            for ib, bb in enumerate(idx):
                if all(bb[d] <= a[d] for d in range(3)):
                    coef = np.prod([math.comb(a[d], bb[d]) * s[d] ** (a[d] - bb[d]) for d in range(3)])
                    shifted[ia] += coef * mo["mom"][c][ib]
        np.testing.assert_allclose(shifted, direct, rtol=1e-9, atol=1e-14 * mo["mass"][c])
    # b_max, B_n against their definition on a few cells
    for c in rng.choice(len(cl["key"]), 10, replace=False):
        b, n = cl["begin"][c], cl["count"][c]
        r = np.linalg.norm(sp[b:b + n] - mo["com"][c], axis=1)
        assert mo["bmax"][c] == pytest.approx(r.max(), rel=1e-14)
        assert mo["B1"][c] == pytest.approx(np.sum(sm[b:b + n] * r ** 5), rel=1e-12)
        assert mo["B2"][c] == pytest.approx(np.sum(sm[b:b + n] * r ** 6), rel=1e-12)


def test_m2p_order0_is_point_mass():
    M = np.array([2.5])
    R = np.array([0.3, -1.2, 0.7])
    eps = 0.2
    a, phi = oracle.m2p(0, M, R, 1.5, eps)
    s = math.sqrt(R @ R + eps * eps)
    np.testing.assert_allclose(a, -1.5 * 2.5 * R / s ** 3, rtol=1e-14)
    assert phi == pytest.approx(-1.5 * 2.5 / s, rel=1e-14)


@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_m2p_single_offset_particle_converges(eps):
    """One particle at offset delta from the expansion centre: moments m delta^a.
    The softened Taylor series converges to the exact softened pair force with
    ratio |delta|/sqrt(|R|^2+eps^2); every derivative order enters (incl. the
    eps-dependent trace terms of the closed form)."""
    m, delta = 1.3, np.array([0.05, -0.08, 0.06])
    R = np.array([0.7, 0.4, -0.5])
    z = np.zeros(3)
    exact_a, exact_phi = oracle.direct(np.array([R, delta]), np.array([0.0, m]), 1.0, eps)
    ratio = np.linalg.norm(delta) / math.sqrt(R @ R + eps * eps)
    prev = np.inf
    for p in range(0, 9):
        M = oracle.moments(delta[None], np.array([m]), z, p)
        a, phi = oracle.m2p(p, M, R, 1.0, eps)
        err = np.linalg.norm(a - exact_a[0]) / np.linalg.norm(exact_a[0])
        assert err < 40 * ratio ** (p + 1)
        assert err < prev or err < 1e-14
        prev = err
    assert err < 1e-7


def test_m2p_error_bound_and_decay():
    """Fig. p8err setup: 512 particles uniform in a unit cube, one sink at distance r.
    The unsoftened error is bounded by E(d) and decays like r^-(p+3)."""
    rng = np.random.default_rng(8)
    x = rng.uniform(-0.5, 0.5, (512, 3))
    m = np.full(512, 1.0 / 512)
    z = x.T @ m / m.sum()
    rr = np.linalg.norm(x - z, axis=1)
    b = rr.max()
    for p in (1, 2, 4, 6, 8):
        M = oracle.moments(x, m, z, p)
        B1 = np.sum(m * rr ** (p + 1))
        B2 = np.sum(m * rr ** (p + 2))
        errs = []
        for dist in (2.0, 4.0, 8.0):
            u = np.array([0.48, -0.6, 0.64])
            X = z + dist * u
            ea, _ = oracle.direct(np.concatenate([X[None], x]), np.concatenate([[0.0], m]), 1.0, 0.0,
                                  sinks=[0])
            a, _ = oracle.m2p(p, M, X - z, 1.0, 0.0)
            e = np.linalg.norm(a - ea[0])
            assert e <= oracle.mac_bound(dist, b, B1, B2, p) * (1 + 1e-9) + 1e-15
            errs.append(e)
        if p <= 4:
            slope = math.log(errs[2] / errs[1]) / math.log(2.0)
            assert -(p + 3) - 1.0 < slope < -(p + 3) + 1.0, (p, slope)
    # "a single p=8 multipole is more accurate than direct summation in single
    # precision at r=4" (caption of Fig. p8err)
    X = z + 4.0 * np.array([0.48, -0.6, 0.64])
    ea, _ = oracle.direct(np.concatenate([X[None], x]), np.concatenate([[0.0], m]), 1.0, 0.0, sinks=[0])
    d32 = (x.astype(np.float32) - X.astype(np.float32))
    r32 = np.sqrt(np.sum(d32 * d32, 1, dtype=np.float32))
    a32 = np.sum((m.astype(np.float32) / r32 ** 3)[:, None] * d32, 0, dtype=np.float32)
    M8 = oracle.moments(x, m, z, 8)
    a8, _ = oracle.m2p(8, M8, X - z, 1.0, 0.0)
    assert np.linalg.norm(a8 - ea[0]) < np.linalg.norm(a32.astype(np.float64) - ea[0])


def test_mac_bound_monotone_positive():
    rng = np.random.default_rng(4)
    for _ in range(50):
        x = rng.standard_normal((30, 3)) * rng.uniform(0.1, 1)
        m = rng.uniform(0.1, 1, 30)
        z = x.T @ m / m.sum()
        r = np.linalg.norm(x - z, axis=1)
        b = r.max()
        p = int(rng.integers(0, 7))
        B1, B2 = np.sum(m * r ** (p + 1)), np.sum(m * r ** (p + 2))
        ds = b * np.linspace(1.01, 50, 200)
        E = [oracle.mac_bound(d, b, B1, B2, p) for d in ds]
        assert all(e > 0 for e in E)
        assert all(E[i + 1] < E[i] for i in range(len(E) - 1))


# --------------------------------------------------------------------------
# Treecode
# --------------------------------------------------------------------------

def test_tree_lists_cover_every_particle_once():
    w = W.make("plummer4096")
    t = oracle.Tree(w.pos, w.mass)
    t.moments(4)
    t.traverse(1e-4)
    cl = t.cells()
    L = t.lists()
    om, cm = L["m2p"]
    op, cp = L["p2p"]
    for g in range(len(om) - 1):
        cov = np.zeros(w.n, dtype=int)
        for c in cm[om[g]:om[g + 1]]:
            cov[cl["begin"][c]:cl["begin"][c] + cl["count"][c]] += 1
        for c in cp[op[g]:op[g + 1]]:
            assert cl["nchild"][c] == 0
            cov[cl["begin"][c]:cl["begin"][c] + cl["count"][c]] += 1
        assert np.all(cov == 1)


def test_tree_reduces_to_direct_sum():
    """A tolerance no cell can meet turns every interaction into P2P, and a set of
    at most group_max particles is a single group: both reduce to the direct sum."""
    w = W.make("plummer4096")
    a0, p0 = oracle.direct(w.pos, w.mass, 1.0, w.eps)
    a1, p1 = oracle.tree_force(w.pos, w.mass, p=4, tol=1e-300, eps=w.eps)
    assert np.max(rel_err(a1, a0)) < 1e-12
    np.testing.assert_allclose(p1, p0, rtol=1e-12)
    x = w.pos[:60]
    a0, _ = oracle.direct(x, w.mass[:60], 1.0, 0.0)
    a1, _ = oracle.tree_force(x, w.mass[:60], p=4, tol=1e-1, eps=0.0)
    assert np.max(rel_err(a1, a0)) < 1e-13


def test_tree_error_within_per_interaction_bound():
    """Unsoftened: each accepted interaction errs by at most tol (the acceptance
    bound is a theorem), so |a_tree - a_direct| <= tol * (#M2P of the sink's group)."""
    rng = np.random.default_rng(2)
    n = 3000
    pos = np.concatenate([rng.standard_normal((n // 2, 3)) * 0.1, rng.uniform(-1, 1, (n - n // 2, 3))])
    mass = np.full(n, 1.0 / n)
    ad, _ = oracle.direct(pos, mass, 1.0, 0.0)
    for p, tol in ((1, 1e-3), (4, 1e-4), (6, 1e-6)):
        t = oracle.Tree(pos, mass)
        t.moments(p)
        t.traverse(tol)
        at, _ = t.force(1.0, 0.0)
        L = t.lists()
        g = t.groups()
        cl = t.cells()
        nm = np.diff(L["m2p"][0])
        k, perm = t.keys()
        bound = np.zeros(n)
        for gi, c in enumerate(g["cell"]):
            b, cnt = cl["begin"][c], cl["count"][c]
            bound[perm[b:b + cnt]] = tol * nm[gi]
        err = np.linalg.norm(at - ad, axis=1)
        assert np.all(err <= bound * (1 + 1e-9) + 1e-13), (p, np.max(err / np.maximum(bound, 1e-300)))


def test_tree_error_shrinks_with_tolerance_and_order():
    w = W.make("plummer4096")
    ad, _ = oracle.direct(w.pos, w.mass, 1.0, w.eps)
    for p in (2, 4, 6):
        errs = []
        for tol in (1e-3, 1e-4, 1e-5, 1e-6):
            at, _ = oracle.tree_force(w.pos, w.mass, p=p, tol=tol, eps=w.eps)
            errs.append(np.sqrt(np.mean(rel_err(at, ad) ** 2)))
        assert all(errs[i + 1] < errs[i] for i in range(3)), (p, errs)
    # the config-1 setting (p = 4, tol = 1e-4) is well inside 1e-3 rms
    assert errs is not None


# --------------------------------------------------------------------------
# Gradients
# --------------------------------------------------------------------------

def test_direct_grad_against_finite_differences_and_invariants():
    rng = np.random.default_rng(12)
    n = 40
    pos = rng.standard_normal((n, 3))
    mass = rng.uniform(0.5, 1.5, n)
    w = rng.standard_normal((n, 3))
    v = rng.standard_normal(n)
    eps = 0.1

    def L(x, m):
        a, p = oracle.direct(x, m, 1.0, eps)
        return np.sum(w * a) + np.sum(v * p)

    gx, gm = oracle.direct_grad(pos, mass, w, v, 1.0, eps)
    h = 1e-5
    for k in range(0, n, 7):
        for d in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[k, d] += h
            xm[k, d] -= h
            fd = (L(xp, mass) - L(xm, mass)) / (2 * h)
            assert fd == pytest.approx(gx[k, d], rel=1e-6, abs=1e-8)
        mp, mm = mass.copy(), mass.copy()
        mp[k] += h
        mm[k] -= h
        assert (L(pos, mp) - L(pos, mm)) / (2 * h) == pytest.approx(gm[k], rel=1e-8, abs=1e-10)
    assert np.all(np.abs(gx.sum(0)) < 1e-10 * np.abs(gx).sum())
    assert np.sum(mass * gm) == pytest.approx(L(pos, mass), rel=1e-12)


def test_frozen_loss_partial_sums():
    """The frozen function at the base point is the tree force; the partial loss of
    particle k changes exactly like the full loss when only k moves; it is linear in mass."""
    rng = np.random.default_rng(13)
    n = 700
    pos = np.concatenate([rng.standard_normal((n // 2, 3)) * 0.05, rng.uniform(-1, 1, (n - n // 2, 3))])
    mass = rng.uniform(0.5, 1.5, n) / n
    w = rng.standard_normal((n, 3))
    v = rng.standard_normal(n)
    eps = 0.01
    t = oracle.Tree(pos, mass)
    t.moments(4)
    t.traverse(1e-5)
    a, p = t.force(1.0, eps)
    Lfull = t.frozen_loss(pos, mass, w, v, 1.0, eps)
    assert Lfull == pytest.approx(np.sum(w * a) + np.sum(v * p), rel=1e-13)
    for k in (0, 17, 350, 699):
        for d in range(3):
            x1 = pos.copy()
            x1[k, d] += 1e-3
            dfull = t.frozen_loss(x1, mass, w, v, 1.0, eps) - Lfull
            dpart = t.frozen_loss(x1, mass, w, v, 1.0, eps, k) - t.frozen_loss(pos, mass, w, v, 1.0, eps, k)
            assert dpart == pytest.approx(dfull, rel=1e-8, abs=1e-12 * abs(Lfull))
    m2 = mass * 1.7
    assert t.frozen_loss(pos, m2, w, v, 1.0, eps) == pytest.approx(1.7 * Lfull, rel=1e-12)


@pytest.mark.parametrize("p", [0, 1, 2, 4, 6])
def test_mac_bound_is_exact_for_collinear_particle(p):
    """For one particle at distance r from the expansion centre, on the line to the
    sink at distance d, the acceleration is 1/(d-r)^2 = d^-2 sum_n (n+1)(r/d)^n and
    the truncated expansion keeps n <= p: the error is the tail sum, which is what
    the acceptance bound E(d) sums in closed form (with B_n = m r^n, b = r)."""
    m, r, d = 0.8, 0.3, 1.1
    M = oracle.moments(np.array([[r, 0.0, 0.0]]), np.array([m]), np.zeros(3), p)
    a, _ = oracle.m2p(p, M, np.array([d, 0.0, 0.0]), 1.0, 0.0)
    exact = -m / (d - r) ** 2
    err = abs(a[0] - exact)
    E = oracle.mac_bound(d, r, m * r ** (p + 1), m * r ** (p + 2), p)
    tail = m / d ** 2 * sum((n + 1) * (r / d) ** n for n in range(p + 1, 400))
    assert E == pytest.approx(tail, rel=1e-12)
    assert err == pytest.approx(E, rel=1e-9)
    assert abs(a[1]) < 1e-15 and abs(a[2]) < 1e-15


def test_frozen_force_is_tree_force_at_its_own_positions():
    rng = np.random.default_rng(14)
    n = 900
    pos = np.concatenate([rng.standard_normal((n // 2, 3)) * 0.05, rng.uniform(-1, 1, (n - n // 2, 3))])
    mass = rng.uniform(0.5, 1.5, n) / n
    t = oracle.Tree(pos, mass)
    t.moments(4)
    t.traverse(1e-5)
    a0, p0 = t.force(1.0, 0.01)
    a1, p1 = t.frozen_force(pos, mass, 1.0, 0.01)
    np.testing.assert_array_equal(a1, a0)
    np.testing.assert_array_equal(p1, p0)
    # and the frozen loss is the weighted sum of the frozen force at moved positions
    x = pos + rng.standard_normal(pos.shape) * 1e-3
    w = rng.standard_normal((n, 3))
    a2, _ = t.frozen_force(x, mass, 1.0, 0.01)
    assert t.frozen_loss(x, mass, w, None, 1.0, 0.01) == pytest.approx(np.sum(w * a2), rel=1e-12)


def _tree(x, m):
    t = oracle.Tree(x, m)
    t.moments(0)
    t.traverse(1e-3)
    return t


def _rebuild_step(x, v, m, dt):
    """One kick-drift-kick step with the tree rebuilt at both force points."""
    t0 = _tree(x, m)
    a0, _ = t0.force(1.0, 0.0)
    t1 = _tree(x + dt * (v + 0.5 * dt * a0), m)
    return oracle.frozen_leapfrog([t0, t1], x, v, m, dt)


def test_leapfrog_two_body_energy_order_and_reversibility():
    """Two equal masses on an eccentric orbit (e about 0.5): the kick-drift-kick scheme of Sec. "Time
    Integration" keeps the energy error bounded at second order in dt over an orbit (the
    largest deviation is taken: at a full period the symplectic error nearly cancels) and
    is time reversible."""
    m = np.array([0.5, 0.5])
    x0 = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    vc = np.sqrt(0.5 / 2.0)  # circular speed: v^2/r = G m / d^2 with r = 0.5, d = 1
    v0 = np.array([[0.0, 0.7 * vc, 0.0], [0.0, -0.7 * vc, 0.0]])
    period = 2 * np.pi * 0.5 / vc  # covers more than one eccentric orbit

    def energy(x, v):
        return 0.5 * np.sum(m[:, None] * v * v) - m[0] * m[1] / np.linalg.norm(x[0] - x[1])

    errs = []
    for nsteps in (400, 800):
        x, v = x0.copy(), v0.copy()
        worst = 0.0
        for _ in range(nsteps):
            x, v = _rebuild_step(x, v, m, period / nsteps)
            worst = max(worst, abs(energy(x, v) - energy(x0, v0)))
        errs.append(worst)
    assert 3.0 < errs[0] / errs[1] < 5.0  # halving dt quarters the error
    x, v = x0.copy(), v0.copy()
    for _ in range(50):
        x, v = _rebuild_step(x, v, m, 0.01)
    v = -v
    for _ in range(50):
        x, v = _rebuild_step(x, v, m, 0.01)
    assert np.max(np.abs(x - x0)) < 1e-12 and np.max(np.abs(v + v0)) < 1e-12


# --------------------------------------------------------------------------
# K1 compensating kernel (Sec. "Force Smoothing").  The paper names Dehnen's K1
# without a formula; the reading is the unit-mass kernel of support eps with density
# rho(x) = 105/(64 pi eps^3) (1 - x^2)(5 - 9 x^2), x = r/eps.  The pins below derive
# the pair force and potential from that density by quadrature (shell theorem), so
# they are independent of the oracle's closed forms.
# --------------------------------------------------------------------------

def _k1_density(r, eps):
    x = r / eps
    return 105.0 / (64.0 * math.pi * eps ** 3) * (1 - x * x) * (5 - 9 * x * x) if x < 1 else 0.0


def test_k1_kernel_defining_properties():
    from scipy.integrate import quad
    eps = 0.37
    mass = quad(lambda r: 4 * math.pi * r * r * _k1_density(r, eps), 0, eps)[0]
    second = quad(lambda r: 4 * math.pi * r ** 4 * _k1_density(r, eps), 0, eps)[0]
    assert abs(mass - 1.0) < 1e-13
    assert abs(second) < 1e-14  # the compensation: zero second moment


@pytest.mark.parametrize("xr", [0.0, 0.05, 0.3, 0.5, 0.7453, 0.9, 0.999, 1.0, 1.2, 3.0])
def test_k1_pair_force_and_potential_from_density(xr):
    from scipy.integrate import quad
    eps = 0.37
    r = xr * eps
    f, f2, psi = oracle.soft_kernel("k1", eps, r)
    if r > 0:
        # shell theorem: enclosed mass M(r), a = M(r)/r^2 along d -> f = M(r)/r^3
        M = quad(lambda t: 4 * math.pi * t * t * _k1_density(t, eps), 0, min(r, eps))[0]
        assert abs(f - M / r ** 3) <= 1e-12 * abs(M / r ** 3)
        # potential: psi(r) = int_r^inf M(t)/t^2 dt
        Mof = lambda t: quad(lambda q: 4 * math.pi * q * q * _k1_density(q, eps), 0, min(t, eps))[0]
        tail = quad(lambda t: Mof(t) / (t * t), r, eps)[0] if r < eps else 0.0
        psi_ref = 1.0 / max(r, eps) + tail if r < eps else 1.0 / r
        assert abs(psi - psi_ref) <= 1e-11 * psi_ref
        # f2 = 2 df/d(r^2), against a central difference in r^2
        h = 1e-6 * r * r
        fp = oracle.soft_kernel("k1", eps, math.sqrt(r * r + h))[0]
        fm = oracle.soft_kernel("k1", eps, math.sqrt(r * r - h))[0]
        if abs(xr - 1.0) > 1e-3:  # f is continuous at the edge, f2 is not
            assert abs(f2 - 2 * (fp - fm) / (2 * h)) <= 1e-6 * abs(f2)
    else:
        # the centre: finite force coefficient and potential 105/(32 eps)
        assert abs(f - 175.0 / 16.0 / eps ** 3) <= 1e-14 * f
        assert abs(psi - 105.0 / (32.0 * eps)) <= 1e-14 * psi
    if xr >= 1.0:
        assert f == pytest.approx(1.0 / r ** 3, rel=1e-15) and psi == pytest.approx(1.0 / r, rel=1e-15)
        assert f2 == pytest.approx(-3.0 / r ** 5, rel=1e-15)


def test_k1_force_is_continuous_and_compensating():
    eps = 0.37
    below = oracle.soft_kernel("k1", eps, eps * (1 - 1e-12))
    above = oracle.soft_kernel("k1", eps, eps * (1 + 1e-12))
    assert abs(below[0] - above[0]) <= 1e-9 * above[0] and abs(below[2] - above[2]) <= 1e-9 * above[2]
    # above the Newtonian force near the edge, below it in the interior
    for x in (0.8, 0.9, 0.97):
        f = oracle.soft_kernel("k1", eps, x * eps)[0]
        assert f * (x * eps) ** 3 > 1.0
    for x in (0.1, 0.3, 0.5):
        f = oracle.soft_kernel("k1", eps, x * eps)[0]
        assert f * (x * eps) ** 3 < 1.0


def test_k1_direct_sum_third_law_and_newtonian_far_field():
    rng = np.random.default_rng(31)
    pos = rng.uniform(-1, 1, (300, 3))
    mass = rng.uniform(0.5, 1.5, 300)
    acc, pot = oracle.direct(pos, mass, 1.0, 0.3, soft="k1")
    assert np.linalg.norm((mass[:, None] * acc).sum(0)) < 1e-12 * np.abs(mass[:, None] * acc).sum()
    # the softening changes the force, so some pairs are inside the support
    a0, _ = oracle.direct(pos, mass, 1.0, 0.0)
    assert np.max(rel_err(acc, a0)) > 1e-3
    # all pairs farther apart than eps: the unsoftened sum, to rounding
    grid = np.stack(np.meshgrid(*[np.arange(4.0)] * 3, indexing="ij"), -1).reshape(-1, 3)
    m = np.ones(len(grid))
    ak, pk = oracle.direct(grid, m, 1.0, 0.9, soft="k1")
    an, pn = oracle.direct(grid, m, 1.0, 0.0)
    assert np.max(rel_err(ak, an)) < 1e-13 and np.max(np.abs(pk - pn) / np.abs(pn)) < 1e-14


def test_k1_tree_guard_and_convergence_to_direct_sum():
    w = W.make("plummer4096")
    eps = 0.05
    ref, rphi = oracle.direct(w.pos, w.mass, 1.0, eps, soft="k1")
    errs = []
    for tol in (1e-3, 1e-5, 1e-7):
        t = oracle.Tree(w.pos, w.mass)
        t.softening("k1", eps)
        t.moments(6)
        t.traverse(tol)
        a, ph = t.force(1.0, eps)
        errs.append(np.sqrt(np.mean(rel_err(a, ref) ** 2)))
        # every accepted cell keeps all its sources at least eps from every sink of the group
        L = t.lists()
        cl = t.cells()
        gr = t.groups()
        mo = t.get_moments()
        om, cells = L["m2p"]
        for g in range(len(gr["cell"])):
            cs = cells[om[g]:om[g + 1]]
            d = np.linalg.norm(mo["com"][cs] - gr["centre"][g], axis=1) - gr["dmax"][g]
            assert np.all(d >= mo["bmax"][cs] + eps)
        with pytest.raises(ValueError):
            t.force(1.0, 2 * eps)  # K1 lists are built for one eps
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6  # rms relative, at an absolute tolerance of 1e-7


def test_k1_direct_grad_against_finite_differences():
    rng = np.random.default_rng(8)
    n, eps = 40, 0.4
    pos = rng.uniform(-1, 1, (n, 3))
    mass = rng.uniform(0.5, 1.5, n)
    w = rng.standard_normal((n, 3))
    v = rng.standard_normal(n)

    def L(p, m):
        a, ph = oracle.direct(p, m, 1.0, eps, soft="k1")
        return float((w * a).sum() + (v * ph).sum())

    gx, gm = oracle.direct_grad(pos, mass, w, v, 1.0, eps, soft="k1")
    h = 1e-6
    for k in (0, 7, 19, 33):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[k, d] += h
            pm[k, d] -= h
            fd = (L(pp, mass) - L(pm, mass)) / (2 * h)
            assert abs(gx[k, d] - fd) <= 1e-7 * max(1.0, abs(fd))
        mp, mm = mass.copy(), mass.copy()
        mp[k] += h
        mm[k] -= h
        fd = (L(pos, mp) - L(pos, mm)) / (2 * h)
        assert abs(gm[k] - fd) <= 1e-7 * max(1.0, abs(fd))


def test_k1_frozen_force_is_tree_force():
    w = W.make("plummer4096")
    t = oracle.Tree(w.pos, w.mass)
    t.softening("k1", 0.05)
    t.moments(4)
    t.traverse(1e-4)
    a, ph = t.force(1.0, 0.05)
    fa, fph = t.frozen_force(w.pos, w.mass, 1.0, 0.05)
    assert np.max(rel_err(fa, a)) < 1e-12 and np.max(np.abs(fph - ph) / np.abs(ph)) < 1e-12


# --------------------------------------------------------------------------
# Cubic spline kernel (Sec. "Force Smoothing" cites it, Springel 2005, without a formula):
# the unit-mass kernel of support eps with density 8/(pi eps^3) w(x), w = 1 - 6x^2 + 6x^3
# for x < 1/2 and 2(1 - x)^3 for 1/2 <= x < 1.  As for K1, the pins derive the pair terms
# from that density by quadrature, independent of the oracle's closed forms.
# --------------------------------------------------------------------------

def _spline_density(r, eps):
    x = r / eps
    if x < 0.5:
        return 8.0 / (math.pi * eps ** 3) * (1 - 6 * x * x + 6 * x ** 3)
    return 8.0 / (math.pi * eps ** 3) * 2 * (1 - x) ** 3 if x < 1 else 0.0


@pytest.mark.parametrize("xr", [0.0, 0.05, 0.3, 0.4999, 0.5, 0.5001, 0.7453, 0.9, 0.999, 1.0, 1.2, 3.0])
def test_spline_pair_force_and_potential_from_density(xr):
    from scipy.integrate import quad
    eps = 0.37
    assert abs(quad(lambda r: 4 * math.pi * r * r * _spline_density(r, eps), 0, eps, points=[eps / 2])[0] - 1) < 1e-13
    r = xr * eps
    f, f2, psi = oracle.soft_kernel("spline", eps, r)

    def Mof(t):
        return quad(lambda q: 4 * math.pi * q * q * _spline_density(q, eps), 0, min(t, eps), points=[eps / 2])[0]
    if r > 0:
        assert abs(f - Mof(r) / r ** 3) <= 1e-12 * abs(f)
        tail = quad(lambda t: Mof(t) / (t * t), r, eps, points=[eps / 2])[0] if r < eps else 0.0
        psi_ref = 1.0 / eps + tail if r < eps else 1.0 / r
        assert abs(psi - psi_ref) <= 1e-11 * psi_ref
        h = 1e-6 * r * r
        fp = oracle.soft_kernel("spline", eps, math.sqrt(r * r + h))[0]
        fm = oracle.soft_kernel("spline", eps, math.sqrt(r * r - h))[0]
        assert abs(f2 - 2 * (fp - fm) / (2 * h)) <= 1e-6 * abs(f2)
    else:
        # the centre: f = (4/3) pi rho(0) / (unit mass) = 32/3 eps^-3, psi = 14/(5 eps)
        assert abs(f - 32.0 / 3.0 / eps ** 3) <= 1e-14 * f
        assert abs(psi - 14.0 / (5.0 * eps)) <= 1e-14 * psi
    if xr >= 1.0:
        assert f == pytest.approx(1.0 / r ** 3, rel=1e-15) and psi == pytest.approx(1.0 / r, rel=1e-15)


def test_spline_force_never_exceeds_newtonian_and_is_continuous():
    """A positive density: the force is below the Newtonian one inside the support (no
    compensation, unlike K1) and the force, its slope and the potential are continuous at
    x = 1/2 and at the edge."""
    eps = 0.37
    for x in (0.1, 0.3, 0.5, 0.8, 0.97):
        f = oracle.soft_kernel("spline", eps, x * eps)[0]
        assert f * (x * eps) ** 3 < 1.0
    for x0 in (0.5, 1.0):
        lo = oracle.soft_kernel("spline", eps, eps * x0 * (1 - 1e-12))
        hi = oracle.soft_kernel("spline", eps, eps * x0 * (1 + 1e-12))
        for k in range(3):
            assert abs(lo[k] - hi[k]) <= 1e-8 * abs(hi[k])


def test_spline_direct_sum_tree_and_gradient():
    """Third law; the unsoftened sum when every pair is farther than eps; the tree with the
    compact-support guard converging to the spline direct sum; the analytic gradient
    against central differences."""
    rng = np.random.default_rng(32)
    pos = rng.uniform(-1, 1, (300, 3))
    mass = rng.uniform(0.5, 1.5, 300)
    acc, _ = oracle.direct(pos, mass, 1.0, 0.3, soft="spline")
    assert np.linalg.norm((mass[:, None] * acc).sum(0)) < 1e-12 * np.abs(mass[:, None] * acc).sum()
    grid = np.stack(np.meshgrid(*[np.arange(4.0)] * 3, indexing="ij"), -1).reshape(-1, 3)
    ak, _ = oracle.direct(grid, np.ones(len(grid)), 1.0, 0.9, soft="spline")
    an, _ = oracle.direct(grid, np.ones(len(grid)), 1.0, 0.0)
    assert np.max(rel_err(ak, an)) < 1e-13
    w = W.make("plummer4096")
    eps = 0.05
    ref, _ = oracle.direct(w.pos, w.mass, 1.0, eps, soft="spline")
    errs = []
    for tol in (1e-3, 1e-5, 1e-7):
        t = oracle.Tree(w.pos, w.mass)
        t.softening("spline", eps)
        t.moments(6)
        t.traverse(tol)
        a, _ = t.force(1.0, eps)
        errs.append(np.sqrt(np.mean(rel_err(a, ref) ** 2)))
        L = t.lists()
        gr, mo = t.groups(), t.get_moments()
        om, cells = L["m2p"]
        for g in range(len(gr["cell"])):
            cs = cells[om[g]:om[g + 1]]
            d = np.linalg.norm(mo["com"][cs] - gr["centre"][g], axis=1) - gr["dmax"][g]
            assert np.all(d >= mo["bmax"][cs] + eps)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-6
    n = 40
    p0, m0 = rng.uniform(-1, 1, (n, 3)), rng.uniform(0.5, 1.5, n)
    wt, v = rng.standard_normal((n, 3)), rng.standard_normal(n)

    def loss(p, m):
        a, ph = oracle.direct(p, m, 1.0, 0.4, soft="spline")
        return float((wt * a).sum() + (v * ph).sum())
    gx, gm = oracle.direct_grad(p0, m0, wt, v, 1.0, 0.4, soft="spline")
    h = 1e-6
    for k in (0, 7, 19, 33):
        for d in range(3):
            pp, pm = p0.copy(), p0.copy()
            pp[k, d] += h
            pm[k, d] -= h
            assert abs(gx[k, d] - (loss(pp, m0) - loss(pm, m0)) / (2 * h)) <= 1e-7 * max(1.0, abs(gx[k, d]))
        mp, mm = m0.copy(), m0.copy()
        mp[k] += h
        mm[k] -= h
        assert abs(gm[k] - (loss(p0, mp) - loss(p0, mm)) / (2 * h)) <= 1e-7 * max(1.0, abs(gm[k]))


# --------------------------------------------------------------------------
# Per-interaction order selection (Sec. "Multipole Error Bounds": the bounds choose
# between expansion orders and refinement).  Reading: among the orders p_lo..p, an
# accepted cell is evaluated at the lowest order whose bound meets the tolerance.
# --------------------------------------------------------------------------

def _ordered_tree(pos, mass, p, p_lo, tol):
    t = oracle.Tree(pos, mass)
    t.moments(p)
    t.order_range(p_lo)
    t.traverse(tol)
    return t


def test_order_selection_takes_the_lowest_order_meeting_the_bound():
    """Brute force: B_n recomputed from each cell's particles; every M2P entry's order q
    meets the bound and order q - 1 (if allowed) does not."""
    w = W.make("plummer4096")
    p, p_lo, tol = 8, 1, 1e-5
    t = _ordered_tree(w.pos, w.mass, p, p_lo, tol)
    L = t.lists()
    cl, gr, mo = t.cells(), t.groups(), t.get_moments()
    _, perm = t.keys()
    sp = w.pos[perm]
    sm = w.mass[perm]
    om, cells = L["m2p"]
    orders = L["m2p_order"]
    assert orders.min() >= p_lo and orders.max() <= p and len(set(orders.tolist())) > 2
    Bcache = {}
    checked = 0
    for g in range(0, len(gr["cell"]), 7):
        for e in range(om[g], om[g + 1]):
            c, q = cells[e], orders[e]
            if c not in Bcache:
                b0, n0 = cl["begin"][c], cl["count"][c]
                r = np.linalg.norm(sp[b0:b0 + n0] - mo["com"][c], axis=1)
                Bcache[c] = [float(np.sum(sm[b0:b0 + n0] * r ** k)) for k in range(p + 3)]
            Bn = Bcache[c]
            d = np.linalg.norm(mo["com"][c] - gr["centre"][g]) - gr["dmax"][g]
            b = mo["bmax"][c]
            assert oracle.mac_bound(d, b, Bn[q + 1], Bn[q + 2], q) <= tol * (1 + 1e-9)
            if q > p_lo:
                assert oracle.mac_bound(d, b, Bn[q], Bn[q + 1], q - 1) > tol * (1 - 1e-9)
            checked += 1
    assert checked > 1000


def test_order_selection_keeps_the_per_interaction_bound():
    """Unsoftened: every accepted interaction still errs by at most tol at its order."""
    rng = np.random.default_rng(2)
    n = 3000
    pos = np.concatenate([rng.standard_normal((n // 2, 3)) * 0.1, rng.uniform(-1, 1, (n - n // 2, 3))])
    mass = np.full(n, 1.0 / n)
    ad, _ = oracle.direct(pos, mass, 1.0, 0.0)
    for p, p_lo, tol in ((6, 0, 1e-5), (8, 2, 1e-6)):
        t = _ordered_tree(pos, mass, p, p_lo, tol)
        at, _ = t.force(1.0, 0.0)
        L = t.lists()
        nm = np.diff(L["m2p"][0])
        g, cl = t.groups(), t.cells()
        _, perm = t.keys()
        bound = np.zeros(n)
        for gi, c in enumerate(g["cell"]):
            b, cnt = cl["begin"][c], cl["count"][c]
            bound[perm[b:b + cnt]] = tol * nm[gi]
        err = np.linalg.norm(at - ad, axis=1)
        assert np.all(err <= bound * (1 + 1e-9) + 1e-13)


def test_order_selection_degenerate_range_is_the_fixed_order():
    w = W.make("plummer4096")
    t0 = oracle.Tree(w.pos, w.mass)
    t0.moments(6)
    t0.traverse(1e-5)
    a0, p0 = t0.force(1.0, w.eps)
    t1 = _ordered_tree(w.pos, w.mass, 6, 6, 1e-5)
    a1, p1 = t1.force(1.0, w.eps)
    L0, L1 = t0.lists(), t1.lists()
    assert np.array_equal(L0["m2p"][1], L1["m2p"][1]) and np.array_equal(L0["p2p"][1], L1["p2p"][1])
    assert np.all(L1["m2p_order"] == 6)
    assert np.max(rel_err(a1, a0)) < 1e-15 and np.max(np.abs(p1 - p0) / np.abs(p0)) < 1e-15


def test_order_selection_lowers_the_cost_within_the_tolerance():
    """Each accepted interaction now spends its error budget (E_q just under tol) where
    the fixed order 8 stays far below it, so the error grows while the cost falls; the
    per-interaction bound (the previous test) is what the tolerance promises."""
    w = W.make("plummer4096")
    ref, _ = oracle.direct(w.pos, w.mass, 1.0, w.eps)
    conv = [32, 40, 82, 164, 307, 534, 874, 1358, 2023]  # flops of one M2P per order
    res = {}
    for p_lo in (None, 0):
        t = oracle.Tree(w.pos, w.mass)
        t.moments(8)
        t.order_range(p_lo)
        t.traverse(1e-5)
        a, _ = t.force(1.0, w.eps)
        L = t.lists()
        ns = t.cells()["count"][t.groups()["cell"]]
        per_group = np.add.reduceat(np.array([conv[q] for q in L["m2p_order"]] + [0]),
                                    np.minimum(L["m2p"][0][:-1], len(L["m2p_order"])))[:len(ns)]
        per_group[np.diff(L["m2p"][0]) == 0] = 0
        res[p_lo] = (float(np.sum(per_group * ns)), np.sqrt(np.mean(rel_err(a, ref) ** 2)))
    cost_fixed, err_fixed = res[None]
    cost_var, err_var = res[0]
    assert cost_var < 0.8 * cost_fixed, (cost_var / cost_fixed)
    assert err_fixed < err_var < 1e-4, (err_fixed, err_var)


# --------------------------------------------------------------------------
# Periodic boundaries (Sec. "Boundary Conditions"): the lattice-sum method -- images
# within ws = 2 directly, all farther ones through a local expansion with lattice-summed
# coefficients -- against Ewald summation (neutralising background, tin-foil boundary).
# --------------------------------------------------------------------------

def test_ewald_wigner_constant_and_invariances():
    from oracle import periodic as PR
    L = 1.7
    # one particle: psi_self L is the simple-cubic Wigner constant -2.837297479...
    _, p = PR.ewald(np.array([[0.3, 0.2, 1.1]]), np.array([1.0]), L)
    assert abs(-p[0] * L - (-2.837297479480620)) < 1e-9
    rng = np.random.default_rng(4)
    x = rng.uniform(0, L, (48, 3))
    m = rng.uniform(0.5, 1.5, 48)
    a1, p1 = PR.ewald(x, m, L)
    a2, p2 = PR.ewald(x, m, L, alpha=4.5 / L, kmax=16)        # the splitting does not matter
    assert np.max(np.abs(a1 - a2)) < 1e-12 * np.max(np.abs(a1))
    assert np.max(np.abs(p1 - p2)) < 1e-12 * np.max(np.abs(p1))
    assert np.max(np.abs((m[:, None] * a1).sum(0))) < 1e-12 * np.abs(m[:, None] * a1).sum()
    a3, p3 = PR.ewald(np.mod(x + np.array([0.4, -1.3, 0.77]), L), m, L)   # translation
    assert np.max(np.abs(a3 - a1)) < 1e-11 * np.max(np.abs(a1))
    assert np.max(np.abs(p3 - p1)) < 1e-11 * np.max(np.abs(p1))


def test_lattice_coefficients_laplace_symmetry_and_direct_sums():
    from oracle import periodic as PR
    L = 1.3
    V = L ** 3
    D = PR.lattice_coefficients(L, 17, ws=2)
    even = {n: max(abs(D[g]) for g in D if sum(g) == n) for n in range(0, 18, 2)}
    # odd orders vanish by symmetry: their scale is that of the neighbouring even orders
    scale = {n: even[n] if n % 2 == 0 else max(even[n - 1], even.get(n + 1, 0.0)) for n in range(18)}
    # the far part is harmonic apart from the background: lap psi_far(0) = 4 pi / V, and
    # every derivative of it is harmonic
    for g in D:
        if sum(g) > 15:
            continue
        lap = D[(g[0] + 2, g[1], g[2])] + D[(g[0], g[1] + 2, g[2])] + D[(g[0], g[1], g[2] + 2)]
        ref = 4 * math.pi / V if sum(g) == 0 else 0.0
        assert abs(lap - ref) <= 1e-8 * scale[sum(g) + 2], g
    # cubic symmetry: odd orders vanish, permutations agree
    for g in D:
        n = sum(g)
        if n % 2 == 1:
            assert abs(D[g]) <= 1e-9 * scale[n]
        else:
            for h in ((g[1], g[0], g[2]), (g[2], g[1], g[0]), (g[0], g[2], g[1])):
                assert abs(D[g] - D[h]) <= 1e-9 * scale[n]
    assert abs(D[(2, 0, 0)] - 4 * math.pi / (3 * V)) < 1e-13 * D[(2, 0, 0)]
    # from order 10 on the lattice sum of derivatives of 1/r converges absolutely and fast:
    # the direct sum over the images beyond ws agrees
    n = PR._images(24)
    n = n[np.max(np.abs(n), axis=1) > 2]
    R = n * L
    u = np.sum(R * R, axis=1)
    F = np.array([(-0.5) ** k * PR._dfact(2 * k - 1) * u ** (-(2 * k + 1) / 2) for k in range(17)])
    Dd = PR._radial_derivs(F, R, 16)
    for g in Dd:
        if sum(g) in (12, 16) and sum(g) % 2 == 0:
            assert abs(D[g] - Dd[g]) <= 1e-8 * scale[sum(g)], g


def test_lattice_method_matches_ewald_and_converges_with_order():
    """Images within ws = 2 by direct summation plus the far images through the local
    expansion of order p: the Ewald result to single-precision accuracy at p = 8 (the
    paper's "one part in 1e7"), the error falling with p."""
    from oracle import periodic as PR
    L = 1.0
    rng = np.random.default_rng(9)
    x = rng.uniform(0, L, (64, 3))
    m = rng.uniform(0.5, 1.5, 64)
    ra, rp = PR.ewald(x, m, L)
    an, pn = PR.near_images_direct(x, m, L)
    D = PR.lattice_coefficients(L, 17)
    errs = []
    for p in (2, 4, 6, 8):
        af, pf = PR.far_field(x, m, L, (0.0, 0.0, 0.0), p=p, D=D)
        errs.append(np.max(rel_err(an + af, ra)))
        if p == 8:
            assert np.max(np.abs(pn + pf - rp) / np.abs(rp)) < 1e-5
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 5e-7


def _periodic_case(n=600, L=1.0, seed=9):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, L, (n, 3)), rng.uniform(0.5, 1.5, n) / n, L


def test_periodic_tree_near_field_is_the_image_sum():
    """With every interaction P2P, the periodic tree (central cube and its images within
    ws = 2) is the plain sum over those images; image indices name real shifts."""
    from oracle import periodic as PR
    x, m, L = _periodic_case()
    an, pn = PR.near_images_direct(x, m, L)
    t = oracle.Tree(x, m, 16, 32)
    t.periodic(L, 2)
    t.moments(4)
    t.traverse(1e-300)
    a, p = t.force(1.0, 0.0)
    assert np.max(rel_err(a, an)) < 1e-12 and np.max(np.abs(p - pn) / np.abs(pn)) < 1e-12
    Ls = t.lists()
    assert Ls["p2p_image"].min() >= 0 and Ls["p2p_image"].max() <= 124
    assert len(set(Ls["p2p_image"].tolist())) == 125


def test_periodic_tree_converges_to_ewald():
    from oracle import periodic as PR
    x, m, L = _periodic_case()
    ra, _ = PR.ewald(x, m, L)
    D = PR.lattice_coefficients(L, 17)
    errs = []
    for tol in (1e-4, 1e-6, 1e-8):
        a, _ = PR.tree_force(x, m, L, (0.0, 0.0, 0.0), p=8, tol=tol, D=D, leaf_max=16, group_max=32)
        errs.append(np.sqrt(np.mean(rel_err(a, ra) ** 2)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-7


def test_periodic_tree_force_is_lattice_translation_invariant():
    """Moving every particle and the cube by a lattice vector changes nothing; a shift
    with wrap-around changes the tree but not the periodic force beyond the method's
    accuracy (p = 8, tol 1e-8: each within 2e-7 rms of Ewald, which the shift leaves
    unchanged)."""
    from oracle import periodic as PR
    rng = np.random.default_rng(19)
    n, L = 200, 1.0
    x = rng.uniform(0, L, (n, 3))
    m = rng.uniform(0.5, 1.5, n) / n
    D = PR.lattice_coefficients(L, 17)
    a0, p0 = PR.tree_force(x, m, L, (0.0, 0.0, 0.0), p=8, tol=1e-8, D=D, leaf_max=16, group_max=32)
    a1, p1 = PR.tree_force(x + [L, -L, 2 * L], m, L, (L, -L, 2 * L), p=8, tol=1e-8, D=D, leaf_max=16,
                           group_max=32)
    assert np.max(rel_err(a1, a0)) < 1e-9 and np.max(np.abs(p1 - p0)) < 1e-9 * np.sqrt(np.mean(p0 ** 2))
    s = np.array([0.37, 0.81, 0.05])
    a2, _ = PR.tree_force(np.mod(x + s, L), m, L, (0.0, 0.0, 0.0), p=8, tol=1e-8, D=D, leaf_max=16, group_max=32)
    ra, _ = PR.ewald(x, m, L)
    rs, _ = PR.ewald(np.mod(x + s, L), m, L)
    assert np.max(rel_err(rs, ra)) < 1e-10
    assert np.sqrt(np.mean(rel_err(a0, ra) ** 2)) < 2e-7 and np.sqrt(np.mean(rel_err(a2, ra) ** 2)) < 2e-7
