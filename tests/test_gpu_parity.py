"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact: frame, keys, sort order, tree topology, sink groups and their centres.
Floating point: moments and acceptance aggregates to ~1e-12 relative; interaction
lists equal as sets (borderline acceptance decisions excepted); forces within the
stated tolerances (FP64 path 1e-11, mixed path rms 1e-5 / max 1e-3 relative).
"""
import numpy as np
import pytest

import oracle
from paper_1310_4502_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_4502_gb300 import hot


def dev():
    return torch.device("cuda:0")


def cases():
    rng = np.random.default_rng(21)
    out = {}
    w = W.make("plummer4096")
    out["plummer4096"] = (w.pos, w.mass, w.eps)
    out["plummer_eps0"] = (w.pos, w.mass, 0.0)  # unsoftened: every pair takes the tested path
    n = 1 << 15
    out["clustered32k"] = (W.clustered(n, seed=3), np.full(n, 1.0 / n), 1e-4)
    n = 20011  # ragged: not a multiple of any tile
    x = rng.uniform(-1, 1, (n, 3))
    x[100:140] = x[99]  # 41 coincident particles -> a level-21 leaf
    out["ragged_dup"] = (x, rng.uniform(0.5, 1.5, n) / n, 0.01)
    out["tiny7"] = (rng.standard_normal((7, 3)), np.full(7, 1.0), 0.0)
    out["one"] = (np.array([[0.3, -0.2, 0.1]]), np.array([2.0]), 0.1)
    return out


CASES = cases()


def build(pos, mass, **kw):
    h = hot.Hot(**kw)
    P = torch.tensor(pos, device=dev())
    M = torch.tensor(mass, device=dev())
    h.build_tree(P, M)
    return h, P, M


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("leaf_max,group_max", [(64, 128), (16, 64), (1, 8)])
def test_keys_sort_topology_groups_bit_exact(name, leaf_max, group_max):
    pos, mass, eps = CASES[name]
    h, _, _ = build(pos, mass, leaf_max=leaf_max, group_max=group_max)
    t = oracle.Tree(pos, mass, leaf_max, group_max)
    lo, L = t.frame()
    fr = h.debug_get("FRAME")
    assert np.array_equal(fr[:3], lo) and fr[3] == L
    k, perm = t.keys()
    assert np.array_equal(h.debug_get("SORTED_KEYS"), k[perm])
    assert np.array_equal(h.debug_get("PERM").astype(np.int64), perm)
    cl = t.cells()
    assert h.sizes()["ncell"] == len(cl["key"])
    assert np.array_equal(h.debug_get("CELL_KEY"), cl["key"])
    assert np.array_equal(h.debug_get("CELL_LEVEL"), cl["level"])
    assert np.array_equal(h.debug_get("CELL_BEGIN").astype(np.int64), cl["begin"])
    assert np.array_equal(h.debug_get("CELL_COUNT").astype(np.int64), cl["count"])
    assert np.array_equal(h.debug_get("CELL_PARENT"), cl["parent"])
    assert np.array_equal(h.debug_get("CELL_NCHILD"), cl["nchild"])
    g = t.groups()
    assert np.array_equal(h.debug_get("GROUP_CELL"), g["cell"])
    assert np.array_equal(h.debug_get("GROUP_CENTRE"), g["centre"])
    assert np.array_equal(h.debug_get("GROUP_DMAX"), g["dmax"])


@pytest.mark.parametrize("name", ["plummer4096", "ragged_dup"])
def test_hash_lookup(name):
    pos, mass, _ = CASES[name]
    h, _, _ = build(pos, mass)
    keys = h.debug_get("CELL_KEY")
    idx = h.lookup(keys)
    assert np.array_equal(idx, np.arange(len(keys), dtype=np.int32))
    absent = (keys[1:] << np.uint64(3)) | np.uint64(7)
    present = set(keys.tolist())
    absent = np.array([a for a in absent.tolist() if a not in present][:1000], dtype=np.uint64)
    assert np.all(h.lookup(absent) == -1)


@pytest.mark.parametrize("p", [0, 1, 4, 6, 8])
@pytest.mark.parametrize("prec,mtol", [("fp64", 1e-10), ("mixed", 3e-6)])
def test_moments(p, prec, mtol):
    """Moments against the oracle's direct sums, relative to m b_max^|a|: float64
    throughout on the FP64 path; leaf sums in float32 on the mixed path (then exact
    float64 translation), hence the float32-level bound there.  Masses, centres and the
    acceptance aggregates are float64 on both paths."""
    pos, mass, eps = CASES["plummer4096"]
    h, _, _ = build(pos, mass, p=p, precision=prec)
    h.compute_moments(p)
    t = oracle.Tree(pos, mass)  # the default leaf and group sizes on both sides
    t.moments(p)
    mo = t.get_moments()
    np.testing.assert_allclose(h.debug_get("CELL_MASS"), mo["mass"], rtol=1e-13)
    scale_x = np.max(np.abs(pos))
    np.testing.assert_allclose(h.debug_get("CELL_COM"), mo["com"], rtol=0, atol=1e-13 * scale_x)
    M = h.debug_get("MOMENTS")
    bm = mo["bmax"]
    idx = oracle.multi_indices(p)
    deg = np.array([sum(a) for a in idx])
    scale = mo["mass"][:, None] * np.maximum(bm, 1e-300)[:, None] ** deg[None, :] + 1e-300
    assert np.max(np.abs(M - mo["mom"]) / scale) < mtol
    np.testing.assert_allclose(h.debug_get("CELL_BMAX"), bm, rtol=1e-11, atol=1e-14 * scale_x)
    np.testing.assert_allclose(h.debug_get("CELL_B1"), mo["B1"], rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(h.debug_get("CELL_B2"), mo["B2"], rtol=1e-10, atol=1e-300)


def lists_match(h, t, cl):
    """Per group, the GPU lists equal the oracle's as sets, up to borderline decisions
    (cells within 1e-9 of a threshold, and their descendants)."""
    L = t.lists()
    om, cm = L["m2p"]
    op, cp = L["p2p"]
    ob, cb = L["border"]
    gm_off = h.debug_get("M2P_OFFSETS")
    gm = h.debug_get("M2P_CELLS")
    gp_off = h.debug_get("P2P_OFFSETS")
    gp = h.debug_get("P2P_CELLS")
    keys = cl["key"]
    level = cl["level"]
    bad = 0
    for g in range(len(om) - 1):
        a = set(cm[om[g]:om[g + 1]].tolist()) ^ set(gm[gm_off[g]:gm_off[g + 1]].tolist())
        b = set(cp[op[g]:op[g + 1]].tolist()) ^ set(gp[gp_off[g]:gp_off[g + 1]].tolist())
        diff = a | b
        if not diff:
            continue
        border = cb[ob[g]:ob[g + 1]]
        for c in diff:
            ok = any(level[c] >= level[x] and (int(keys[c]) >> (3 * (level[c] - level[x]))) == int(keys[x])
                     for x in border)
            bad += 0 if ok else 1
    return bad


@pytest.mark.parametrize("name", ["plummer4096", "plummer_eps0", "clustered32k", "ragged_dup", "tiny7", "one"])
@pytest.mark.parametrize("p", [1, 4, 6])
def test_lists_and_forces(name, p):
    pos, mass, eps = CASES[name]
    tol = 1e-4 if name != "ragged_dup" else 1e-5
    t = oracle.Tree(pos, mass)  # the default leaf and group sizes on both sides
    t.moments(p)
    t.traverse(tol)
    ra, rp = t.force(1.0, eps)
    cl = t.cells()
    for prec in ("fp64", "mixed"):
        h, P, M = build(pos, mass, p=p, tol=tol, eps=eps, precision=prec)
        h.compute_moments(p)
        h.traverse(tol)
        assert lists_match(h, t, cl) == 0
        acc = torch.empty_like(P)
        pot = torch.empty_like(M)
        h.evaluate_forces(acc, pot)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        ph = pot.cpu().numpy()
        if len(mass) == 1:
            assert np.all(a == 0) and np.all(ph == 0)
            continue
        na = np.linalg.norm(ra, axis=1)
        rel = np.linalg.norm(a - ra, axis=1) / na
        prel = np.abs(ph - rp) / np.abs(rp)
        if prec == "fp64":
            assert rel.max() < 1e-11, rel.max()
            assert prel.max() < 1e-11, prel.max()
        else:
            assert np.sqrt(np.mean(rel ** 2)) < 1e-5, np.sqrt(np.mean(rel ** 2))
            assert rel.max() < 1e-3, rel.max()
            assert prel.max() < 1e-4, prel.max()


@pytest.mark.parametrize("name", ["plummer4096", "clustered32k", "ragged_dup"])
def test_lists_and_forces_order8(name):
    """p = 8, the paper's highest order: lists and forces against the oracle (same
    tolerances as the lower orders)."""
    test_lists_and_forces(name, 8)


def test_adjoint_refuses_orders_above_6():
    pos, mass, eps = CASES["plummer4096"]
    h, P, M = build(pos, mass, p=8, tol=1e-4, eps=eps)
    h.compute_moments(8)
    h.traverse(1e-4)
    acc = torch.empty_like(P)
    h.evaluate_forces(acc)
    with pytest.raises(hot.HotError) as e:
        h.adjoint(torch.ones_like(P), None, torch.empty_like(P), torch.empty_like(M))
    assert e.value.code == hot.HOT_EINVAL


def test_call_order_and_bad_arguments():
    pos, mass, _ = CASES["tiny7"]
    h = hot.Hot()
    acc = torch.empty((7, 3), dtype=torch.float64, device=dev())
    with pytest.raises(hot.HotError) as e:
        h.evaluate_forces(acc)
    assert e.value.code == hot.HOT_ESTATE
    with pytest.raises(hot.HotError) as e:
        h.compute_moments(4)
    assert e.value.code == hot.HOT_ESTATE
    P = torch.tensor(pos, device=dev())
    M = torch.tensor(mass, device=dev())
    bad = P.clone()
    bad[3, 1] = float("nan")
    with pytest.raises(hot.HotError) as e:
        h.build_tree(bad, M)
    assert e.value.code == hot.HOT_EINPUT
    with pytest.raises(hot.HotError) as e:
        h.build_tree(P, -M)
    assert e.value.code == hot.HOT_EINPUT
    h.build_tree(P, M)
    with pytest.raises(hot.HotError) as e:
        h.compute_moments(9)
    assert e.value.code == hot.HOT_EINVAL
    h.compute_moments(4)
    with pytest.raises(hot.HotError) as e:
        h.traverse(0.0)
    assert e.value.code == hot.HOT_EINVAL


K1_CASES = {
    # support 0.05 in a unit-scale Plummer sphere: a large share of the P2P pairs inside it
    "plummer4096_k1": lambda: (W.make("plummer4096").pos, W.make("plummer4096").mass, 0.05),
    "clustered32k_k1": lambda: (CASES["clustered32k"][0], CASES["clustered32k"][1], 2e-3),
    "ragged_dup_k1": lambda: (CASES["ragged_dup"][0], CASES["ragged_dup"][1], 0.02),
}


@pytest.mark.parametrize("soft", ["k1", "spline"])
@pytest.mark.parametrize("name", list(K1_CASES))
@pytest.mark.parametrize("p", [4, 6])
def test_compact_lists_and_forces(name, p, soft):
    """Kernels of compact support (K1 compensating smoothing, the cubic spline): the lists
    (with the d >= b_max + eps guard) and the forces against the oracle's tree with the
    same kernel, at the tolerances of the Plummer parity test."""
    pos, mass, eps = K1_CASES[name]()
    tol = 1e-4
    t = oracle.Tree(pos, mass)
    t.softening(soft, eps)
    t.moments(p)
    t.traverse(tol)
    ra, rp = t.force(1.0, eps)
    cl = t.cells()
    for prec in ("fp64", "mixed"):
        h, P, M = build(pos, mass, p=p, tol=tol, eps=eps, precision=prec, softening=soft)
        h.compute_moments(p)
        h.traverse(tol)
        assert lists_match(h, t, cl) == 0
        acc = torch.empty_like(P)
        pot = torch.empty_like(M)
        h.evaluate_forces(acc, pot)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        ph = pot.cpu().numpy()
        rel = np.linalg.norm(a - ra, axis=1) / np.linalg.norm(ra, axis=1)
        prel = np.abs(ph - rp) / np.abs(rp)
        if prec == "fp64":
            assert rel.max() < 1e-11, rel.max()
            assert prel.max() < 1e-11, prel.max()
        else:
            assert np.sqrt(np.mean(rel ** 2)) < 1e-5, np.sqrt(np.mean(rel ** 2))
            assert rel.max() < 1e-3, rel.max()
            assert prel.max() < 1e-4, prel.max()


@pytest.mark.parametrize("soft", ["k1", "spline"])
@pytest.mark.parametrize("prec,bound", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_compact_pair_functions(soft, prec, bound):
    """The device pair functions against the oracle's at 400 separations from 0 to 1.5 eps
    (both branches of the spline, the edge, the Newtonian range): a unit mass at the origin
    and massless-in-effect probes (mass 1e-30) around it, one group, every interaction P2P,
    so each probe's acceleration is f(r) d and its potential -psi(r) to within 1e-30."""
    eps = 0.01
    n = 400
    rng = np.random.default_rng(17)
    r = np.linspace(0.0, 1.5 * eps, n + 1)[1:]
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pos = np.concatenate([np.zeros((1, 3)), r[:, None] * d])
    mass = np.concatenate([[1.0], np.full(n, 1e-30)])
    h = hot.Hot(p=4, tol=1e-4, eps=eps, precision=prec, softening=soft, group_max=512, leaf_max=512)
    P = torch.tensor(pos, device=dev())
    M = torch.tensor(mass, device=dev())
    acc = torch.empty_like(P)
    pot = torch.empty_like(M)
    h.force(P, M, acc, pot)
    torch.cuda.synchronize()
    a = acc.cpu().numpy()[1:]
    ph = pot.cpu().numpy()[1:]
    ref = np.array([oracle.soft_kernel(soft, eps, x) for x in r])
    f_ref, psi_ref = ref[:, 0], ref[:, 2]
    # a = f(r) (0 - x) = -f(r) r d
    f_got = -np.sum(a * d, axis=1) / r
    assert np.max(np.abs(f_got - f_ref) / f_ref) < bound
    assert np.max(np.abs(-ph - psi_ref) / psi_ref) < bound


def test_k1_differs_from_plummer_and_changing_it_recomputes():
    """The smoothing is part of the parameters: switching it on a built tree recomputes
    moments and lists, and the two kernels give different forces at short range."""
    pos, mass, eps = K1_CASES["plummer4096_k1"]()
    h, P, M = build(pos, mass, p=4, tol=1e-4, eps=eps)
    h.compute_moments(4)
    h.traverse(1e-4)
    acc = torch.empty_like(P)
    h.evaluate_forces(acc)
    a_pl = acc.cpu().numpy()
    h.set_params(p=4, tol=1e-4, eps=eps, softening="k1")
    with pytest.raises(hot.HotError) as e:
        h.evaluate_forces(acc)
    assert e.value.code == hot.HOT_ESTATE
    h.compute_moments(4)
    h.traverse(1e-4)
    h.evaluate_forces(acc)
    a_k1 = acc.cpu().numpy()
    ref, _ = oracle.direct(pos, mass, 1.0, eps, soft="k1")
    assert np.max(np.linalg.norm(a_k1 - a_pl, axis=1) / np.linalg.norm(ref, axis=1)) > 1e-2
    assert np.sqrt(np.mean((np.linalg.norm(a_k1 - ref, axis=1) / np.linalg.norm(ref, axis=1)) ** 2)) < 1e-4


@pytest.mark.parametrize("name", ["plummer4096", "clustered32k", "ragged_dup"])
@pytest.mark.parametrize("p,p_min", [(8, 0), (6, 2)])
def test_order_selection_lists_orders_and_forces(name, p, p_min):
    """Per-interaction order selection: the lists, the order of every M2P entry (the
    lowest order in [p_min, p] meeting the bound) and the forces against the oracle."""
    pos, mass, eps = CASES[name]
    tol = 1e-4 if name != "ragged_dup" else 1e-5
    t = oracle.Tree(pos, mass)
    t.moments(p)
    t.order_range(p_min)
    t.traverse(tol)
    ra, rp = t.force(1.0, eps)
    cl = t.cells()
    L = t.lists()
    om, cm = L["m2p"]
    qo = L["m2p_order"]
    ob, cb = L["border"]
    assert len(set(qo.tolist())) > 1
    for prec in ("fp64", "mixed"):
        h, P, M = build(pos, mass, p=p, tol=tol, eps=eps, precision=prec, p_min=p_min)
        h.compute_moments(p)
        h.traverse(tol)
        assert lists_match(h, t, cl) == 0
        goff = h.debug_get("M2P_OFFSETS")
        gcells = h.debug_get("M2P_CELLS")
        gq = h.debug_get("M2P_ORDERS")
        for g in range(len(om) - 1):
            border = set(cb[ob[g]:ob[g + 1]].tolist())
            ref = dict(zip(cm[om[g]:om[g + 1]].tolist(), qo[om[g]:om[g + 1]].tolist()))
            got = dict(zip(gcells[goff[g]:goff[g + 1]].tolist(), gq[goff[g]:goff[g + 1]].tolist()))
            for c in ref.keys() & got.keys():
                assert ref[c] == got[c] or c in border, (g, c, ref[c], got[c])
        acc = torch.empty_like(P)
        pot = torch.empty_like(M)
        h.evaluate_forces(acc, pot)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        ph = pot.cpu().numpy()
        rel = np.linalg.norm(a - ra, axis=1) / np.linalg.norm(ra, axis=1)
        prel = np.abs(ph - rp) / np.abs(rp)
        if prec == "fp64":
            assert rel.max() < 1e-11, rel.max()
            assert prel.max() < 1e-11, prel.max()
        else:
            assert np.sqrt(np.mean(rel ** 2)) < 1e-5, np.sqrt(np.mean(rel ** 2))
            assert rel.max() < 1e-3, rel.max()
            assert prel.max() < 1e-4, prel.max()
        if prec == "mixed":
            with pytest.raises(hot.HotError) as e:
                h.adjoint(torch.ones_like(P), None, torch.empty_like(P), torch.empty_like(M))
            assert e.value.code == hot.HOT_EINVAL


def test_order_range_is_validated():
    with pytest.raises(hot.HotError) as e:
        hot.Hot(p=4, p_min=5)
    assert e.value.code == hot.HOT_EINVAL
    pos, mass, _ = CASES["plummer4096"]
    h, _, _ = build(pos, mass, p=6, p_min=3)
    with pytest.raises(hot.HotError) as e:
        h.compute_moments(2)
    assert e.value.code == hot.HOT_EINVAL
