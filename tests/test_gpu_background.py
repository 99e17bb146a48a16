"""Background subtraction (Sec. "Background Subtraction") on the GPU against the oracle's
tree code on the density contrast (oracle/background.py).

Compared per sink group: the surrounding cube; the interaction lists as sets -- matter
expansions, contrast expansions of cells and of empty octants, particle-particle leaves,
analytic cubes of leaves and of empty octants; the interaction counts; and the forces.
Force tolerances are relative to the magnitudes the sums cancel from, the unsubtracted
field's rms over the sinks (the contrast field is a few per cent of it on the lattices):
the FP64 path to 1e-10 (max), the mixed path to 1e-5 rms / 1e-4 max (float32 cube fields
on float64 corner offsets, float32 expansions).

Inputs: perturbed lattices (amplitude 0.05 spacings) with eight particles of mass 1e-30 at
the unit cube's corners, so that the root cube is the cube the matter fills, at 16^3 (leaf
16, group 32) and 24^3 (the default sizes), and the clustered recipe at N = 2048 (leaf 16,
group 32, S one level up), whose voids give empty octants.
"""
import numpy as np
import pytest

import oracle
from oracle import background as BG
from paper_1310_4502_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_4502_gb300 import hot


def lattice(n, amp, seed):
    rng = np.random.default_rng(seed)
    g = (np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) / n
    x = g + amp / n * rng.standard_normal(g.shape)
    c = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float) * (1 - 1e-12)
    return np.vstack([x, c]), np.concatenate([np.full(len(x), 1.0 / len(x)), np.full(8, 1e-30)])


CASES = {
    "lattice16": lambda: lattice(16, 0.05, 6) + (16, 32, 2, 0.02 / 16),
    "lattice24": lambda: lattice(24, 0.05, 5) + (64, 128, 2, 0.02 / 24),
    "clustered2048": lambda: (W.clustered(2048, seed=1), np.full(2048, 1.0 / 2048), 16, 32, 1, 1e-3),
}
TOL, P = 1e-4, 4
_ref = {}


def reference(name):
    if name not in _ref:
        x, m, lm, gm, up, eps = CASES[name]()
        bt = BG.BackgroundTree(x, m, p=P, leaf_max=lm, group_max=gm, up=up)
        a, ph, cnt = bt.force(TOL, 1.0, eps, record=True)
        full, fullp = oracle.direct(x, m, 1.0, eps)
        _ref[name] = (x, m, lm, gm, up, eps, a, ph, cnt, bt, full, fullp)
    return _ref[name]


def borderline(bt, g, c):
    """Whether the test of leaf c for group g lies at its threshold within rounding: d
    within 1e-12 of b relative to the distances d was formed from (|z - g| and Delta_max),
    or E within 1e-9 of tol, by the oracle's own numbers (the matter test inside the
    surrounding cube, the contrast test outside it).  Such decisions may differ between
    two correct evaluations (a norm rounded differently)."""
    S = bt.surround[g]
    gcen, dmax = bt.gcen[g], bt.gdmax[g]
    if S <= c < bt.cend[S]:
        dist = float(np.linalg.norm(bt.com[c] - gcen))
        d = dist - dmax
        b = bt.bmax[c]
        E = oracle.mac_bound(d, b, bt.B1[c], bt.B2[c], P) if d > b else np.inf
    else:
        dist = float(np.linalg.norm(bt.centre[c] - gcen))
        d = dist - dmax
        b = 0.5 * np.sqrt(3.0) * bt.side[c]
        E = (1.0 / (1.0 - b / d) ** 2 * ((P + 2) * bt.cQ[c][0] / d ** (P + 3) + (P + 3) * bt.cQ[c][1] / d ** (P + 4))
             if d > b else np.inf)
    return abs(d - b) <= 1e-12 * max(dist, dmax) or abs(E / TOL - 1.0) <= 1e-9


def gpu_lists(h):
    """Per group the set of interactions in the oracle's notation."""
    s = h.sizes()
    nc = s["ncell"]
    ep, eo = h.debug_get("BG_EMPTY_PARENT"), h.debug_get("BG_EMPTY_OCTANT")
    mo, mc = h.debug_get("M2P_OFFSETS"), h.debug_get("M2P_CELLS")
    po, pc = h.debug_get("P2P_OFFSETS"), h.debug_get("P2P_CELLS")
    bo, bc = h.debug_get("BG_CUBE_OFFSETS"), h.debug_get("BG_CUBES")
    out = []
    for g in range(s["ngroup"]):
        r = set()
        for e in mc[mo[g]:mo[g + 1]].tolist():
            if e < nc:
                r.add(("m", e))
            elif e < 2 * nc:
                r.add(("c", e - nc))
            else:
                r.add(("e", int(ep[e - 2 * nc]), int(eo[e - 2 * nc])))
        for e in pc[po[g]:po[g + 1]].tolist():
            r.add(("p", e))
        for e in bc[bo[g]:bo[g + 1]].tolist():
            r.add(("b", e) if e < nc else ("be", int(ep[e - nc]), int(eo[e - nc])))
        out.append(r)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_background_lists_counts_and_forces(name):
    x, m, lm, gm, up, eps, ra, rp, cnt, bt, full, fullp = reference(name)
    rl, rS = bt.lists, bt.surround
    dev = torch.device("cuda:0")
    P_ = torch.tensor(x, device=dev)
    M_ = torch.tensor(m, device=dev)
    scale_a = np.sqrt(np.mean(np.sum(full ** 2, 1)))
    scale_p = np.sqrt(np.mean(fullp ** 2))
    for prec in ("fp64", "mixed"):
        h = hot.Hot(p=P, tol=TOL, eps=eps, precision=prec, leaf_max=lm, group_max=gm, background=True, bg_up=up)
        acc = torch.empty_like(P_)
        pot = torch.empty_like(M_)
        h.force(P_, M_, acc, pot)
        h.synchronize()
        assert np.array_equal(h.debug_get("BG_GROUP_S"), rS)
        gl = gpu_lists(h)
        assert len(gl) == len(rl)
        # differences only where a leaf's test sits at its threshold: the same leaf taken
        # whole on one side and particle by particle on the other
        flips = 0
        for g in range(len(gl)):
            d = gl[g] ^ rl[g]
            if not d:
                continue
            leaves = {e[1] for e in d}
            assert all(e[0] in ("m", "c", "p", "b") for e in d), (prec, g, sorted(d))
            assert all(borderline(bt, g, c) for c in leaves), (prec, g, sorted(d))
            flips += 1
        assert flips <= 2, (prec, flips)
        bs = h.bg_sizes()
        if flips == 0:
            assert bs["m2p_contrast"] == cnt["m2p_contrast"] and bs["m2p_empty"] == cnt["m2p_empty"]
            assert bs["m2p_matter"] == cnt["m2p_matter"] and bs["cube_evals"] == cnt["cube_fields"]
        a = acc.cpu().numpy()
        ph = pot.cpu().numpy()
        ea = np.linalg.norm(a - ra, axis=1) / scale_a
        ep = np.abs(ph - rp) / scale_p
        if prec == "fp64":
            assert ea.max() < 1e-10, ea.max()
            assert ep.max() < 1e-10, ep.max()
        else:
            assert np.sqrt(np.mean(ea ** 2)) < 1e-5 and ea.max() < 1e-4, (np.sqrt(np.mean(ea ** 2)), ea.max())
            assert np.sqrt(np.mean(ep ** 2)) < 1e-5 and ep.max() < 1e-4, (np.sqrt(np.mean(ep ** 2)), ep.max())
        h.close()


@pytest.mark.parametrize("up", [0, 2])
def test_background_without_expansions_is_exact(up):
    """At a tolerance that accepts nothing every interaction is a particle pair or an
    analytic cube: the direct sum less the root cube's field (the oracle's closed form)."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (400, 3))
    m = rng.uniform(0.5, 1.5, 400) / 400
    bt = BG.BackgroundTree(x, m, p=4, leaf_max=16, group_max=32, up=up)
    ra, rp = bt.exact()
    dev = torch.device("cuda:0")
    for prec, bound in (("fp64", 1e-11), ("mixed", 2e-5)):
        acc, pot = hot.tree_force(torch.tensor(x, device=dev), torch.tensor(m, device=dev), p=4, tol=1e-300,
                                  precision=prec, leaf_max=16, group_max=32, background=True, bg_up=up)
        a = acc.cpu().numpy()
        assert np.max(np.linalg.norm(a - ra, axis=1)) < bound * np.max(np.linalg.norm(ra, axis=1)), prec
        assert np.max(np.abs(pot.cpu().numpy() - rp)) < bound * np.max(np.abs(rp)), prec


def test_background_refuses_what_it_does_not_cover():
    """Background subtraction takes Plummer smoothing, open boundaries, a fixed order up to
    6, and no adjoint."""
    for kw in ({"softening": "k1"}, {"box": 1.0}, {"p": 8}, {"p_min": 0}, {"bg_up": -1}):
        args = dict(p=4, tol=1e-4, eps=0.01, background=True)
        args.update(kw)
        with pytest.raises(hot.HotError) as e:
            hot.Hot(**args)
        assert e.value.code == hot.HOT_EINVAL
    x, m = lattice(6, 0.05, 1)
    dev = torch.device("cuda:0")
    h = hot.Hot(p=4, tol=1e-4, eps=0.01, background=True)
    P_ = torch.tensor(x, device=dev)
    M_ = torch.tensor(m, device=dev)
    h.force(P_, M_, torch.empty_like(P_))
    with pytest.raises(hot.HotError) as e:
        h.adjoint(torch.zeros_like(P_), None, torch.empty_like(P_), torch.empty_like(M_))
    assert e.value.code == hot.HOT_EINVAL
