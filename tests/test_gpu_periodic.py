"""GPU parity for periodic boundaries (Sec. "Boundary Conditions"): the CUDA path (through
the C ABI) against the oracle's periodic tree code and against Ewald summation.

The tree serves the central cube and its images within ws = 2; the list entries carry
their image, and per group the (cell, image) pairs equal the oracle's as sets, borderline
acceptance decisions excepted.  Forces (the images' interactions plus the far images'
local expansion of order 8) against the oracle's.  The two parts cancel: for a nearly
uniform cube the far acceleration is several times the total and the far potential's
constant ~60 G M / L against a total of ~0.05 G M / L, and a particle's net force can be a
hundredth of its parts.  So the FP64 path is held to 1e-9 of |a| (the open boundaries'
1e-11 loses a digit or two) and the potential to 1e-9 of its rms (a periodic potential
with a neutralising background has zero mean); the mixed path, whose float32 sums work
on the parts, to rms 1e-5 / max 1e-3 of |a_near| + |a_far| (the open boundaries' bounds,
on the magnitudes the arithmetic sees) and its potential to 2e-6 of |phi_near|.  One
more term for coincident particles under Plummer softening: the mixed path rounds
positions to float32 relative to the group centre (a few roundings at 2^-24 of offsets
up to ~L: |delta| <= 2^-21 L), so a pair at zero separation, whose force is exactly 0,
comes out as up to G m delta / eps^3;
each of the ragged case's 11 coincident particles is allowed k G m delta / eps^3 for its
k partners on top of the bound above (the open-boundary path has the same property,
hidden there by the larger net field).
"""
import numpy as np
import pytest

import oracle
from oracle import periodic as PR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_4502_gb300 import hot


def dev():
    return torch.device("cuda:0")


def cases():
    rng = np.random.default_rng(31)
    out = {}
    n = 2000
    out["uniform2000"] = (rng.uniform(0.0, 1.0, (n, 3)), rng.uniform(0.5, 1.5, n) / n, 1.0, (0.0, 0.0, 0.0), 0.0)
    # clumps wrapped into a cube of side 2 at an offset corner, softened
    n = 4096
    c = rng.uniform(0.0, 1.0, (16, 3))
    x = (c[rng.integers(0, 16, n)] + 0.04 * rng.standard_normal((n, 3))) % 1.0
    lo = np.array([-1.0, -0.5, 0.25])
    out["clumps4096"] = (lo + 2.0 * x, np.full(n, 1.0 / n), 2.0, tuple(lo), 0.01)
    # ragged size, coincident particles, particles on the faces of the cube
    n = 1001
    lo = np.array([0.5, -2.0, 1.0])
    x = lo + 3.0 * rng.uniform(0.0, 1.0, (n, 3))
    x[10:20] = x[9]
    x[30, 0] = lo[0]
    x[31, 1] = lo[1] + 3.0 * (1 - 1e-12)
    out["ragged1001"] = (x, rng.uniform(0.5, 1.5, n) / n, 3.0, tuple(lo), 0.02)
    return out


COINCIDENT = {"ragged1001": np.arange(9, 20)}


CASES = cases()
D17 = {}


def lattice(L):
    if L not in D17:
        D17[L] = PR.lattice_coefficients(L, 17, 2)
    return D17[L]


def periodic_lists_match(h, t, cl):
    """Per group, the GPU's (cell, image) pairs equal the oracle's as sets, up to
    borderline decisions (a cell within 1e-9 of a threshold, and its descendants)."""
    Ls = t.lists()
    om, cm = Ls["m2p"]
    op, cp = Ls["p2p"]
    mi, pi = Ls["m2p_image"], Ls["p2p_image"]
    ob, cb = Ls["border"]
    gmo, gm, gmi = h.debug_get("M2P_OFFSETS"), h.debug_get("M2P_CELLS"), h.debug_get("M2P_IMAGES")
    gpo, gp, gpi = h.debug_get("P2P_OFFSETS"), h.debug_get("P2P_CELLS"), h.debug_get("P2P_IMAGES")
    assert gmi.min(initial=0) >= 0 and gmi.max(initial=0) <= 124 and gpi.max(initial=0) <= 124
    keys, level = cl["key"], cl["level"]
    bad = 0
    for g in range(len(om) - 1):
        a = set(zip(cm[om[g]:om[g + 1]].tolist(), mi[om[g]:om[g + 1]].tolist())) ^ \
            set(zip(gm[gmo[g]:gmo[g + 1]].tolist(), gmi[gmo[g]:gmo[g + 1]].tolist()))
        b = set(zip(cp[op[g]:op[g + 1]].tolist(), pi[op[g]:op[g + 1]].tolist())) ^ \
            set(zip(gp[gpo[g]:gpo[g + 1]].tolist(), gpi[gpo[g]:gpo[g + 1]].tolist()))
        diff = {c for c, _ in a | b}
        border = cb[ob[g]:ob[g + 1]]
        for c in diff:
            ok = any(level[c] >= level[x] and (int(keys[c]) >> (3 * (level[c] - level[x]))) == int(keys[x])
                     for x in border)
            bad += 0 if ok else 1
    return bad


def gpu_periodic(pos, mass, L, lo, p, tol, eps, prec, **kw):
    h = hot.Hot(p=p, tol=tol, eps=eps, precision=prec, box=L, ws=2, box_lo=lo, **kw)
    P = torch.tensor(pos, device=dev())
    M = torch.tensor(mass, device=dev())
    h.build_tree(P, M)
    h.compute_moments(p)
    h.traverse(tol)
    acc = torch.empty_like(P)
    pot = torch.empty_like(M)
    h.evaluate_forces(acc, pot)
    torch.cuda.synchronize()
    return h, acc.cpu().numpy(), pot.cpu().numpy()


def check(a, ph, an, af, pn, pf, prec, mass=None, L=1.0, eps=0.0, coincident=()):
    ra, rp = an + af, pn + pf
    err = np.linalg.norm(a - ra, axis=1)
    if prec == "fp64":
        rel = err / np.linalg.norm(ra, axis=1)
        prel = np.abs(ph - rp) / np.sqrt(np.mean(rp ** 2))
        assert rel.max() < 1e-9, rel.max()
        assert prel.max() < 1e-9, prel.max()
    else:
        parts = np.linalg.norm(an, axis=1) + np.linalg.norm(af, axis=1)
        if len(coincident):
            k = len(coincident) - 1
            allow = k * mass[coincident] * 2.0 ** -21 * L / eps ** 3
            assert np.all(err[coincident] <= 1e-3 * parts[coincident] + allow), (err[coincident], allow)
            keep = np.setdiff1d(np.arange(len(err)), coincident)
            err, parts = err[keep], parts[keep]
        rel = err / parts
        prel = np.abs(ph - rp) / np.abs(pn)
        assert np.sqrt(np.mean(rel ** 2)) < 1e-5, np.sqrt(np.mean(rel ** 2))
        assert rel.max() < 1e-3, rel.max()
        assert prel.max() < 2e-6, prel.max()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("p", [4, 8])
def test_periodic_lists_and_forces(name, p):
    pos, mass, L, lo, eps = CASES[name]
    tol = 1e-5
    t = oracle.Tree(pos, mass)
    t.periodic(L, 2)
    t.moments(p)
    t.traverse(tol)
    an, pn = t.force(1.0, eps)
    af, pf = PR.far_field(pos, mass, L, lo, p=8, ws=2, D=lattice(L))
    cl = t.cells()
    for prec in ("fp64", "mixed"):
        h, a, ph = gpu_periodic(pos, mass, L, lo, p, tol, eps, prec)
        assert periodic_lists_match(h, t, cl) == 0
        assert len(set(h.debug_get("P2P_IMAGES").tolist())) > 1
        check(a, ph, an, af, pn, pf, prec, mass, L, eps, COINCIDENT.get(name, ()))


def test_periodic_matches_ewald():
    """The method's periodic forces converge to the exact (Ewald) ones: FP64 path at p = 8
    and tol = 1e-8 within 1e-7 rms (potential: of its rms), the mixed path at tol = 1e-6
    within 1e-5 rms (potential: 2e-6 of the images' sum |phi_near| its float32 arithmetic
    works on)."""
    rng = np.random.default_rng(9)
    n, L = 600, 1.0
    x, m = rng.uniform(0, L, (n, 3)), rng.uniform(0.5, 1.5, n) / n
    ra, rp = PR.ewald(x, m, L)
    _, pnear = PR.near_images_direct(x, m, L)
    for prec, tol, bound in (("fp64", 1e-8, 1e-7), ("mixed", 1e-6, 1e-5)):
        _, a, ph = gpu_periodic(x, m, L, (0.0, 0.0, 0.0), 8, tol, 0.0, prec, leaf_max=16, group_max=32)
        rel = np.linalg.norm(a - ra, axis=1) / np.linalg.norm(ra, axis=1)
        assert np.sqrt(np.mean(rel ** 2)) < bound, (prec, np.sqrt(np.mean(rel ** 2)))
        if prec == "fp64":
            assert np.sqrt(np.mean((ph - rp) ** 2) / np.mean(rp ** 2)) < bound
        else:
            assert np.max(np.abs(ph - rp) / np.abs(pnear)) < 2e-6


def test_switching_boundaries_on_one_tree():
    """The same tree and context serve open and periodic boundaries in turn."""
    pos, mass, L, lo, eps = CASES["uniform2000"]
    t = oracle.Tree(pos, mass)
    t.moments(4)
    t.traverse(1e-5)
    ro, _ = t.force(1.0, eps)
    h = hot.Hot(p=4, tol=1e-5, eps=eps, precision="fp64")
    P = torch.tensor(pos, device=dev())
    M = torch.tensor(mass, device=dev())
    h.build_tree(P, M)
    acc = torch.empty_like(P)
    for box in (0.0, L, 0.0):
        h.set_params(p=4, tol=1e-5, eps=eps, precision="fp64", box=box, box_lo=lo)
        h.compute_moments(4)
        h.traverse(1e-5)
        h.evaluate_forces(acc, None)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        if box == 0.0:
            assert np.max(np.linalg.norm(a - ro, axis=1) / np.linalg.norm(ro, axis=1)) < 1e-11
            assert h.debug_get("P2P_IMAGES").max() == 0
        else:
            assert np.max(np.linalg.norm(a - ro, axis=1) / np.linalg.norm(ro, axis=1)) > 1e-3


def test_periodic_arguments_are_validated():
    for kw in (dict(box=-1.0), dict(box=float("nan")), dict(box=1.0, ws=0), dict(box=1.0, ws=3),
               dict(box=1.0, p_min=2), dict(box=1.0, box_lo=(0.0, float("inf"), 0.0))):
        with pytest.raises(hot.HotError) as e:
            hot.Hot(p=4, **kw)
        assert e.value.code == hot.HOT_EINVAL, kw
    pos, mass, L, lo, eps = CASES["uniform2000"]
    h, _, _ = gpu_periodic(pos[:300], mass[:300], L, lo, 4, 1e-4, 0.0, "mixed")
    P = torch.tensor(pos[:300], device=dev())
    with pytest.raises(hot.HotError) as e:
        h.adjoint(torch.ones_like(P), None, torch.empty_like(P), torch.empty(300, dtype=torch.float64, device=dev()))
    assert e.value.code == hot.HOT_EINVAL
