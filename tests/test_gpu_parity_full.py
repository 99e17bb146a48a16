"""GPU parity at the benchmark's full sizes.

Bit-exact on every element: the key frame, the sorted keys, the sort permutation, every
cell array (key, level, first slot, count, parent, child count) and the sink groups with
their centres and extents, at 2^20 (clustered), 128^3 and 256^3 (lattices) -- the radix
sort's multi-tile scans and the tree builder's long runs at the sizes the benchmark
times.

Forces on sampled outputs: the CUDA path runs the whole workload in the launch
configuration the benchmark times (default tree sizes, one context per precision); the
oracle builds the same tree but traverses and evaluates only a seeded sample of sink
groups, whose sinks' forces it computes one group at a time.  Compared on those sinks: the FP64 path to 1e-11 relative, the mixed
path to 1e-5 rms / 1e-3 max relative (acceleration) and 1e-4 max relative (potential),
the tolerances of the small-size parity tests.

Workloads: the clustered box at N = 2^20 (p = 4 and p = 6; p = 4 with K1 smoothing; p = 8
with per-interaction order selection over 0..8), the Zel'dovich lattice at 128^3 (p = 6)
and, as the largest size, 256^3 (p = 6, mixed only).
"""
import numpy as np
import pytest

import oracle
from paper_1310_4502_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_4502_gb300 import hot

NGROUP_SAMPLE = 256

_cache = {}


def workload(name):
    if name not in _cache:
        _cache.clear()
        w = W.make(name)
        t = oracle.Tree(w.pos, w.mass)
        _cache[name] = (w, t)
    return _cache[name]


def sample_groups(t, seed):
    ng = t.info()["ngroup"]
    rng = np.random.default_rng(seed)
    gs = rng.choice(ng, min(NGROUP_SAMPLE, ng), replace=False)
    # the groups holding the largest sink counts are the ragged edge of the warp tiling
    # (more than one pass of 32 sinks): always include the largest one
    cl = t.cells()
    gc = t.groups()["cell"]
    gs = np.union1d(gs, [int(np.argmax(cl["count"][gc]))])
    return gs.astype(np.int64)


def sinks_of(t, gs):
    _, perm = t.keys()
    cl = t.cells()
    gc = t.groups()["cell"]
    idx = [perm[cl["begin"][c]:cl["begin"][c] + cl["count"][c]] for c in gc[gs]]
    return np.concatenate(idx)


@pytest.mark.parametrize("name", ["clustered20", "zeldovich128", "zeldovich256"])
def test_full_size_tree_bit_exact(name):
    w, t = workload(name)
    dev = torch.device("cuda:0")
    P = torch.tensor(w.pos, device=dev)
    M = torch.tensor(w.mass, device=dev)
    h = hot.Hot(p=w.p, tol=w.tol, eps=w.eps, precision="mixed")
    h.build_tree(P, M)
    lo, L = t.frame()
    fr = h.debug_get("FRAME")
    assert np.array_equal(fr[:3], lo) and fr[3] == L
    k, perm = t.keys()
    assert np.array_equal(h.debug_get("PERM").astype(np.int64), perm)
    assert np.array_equal(h.debug_get("SORTED_KEYS"), k[perm])
    del k, perm
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
    # every cell key is found by the hash table at its own index
    keys = h.debug_get("CELL_KEY")
    assert np.array_equal(h.lookup(keys), np.arange(len(keys), dtype=np.int32))
    h.close()
    del P, M
    torch.cuda.empty_cache()


@pytest.mark.parametrize("name,p,precisions,opts", [
    ("clustered20", 4, ("mixed", "fp64"), {}),
    ("clustered20", 6, ("mixed", "fp64"), {}),
    ("clustered20", 4, ("mixed", "fp64"), {"softening": "k1"}),
    ("clustered20", 4, ("mixed", "fp64"), {"softening": "spline"}),
    ("clustered20", 8, ("mixed", "fp64"), {"p_min": 0}),
    ("zeldovich128", 6, ("mixed", "fp64"), {}),
    ("zeldovich256", 6, ("mixed",), {}),
])
def test_full_size_sampled_forces(name, p, precisions, opts):
    w, t = workload(name)
    t.softening(opts.get("softening", "plummer"), w.eps)
    t.moments(p)
    t.order_range(opts.get("p_min"))
    gs = sample_groups(t, seed=100 + p)
    t.traverse(w.tol, groups=gs)
    ra, rp = t.force(1.0, w.eps, groups=gs)
    idx = sinks_of(t, gs)
    assert len(idx) > 0
    ra, rp = ra[idx], rp[idx]
    na = np.linalg.norm(ra, axis=1)
    dev = torch.device("cuda:0")
    P = torch.tensor(w.pos, device=dev)
    M = torch.tensor(w.mass, device=dev)
    for prec in precisions:
        h = hot.Hot(p=p, tol=w.tol, eps=w.eps, precision=prec, **opts)
        h.build_tree(P, M)
        # the group cells the oracle sampled are the GPU's groups too
        gcell = h.debug_get("GROUP_CELL")
        assert np.array_equal(gcell[gs], t.groups()["cell"][gs])
        h.compute_moments(p)
        h.traverse(w.tol)
        acc = torch.empty_like(P)
        pot = torch.empty_like(M)
        h.evaluate_forces(acc, pot)
        h.synchronize()
        a = acc[torch.from_numpy(idx).to(dev)].cpu().numpy()
        ph = pot[torch.from_numpy(idx).to(dev)].cpu().numpy()
        del h, acc, pot
        rel = np.linalg.norm(a - ra, axis=1) / na
        prel = np.abs(ph - rp) / np.abs(rp)
        if prec == "fp64":
            assert rel.max() < 1e-11, rel.max()
            assert prel.max() < 1e-11, prel.max()
        else:
            assert np.sqrt(np.mean(rel ** 2)) < 1e-5, np.sqrt(np.mean(rel ** 2))
            assert rel.max() < 1e-3, rel.max()
            assert prel.max() < 1e-4, prel.max()
    del P, M
    torch.cuda.empty_cache()
