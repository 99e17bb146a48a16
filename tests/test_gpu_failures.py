"""Overflow and timeout paths on the GPU, forced through the test knobs of hot_debug_set on
small inputs.  Nothing here faults, traps or hangs the device: every path ends in a status
code that the host reads, and the context stays usable.

* list slots too small: the one-pass traversal falls back to count/scan/fill and produces
  the same lists and forces;
* traversal frontier too small: the call retries with larger capacities (same lists), or
  returns HOT_EOVERFLOW when the retries run out, after which the forces are refused until
  a traversal succeeds;
* an expired wait in the interaction kernel (a barrier nothing completes, polled a bounded
  number of times): HOT_ETIMEOUT at the next synchronisation, for the forces and for the
  adjoint; the next evaluation without the setting is exact again.
"""
import numpy as np
import pytest

from paper_1310_4502_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_4502_gb300 import hot


def dev():
    return torch.device("cuda:0")


def _run(pos, mass, knobs=(), p=4, tol=1e-4, eps=0.01, **kw):
    h = hot.Hot(p=p, tol=tol, eps=eps, **kw)
    for what, value in knobs:
        h.debug_set(what, value)
    P = torch.tensor(pos, device=dev())
    M = torch.tensor(mass, device=dev())
    h.build_tree(P, M)
    h.compute_moments(p)
    h.traverse(tol)
    acc = torch.empty_like(P)
    pot = torch.empty_like(M)
    h.evaluate_forces(acc, pot)
    h.synchronize()
    lists = [h.debug_get(k) for k in ("M2P_OFFSETS", "M2P_CELLS", "P2P_OFFSETS", "P2P_CELLS")]
    return h, P, M, lists, acc.cpu().numpy(), pot.cpu().numpy()


def test_slot_overflow_falls_back_to_count_and_fill():
    w = W.make("plummer4096")
    _, _, _, ref_lists, ref_a, ref_p = _run(w.pos, w.mass)
    h, P, M, lists, a, ph = _run(w.pos, w.mass, knobs=[(hot.HOT_DBGSET_SLOT_CAP, 1)])
    for x, y in zip(lists, ref_lists):
        assert np.array_equal(x, y)
    assert np.array_equal(a, ref_a) and np.array_equal(ph, ref_p)
    # the slots are sized from the counts for the next traversal, which fits again
    h.traverse(1e-4)
    for k, y in zip(("M2P_OFFSETS", "M2P_CELLS", "P2P_OFFSETS", "P2P_CELLS"), ref_lists):
        assert np.array_equal(h.debug_get(k), y)


def test_frontier_overflow_retries_then_reports():
    w = W.make("plummer4096")
    # a deep tree and a tight tolerance: wide traversal frontiers
    kw = dict(leaf_max=1, group_max=8)
    _, _, _, ref_lists, ref_a, _ = _run(w.pos, w.mass, tol=1e-7, **kw)
    # a small capacity is grown by the retries (256 -> 1024 -> 4096 -> 16384): identical
    # lists and forces
    _, _, _, lists, a, _ = _run(w.pos, w.mass, knobs=[(hot.HOT_DBGSET_FRONTIER_CAP, 256)], tol=1e-7, **kw)
    for x, y in zip(lists, ref_lists):
        assert np.array_equal(x, y)
    assert np.array_equal(a, ref_a)
    # capacity 1 grows to 64 at most: the frontier does not fit, the call reports it
    h = hot.Hot(p=4, tol=1e-10, eps=0.01, **kw)
    h.debug_set(hot.HOT_DBGSET_FRONTIER_CAP, 1)
    P = torch.tensor(w.pos, device=dev())
    M = torch.tensor(w.mass, device=dev())
    h.build_tree(P, M)
    h.compute_moments(4)
    with pytest.raises(hot.HotError) as e:
        h.traverse(1e-10)
    assert e.value.code == hot.HOT_EOVERFLOW
    acc = torch.empty_like(P)
    with pytest.raises(hot.HotError) as e:
        h.evaluate_forces(acc)
    assert e.value.code == hot.HOT_ESTATE
    # the context recovers with an adequate capacity
    h.debug_set(hot.HOT_DBGSET_FRONTIER_CAP, 4096)
    h.traverse(1e-10)
    h.evaluate_forces(acc)
    h.synchronize()


def test_expired_wait_reports_timeout_and_context_recovers():
    w = W.make("plummer4096")
    h, P, M, _, ref_a, ref_p = _run(w.pos, w.mass)
    acc = torch.empty_like(P)
    pot = torch.empty_like(M)
    # every group's M2P pass first waits, for at most 64 polls, on a barrier that nothing
    # completes
    h.debug_set(hot.HOT_DBGSET_WAIT_POLLS, 64)
    h.debug_set(hot.HOT_DBGSET_WAIT_PROBE, 1)
    h.evaluate_forces(acc, pot)
    with pytest.raises(hot.HotError) as e:
        h.synchronize()
    assert e.value.code == hot.HOT_ETIMEOUT
    # the adjoint's sink pass takes the same path
    gw = torch.ones_like(P)
    gx = torch.empty_like(P)
    gm = torch.empty_like(M)
    h.adjoint(gw, None, gx, gm)
    with pytest.raises(hot.HotError) as e:
        h.synchronize()
    assert e.value.code == hot.HOT_ETIMEOUT
    h.debug_set(hot.HOT_DBGSET_WAIT_PROBE, 0)
    h.debug_set(hot.HOT_DBGSET_WAIT_POLLS, 0)
    h.evaluate_forces(acc, pot)
    h.synchronize()
    assert np.array_equal(acc.cpu().numpy(), ref_a) and np.array_equal(pot.cpu().numpy(), ref_p)


def test_debug_knobs_reject_bad_values():
    h = hot.Hot()
    for what, value in ((hot.HOT_DBGSET_FRONTIER_CAP, 0), (hot.HOT_DBGSET_SLOT_CAP, -1),
                        (hot.HOT_DBGSET_WAIT_POLLS, -1), (hot.HOT_DBGSET_WAIT_PROBE, 2), (99, 1)):
        with pytest.raises(hot.HotError) as e:
            h.debug_set(what, value)
        assert e.value.code == hot.HOT_EINVAL
