"""GPU kick-drift-kick leapfrog and its checkpoint-and-recompute backward against the oracle.

* Forward: the device trajectory (tree rebuilt at every force point) against the
  oracle's leapfrog over oracle trees built along its own trajectory.
* Time reversibility: S steps, velocities negated, S steps return to the start.
* Backward: dL/dx0, dL/dv0, dL/dm of L = wx.x_S + wv.v_S against fourth-order central
  differences of the oracle's leapfrog with every tree frozen along the unperturbed
  trajectory (lists and centres fixed, moments from the perturbed particles).  Besides
  the whole gradient, the part due to the forces (the gradient minus its force-free
  value wx, S dt wx + wv, 0) is compared, since the identity part dominates.
* The checkpoint interval changes the work, not the gradient; autograd wrappers agree
  with the direct calls.
"""
import numpy as np
import pytest

import oracle
from paper_1310_4502_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1310_4502_gb300 import hot
    from paper_1310_4502_gb300 import leapfrog as LF

P, TOL = 4, 1e-4


def dev():
    return torch.device("cuda:0")


def _case(n=1024):
    w = W.make("plummer4096")
    x = w.pos[:n].copy()
    m = np.full(n, 1.0 / n)
    rng = np.random.default_rng(11)
    r = np.linalg.norm(x, axis=1, keepdims=True)
    vc = np.sqrt(r ** 2 / (r ** 2 + 1) ** 1.5)  # roughly the Plummer circular speed
    v = 0.5 * vc * rng.standard_normal((n, 3)) / np.sqrt(3)
    wx = rng.standard_normal((n, 3))
    wv = rng.standard_normal((n, 3))
    return x, v, m, wx, wv, 0.02


def _otree(x, m):
    t = oracle.Tree(x, m)
    t.moments(P)
    t.traverse(TOL)
    return t


def oracle_trajectory(x, v, m, dt, S, eps):
    """Trees rebuilt at the oracle's own force points; returns (trees, x_S, v_S)."""
    trees = [_otree(x, m)]
    a, _ = trees[0].frozen_force(x, m, 1.0, eps)
    x, v = x.copy(), v.copy()
    for _ in range(S):
        xn = x + dt * (v + 0.5 * dt * a)
        trees.append(_otree(xn, m))
        x, v = oracle.frozen_leapfrog(trees[-2:], x, v, m, dt, 1.0, eps)
        a, _ = trees[-1].frozen_force(x, m, 1.0, eps)
    return trees, x, v


def gpu_run(x, v, m, dt, S, eps, prec, every=1, wx=None, wv=None):
    h = hot.Hot(p=P, tol=TOL, eps=eps, precision=prec)
    T = lambda a: torch.tensor(a, device=dev())  # noqa: E731
    integ = LF.KDK(h, dt, S, every)
    xs, vs = integ.forward(T(x), T(v), T(m))
    g = None
    if wx is not None:
        g = [t.cpu().numpy() for t in integ.backward(T(wx), T(wv))]
    torch.cuda.synchronize()
    return xs.cpu().numpy(), vs.cpu().numpy(), g


@pytest.mark.parametrize("prec,bx,bv", [("fp64", 1e-12, 1e-12), ("mixed", 1e-7, 1e-6)])
def test_forward_matches_oracle_trajectory(prec, bx, bv):
    """Absolute bounds: FP64 forces agree with the oracle to about 1e-12 and mixed ones to
    about 1e-6 of |a| at worst; 8 steps of dt = 0.01 scale these by S dt (v) and S^2 dt^2 (x)."""
    x, v, m, _, _, eps = _case()
    dt, S = 0.01, 8
    _, ox, ov = oracle_trajectory(x, v, m, dt, S, eps)
    gx, gv, _ = gpu_run(x, v, m, dt, S, eps, prec)
    assert np.max(np.abs(gx - ox)) < bx
    assert np.max(np.abs(gv - ov)) < bv


def test_time_reversible_fp64():
    x, v, m, _, _, eps = _case()
    dt, S = 0.01, 6
    x1, v1, _ = gpu_run(x, v, m, dt, S, eps, "fp64")
    x2, v2, _ = gpu_run(x1, -v1, m, dt, S, eps, "fp64")
    assert np.max(np.abs(x2 - x)) < 1e-12
    assert np.max(np.abs(-v2 - v)) < 1e-11


def _fd(trees, x, v, m, wx, wv, dt, eps, ks, h=1e-4):
    """Fourth-order central differences.  The loss difference sums 3N coordinates of two
    separately rounded trajectories, about 1e-13 of noise, so h = 1e-6 would leave ~1e-8
    in the derivative; at h = 1e-4 noise and truncation (h^4 terms) are both ~1e-10."""
    def L(x_, v_, m_):
        xs, vs = oracle.frozen_leapfrog(trees, x_, v_, m_, dt, 1.0, eps)
        return xs, vs

    def dL(p1, m1, p2, m2):
        (a, b), (c, d) = p1, p2
        return np.sum(wx * (a - c)) + np.sum(wv * (b - d))

    gx = np.zeros((len(ks), 3))
    gv = np.zeros((len(ks), 3))
    gm = np.zeros(len(ks))
    for r, k in enumerate(ks):
        for d in range(3):
            for which, out in ((0, gx), (1, gv)):
                res = []
                for s in (1, -1, 2, -2):
                    xx, vv = x.copy(), v.copy()
                    (xx if which == 0 else vv)[k, d] += s * h
                    res.append(L(xx, vv, m))
                out[r, d] = (8 * dL(res[0], 0, res[1], 0) - dL(res[2], 0, res[3], 0)) / (12 * h)
        hm = 1e-2 * m[k]
        res = []
        for s in (1, -1, 2, -2):
            mm = m.copy()
            mm[k] += s * hm
            res.append(L(x, v, mm))
        gm[r] = (8 * dL(res[0], 0, res[1], 0) - dL(res[2], 0, res[3], 0)) / (12 * hm)
    return gx, gv, gm


KS = [0, 333]
FD_DT, FD_S = 0.05, 4


@pytest.fixture(scope="module")
def fd_ref():
    x, v, m, wx, wv, eps = _case()
    trees, _, _ = oracle_trajectory(x, v, m, FD_DT, FD_S, eps)
    return _fd(trees, x, v, m, wx, wv, FD_DT, eps, KS)


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-8), ("mixed", 1e-5)])
def test_backward_against_finite_differences(fd_ref, prec, bound):
    x, v, m, wx, wv, eps = _case()
    dt, S, ks = FD_DT, FD_S, KS
    fx, fv, fm = fd_ref
    _, _, (gx, gv, gm) = gpu_run(x, v, m, dt, S, eps, prec, wx=wx, wv=wv)
    gx, gv, gm = gx[ks], gv[ks], gm[ks]
    # whole gradient, relative
    for g, f in ((gx, fx), (gv, fv)):
        assert np.max(np.linalg.norm(g - f, axis=1) / np.linalg.norm(f, axis=1)) < bound
    assert np.max(np.abs(gm - fm) / np.abs(fm)) < bound
    # force-induced part, relative to its own size
    free_x, free_v = wx[ks], S * dt * wx[ks] + wv[ks]
    for g, f, free in ((gx, fx, free_x), (gv, fv, free_v)):
        scale = np.max(np.linalg.norm(f - free, axis=1))
        assert np.max(np.linalg.norm(g - f, axis=1)) / scale < 100 * bound


def test_checkpoint_interval_gives_identical_gradients():
    x, v, m, wx, wv, eps = _case(2048)
    dt, S = 0.02, 6
    ref = gpu_run(x, v, m, dt, S, eps, "mixed", every=1, wx=wx, wv=wv)
    for every in (2, 3, 6):
        out = gpu_run(x, v, m, dt, S, eps, "mixed", every=every, wx=wx, wv=wv)
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        for a, b in zip(out[2], ref[2]):
            assert np.array_equal(a, b), every


def test_autograd_wrappers_match_direct_calls():
    x, v, m, wx, wv, eps = _case()
    h = hot.Hot(p=P, tol=TOL, eps=eps, precision="fp64")
    X = torch.tensor(x, device=dev(), requires_grad=True)
    M = torch.tensor(m, device=dev(), requires_grad=True)
    Wx = torch.tensor(wx, device=dev())
    acc, pot = LF.tree_force_fn(X, M, h)
    # another tree in between: backward must rebuild from the saved positions
    h.force(X.detach() + 0.1, M.detach(), torch.empty_like(acc))
    (acc * Wx).sum().backward()
    h2 = hot.Hot(p=P, tol=TOL, eps=eps, precision="fp64")
    gx = torch.empty_like(acc)
    gm = torch.empty_like(pot)
    h2.force(X.detach(), M.detach(), torch.empty_like(acc))
    h2.adjoint(Wx, None, gx, gm)
    assert torch.equal(X.grad, gx) and torch.equal(M.grad, gm)

    V = torch.tensor(v, device=dev(), requires_grad=True)
    X.grad = None
    M.grad = None
    xs, vs = LF.leapfrog_fn(X, V, M, h, 0.02, 3)
    ((xs * Wx).sum() + (vs * torch.tensor(wv, device=dev())).sum()).backward()
    _, _, (rx, rv, rm) = gpu_run(x, v, m, 0.02, 3, eps, "fp64", wx=wx, wv=wv)
    assert np.array_equal(X.grad.cpu().numpy(), rx)
    assert np.array_equal(V.grad.cpu().numpy(), rv)
    assert np.array_equal(M.grad.cpu().numpy(), rm)
