"""Host logic of the kick-drift-kick integrator and its reverse sweep (no GPU).

The integrator only calls force / build / adjoint / axpy on its context, so a
stand-in context whose force is the oracle's softened direct sum (and whose adjoint
is the oracle's analytic direct-sum gradient) exercises the sweep, the checkpoint
segments and the dt vs dt/2 factors on the CPU.  The reference is a central finite
difference of a plain numpy leapfrog over the same direct sum.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
from paper_1310_4502_gb300.leapfrog import KDK  # noqa: E402


class _P:
    p, tol = 4, 1e-4


class DirectCtx:
    """Duck-typed library context computing on CPU float64 tensors with the oracle."""

    def __init__(self, eps):
        self.eps = eps
        self.params = _P()
        self.generation = 0
        self.forces = 0
        self.builds = 0

    def build_tree(self, pos, mass):
        self.generation += 1
        self.builds += 1
        self._pos = pos.numpy().copy()
        self._mass = mass.numpy().copy()

    def compute_moments(self, p):
        pass

    def traverse(self, tol):
        pass

    def evaluate_forces(self, acc, pot=None):
        a, ph = oracle.direct(self._pos, self._mass, 1.0, self.eps)
        acc.copy_(torch.from_numpy(a))
        if pot is not None:
            pot.copy_(torch.from_numpy(ph))

    def force(self, pos, mass, acc, pot=None):
        self.forces += 1
        self.build_tree(pos, mass)
        self.evaluate_forces(acc, pot)

    def adjoint(self, g_acc, g_pot, g_pos, g_mass):
        gx, gm = oracle.direct_grad(self._pos, self._mass, g_acc.numpy(), None, 1.0, self.eps)
        g_pos.copy_(torch.from_numpy(gx))
        g_mass.copy_(torch.from_numpy(gm))

    def axpy(self, y, x, alpha):
        y.add_(x, alpha=alpha)


def numpy_leapfrog(x, v, m, dt, S, eps):
    x, v = x.copy(), v.copy()
    a, _ = oracle.direct(x, m, 1.0, eps)
    for _ in range(S):
        v += 0.5 * dt * a
        x += dt * v
        a, _ = oracle.direct(x, m, 1.0, eps)
        v += 0.5 * dt * a
    return x, v


def _case(n=24, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 3))
    v = 0.3 * rng.standard_normal((n, 3))
    m = rng.uniform(0.5, 1.5, n) / n
    wx = rng.standard_normal((n, 3))
    wv = rng.standard_normal((n, 3))
    return x, v, m, wx, wv


@pytest.mark.parametrize("S,every", [(1, 1), (5, 1), (5, 2), (6, 3), (5, 7)])
def test_reverse_sweep_matches_finite_differences(S, every):
    x, v, m, wx, wv = _case()
    dt, eps = 0.2, 0.1

    def loss(x_, v_, m_):
        xs, vs = numpy_leapfrog(x_, v_, m_, dt, S, eps)
        return np.sum(wx * xs) + np.sum(wv * vs)

    ctx = DirectCtx(eps)
    integ = KDK(ctx, dt, S, every)
    T = torch.from_numpy
    xs, vs = integ.forward(T(x), T(v), T(m))
    rx, rv = numpy_leapfrog(x, v, m, dt, S, eps)
    assert np.allclose(xs.numpy(), rx, rtol=0, atol=1e-13) and np.allclose(vs.numpy(), rv, rtol=0, atol=1e-13)
    assert ctx.forces == S + 1
    gx, gv, gm = integ.backward(T(wx), T(wv))
    h = 1e-5
    for i in (0, 7, 23):
        for d in range(3):
            for arr, g in ((x, gx), (v, gv)):
                ap, am = arr.copy(), arr.copy()
                ap[i, d] += h
                am[i, d] -= h
                args_p = (ap, v, m) if arr is x else (x, ap, m)
                args_m = (am, v, m) if arr is x else (x, am, m)
                fd = (loss(*args_p) - loss(*args_m)) / (2 * h)
                assert g[i, d].item() == pytest.approx(fd, rel=1e-6, abs=1e-7)
        mp, mm = m.copy(), m.copy()
        mp[i] += h * m[i]
        mm[i] -= h * m[i]
        fd = (loss(x, v, mp) - loss(x, v, mm)) / (2 * h * m[i])
        assert gm[i].item() == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_checkpoint_interval_changes_nothing_but_work():
    x, v, m, wx, wv = _case(seed=3)
    T = torch.from_numpy
    out = []
    for every in (1, 2, 4, 8):
        ctx = DirectCtx(0.05)
        integ = KDK(ctx, 0.1, 8, every)
        integ.forward(T(x), T(v), T(m))
        f0 = ctx.forces
        g = integ.backward(T(wx), T(wv))
        out.append((g, ctx.forces - f0))
    for g, _ in out[1:]:
        for a, b in zip(g, out[0][0]):
            assert torch.allclose(a, b, rtol=1e-13, atol=1e-15)
    # every = 1 recomputes nothing; every = k > 1 re-runs the forward over each segment of
    # k steps from its checkpoint: k force evaluations per segment, S in all
    assert [f for _, f in out] == [0, 8, 8, 8]


def test_backward_needs_forward_and_rejects_bad_sizes():
    with pytest.raises(ValueError):
        KDK(DirectCtx(0.1), 0.1, 0)
    with pytest.raises(RuntimeError):
        KDK(DirectCtx(0.1), 0.1, 2).backward(None, None)


def test_periodic_contexts_are_refused():
    """The reverse sweep is hot_adjoint, which periodic boundaries do not have."""
    ctx = DirectCtx(0.1)

    class _Per(_P):
        box = 1.0
    ctx.params = _Per()
    with pytest.raises(ValueError):
        KDK(ctx, 0.1, 2)
