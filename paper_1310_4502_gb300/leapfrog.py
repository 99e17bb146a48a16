"""Kick-drift-kick leapfrog over the tree force, its adjoint, and the autograd wrappers.

Time stepping follows Sec. "Time Integration" (kick-drift-kick leapfrog).  Step k = 1..S
with the tree rebuilt at every force point:

    v += dt/2 a(x_{k-1});   x += dt v;   a_k = a(x_k);   v += dt/2 a_k

The force at x_k is shared by the closing kick of step k and the opening kick of step
k+1, so S steps take S+1 force evaluations.

Backward.  The derivative is the one of the discrete map with each force point's tree
(interaction lists and expansion centres) frozen at the positions it was built from; the
moments remain functions of positions and masses (the same convention as hot_adjoint).
With adjoint variables xb = dL/dx_S, vb = dL/dv_S, the reverse sweep is

    point S:           a-bar = dt/2 vb           xb += J_S^T a-bar,  mb += ...
    for k = S .. 1:    vb += dt xb                            (adjoint of the drift)
                       a-bar = dt vb  (dt/2 vb at point 0)    xb += J_{k-1}^T a-bar, ...

because the closing kick of step k-1 and the opening kick of step k both read a_{k-1}
with the same adjoint velocity.  hot_adjoint is linear in its weights, so it is called
with vb itself and its outputs are added with the factor dt or dt/2.

Checkpoint-and-recompute: the forward keeps (x, v) at every `every`-th step point and
the final positions; nothing of the trees or lists.  The backward walks the segments
from last to first, re-runs the forward over a segment from its checkpoint to recover
the positions of its force points (bit-identical: every stage is deterministic), then
rebuilds the tree at each of those points, newest first, for the adjoint.  With
every = 1 the recomputation is only the rebuild that the adjoint needs in any case.

All arithmetic runs in libhot.so: the kicks and drifts and their adjoints are hot_axpy,
forces and their adjoints the tree path.  Tensors are contiguous float64 on the device.
"""
from __future__ import annotations

from . import hot as _hot


class KDK:
    """S kick-drift-kick steps of size dt on one library context."""

    def __init__(self, ctx: "_hot.Hot", dt: float, steps: int, every: int = 1):
        if steps < 1 or every < 1:
            raise ValueError("steps and every must be >= 1")
        if getattr(ctx.params, "box", 0.0) > 0.0:
            # the backward is hot_adjoint, which periodic boundaries do not have, and the
            # drifts would carry particles out of the cube the forces assume
            raise ValueError("the leapfrog runs on open boundaries only")
        self.h = ctx
        self.dt = float(dt)
        self.S = int(steps)
        self.every = int(every)
        self._ckpt = None

    # ---- forward -----------------------------------------------------------------
    def _advance(self, x, v, a, mass, k0, k1, keep=None):
        """Steps k0+1 .. k1 starting from (x, v) with a = a(x) already computed; when
        keep is a list, the positions of the force points k0+1 .. k1-1 are appended."""
        h, dt = self.h, self.dt
        for k in range(k0 + 1, k1 + 1):
            h.axpy(v, a, 0.5 * dt)
            h.axpy(x, v, dt)
            if keep is not None and k < k1:
                keep.append(x.clone())
            h.force(x, mass, a)
            h.axpy(v, a, 0.5 * dt)

    def forward(self, x0, v0, mass):
        """Returns (x_S, v_S); keeps the checkpoints for backward."""
        import torch
        x = x0.clone()
        v = v0.clone()
        a = torch.empty_like(x)
        self.h.force(x, mass, a)
        ckpt = {}
        k = 0
        while k < self.S:
            ckpt[k] = (x.clone(), v.clone())
            k1 = min(k + self.every, self.S)
            self._advance(x, v, a, mass, k, k1)
            k = k1
        self._ckpt = ckpt
        self._xS = x.clone()
        self._gen = self.h.generation  # the context now holds the tree at x_S
        self._mass = mass
        return x, v

    # ---- backward ----------------------------------------------------------------
    def _adjoint_at(self, x, fresh, vb, alpha, xb, mb, gp, gm):
        """xb += alpha J^T vb, mb += alpha (dL/dm) at the force point x; the tree is
        rebuilt there unless `fresh` says the context already holds it."""
        h = self.h
        if not fresh:
            h.build_tree(x, self._mass)
            h.compute_moments(h.params.p)
            h.traverse(h.params.tol)
        h.adjoint(vb, None, gp, gm)
        h.axpy(xb, gp, alpha)
        h.axpy(mb, gm, alpha)

    def backward(self, gx, gv):
        """Given dL/dx_S and dL/dv_S (either may be None), returns dL/dx_0, dL/dv_0 and
        dL/dm of the whole trajectory."""
        import torch
        if self._ckpt is None:
            raise RuntimeError("backward before forward")
        h, dt, mass = self.h, self.dt, self._mass
        xb = torch.zeros_like(self._xS) if gx is None else gx.clone()
        vb = torch.zeros_like(self._xS) if gv is None else gv.clone()
        mb = torch.zeros_like(mass)
        gp = torch.empty_like(xb)
        gm = torch.empty_like(mb)
        a = torch.empty_like(xb)
        fresh = h.generation == self._gen
        self._adjoint_at(self._xS, fresh, vb, 0.5 * dt, xb, mb, gp, gm)
        starts = sorted(self._ckpt, reverse=True)
        end = self.S
        for c in starts:
            # positions of the force points c .. end-1 of this segment
            xc, vc = self._ckpt[c]
            pts = [xc]
            if end - c > 1:
                x = xc.clone()
                v = vc.clone()
                h.force(x, mass, a)
                self._advance(x, v, a, mass, c, end - 1, keep=pts)
                pts.append(x)
            last_built = end - 1 if end - c > 1 else None
            for k in range(end, c, -1):
                h.axpy(vb, xb, dt)  # adjoint of the drift x += dt v
                j = k - 1
                self._adjoint_at(pts[j - c], j == last_built, vb, dt if j > 0 else 0.5 * dt,
                                 xb, mb, gp, gm)
                last_built = None
            end = c
        return xb, vb, mb


def _autograd():
    import torch

    class TreeForce(torch.autograd.Function):
        """acc, pot = tree force of (pos, mass) on a context; the backward is hot_adjoint
        through the lists and centres of this forward (rebuilt from the saved positions
        when the context has moved on to another tree)."""

        @staticmethod
        def forward(fctx, pos, mass, h):
            pos = pos.contiguous()
            mass = mass.contiguous()
            acc = torch.empty_like(pos)
            pot = torch.empty_like(mass)
            h.force(pos, mass, acc, pot)
            fctx.h = h
            fctx.gen = h.generation
            fctx.save_for_backward(pos, mass)
            return acc, pot

        @staticmethod
        def backward(fctx, g_acc, g_pot):
            pos, mass = fctx.saved_tensors
            h = fctx.h
            if h.generation != fctx.gen:
                h.build_tree(pos, mass)
                h.compute_moments(h.params.p)
                h.traverse(h.params.tol)
            ga = torch.zeros_like(pos) if g_acc is None else g_acc.contiguous()
            gpot = None if g_pot is None else g_pot.contiguous()
            gx = torch.empty_like(pos)
            gm = torch.empty_like(mass)
            h.adjoint(ga, gpot, gx, gm)
            return gx, gm, None

    class Leapfrog(torch.autograd.Function):
        """(x_S, v_S) after S kick-drift-kick steps; backward by checkpoint-and-recompute."""

        @staticmethod
        def forward(fctx, x0, v0, mass, h, dt, steps, every):
            integ = KDK(h, dt, steps, every)
            x, v = integ.forward(x0.contiguous(), v0.contiguous(), mass.contiguous())
            fctx.integ = integ
            return x, v

        @staticmethod
        def backward(fctx, gx, gv):
            xb, vb, mb = fctx.integ.backward(None if gx is None else gx.contiguous(),
                                             None if gv is None else gv.contiguous())
            fctx.integ = None
            return xb, vb, mb, None, None, None, None

    return TreeForce, Leapfrog


def tree_force_fn(pos, mass, h):
    """Differentiable tree force: (acc, pot) with autograd through hot_adjoint."""
    return _autograd()[0].apply(pos, mass, h)


def leapfrog_fn(x0, v0, mass, h, dt, steps, every=1):
    """Differentiable S-step kick-drift-kick leapfrog: (x_S, v_S)."""
    return _autograd()[1].apply(x0, v0, mass, h, dt, steps, every)
