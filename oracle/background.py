"""Background subtraction (Sec. "Background Subtraction") for the CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU legs may use
it; the CUDA path never does, and it shares no code with the CUDA library.

The paper turns the always-positive mass into density contrasts: the field computed is
that of the particles minus a uniform background.  Readings (the paper describes the
technique, not its formulas):

* Background: the mean density rho = M / L^3 over the tree's root cube [lo, lo + L)^3 (the
  key frame), not softened.  The quantity is
      a_i   = G sum_{j != i} m_j (x_j - x_i) / s_ij^3  -  G rho int_root (x - x_i) / |x - x_i|^3 dV
      phi_i = -G sum_{j != i} m_j / s_ij  +  G rho int_root dV / |x - x_i|,
  s_ij the Plummer-softened separation; the background's field is that of a uniform
  cube (Waldvogel's closed form).
* Far field: a cell's expansion is that of its contrast, the particles' moments about the
  cube's geometric centre minus those of a uniform cube of density rho, both to order p
  (so dipoles appear, and the background is subtracted only to the matter's order).
* Near field: the group's surrounding cube S is its cell's ancestor `up` levels above
  (two by default, the paper's "larger cube" around the near field: with the parent alone
  the conservative test of the contrast turns too many neighbours into particle pairs;
  the root if there are fewer levels).  The background of S is
  removed by the analytic field of a uniform cube; the cells inside S therefore interact
  by their matter alone, as in the plain method (centre-of-mass expansions, the same
  acceptance test), and their empty octants need nothing.
* Outside S: an accepted cell interacts by its contrast expansion; a leaf taken
  particle by particle also removes the analytic field of its cube; the empty octants of
  every opened cell (child cubes holding no particle, absent from the tree) are cells of
  pure negative density, taken by their expansion when accepted, otherwise by the
  analytic field of their cube.
* Acceptance of a contrast expansion: the bound of Sec. "Multipole Error Bounds" rests on
  radial moments B_n of a positive distribution; for the contrast (a signed one) the
  test uses the sizes of its first two omitted multipoles instead,
      E(d) = G / (1 - b/d)^2 [(p+2) Q_{p+1} / d^{p+3} + (p+3) Q_{p+2} / d^{p+4}] <= tol,
      Q_n = ( sum_{|a| = n} n! / a! M_a^2 )^(1/2)   (M_a the contrast's moments about c),
  d = |c - g| - Delta_max from the cube's centre c, b = the half-diagonal sqrt(3) s / 2.
  Q_n is near zero for a cell that its particles fill uniformly, which is what lets far
  cells be accepted sooner; both orders are needed, a uniform cube's odd multipoles
  vanishing.  It is an estimate, not a bound.
"""
from __future__ import annotations

import math

import numpy as np

from . import Tree, direct, m2p_points, mac_bound, moments, multi_indices


# ---- the uniform cube ----

def _log_plus_r(a, r):
    """ln(a + r), r = |(a, b, c)| >= |a|, without cancellation for a < 0:
    a + r = (b^2 + c^2) / (r - a)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(a >= 0, np.log(a + r), np.log(np.maximum(r * r - a * a, 0.0)) - np.log(r - a))


def _safe(prod, val):
    """prod * val, taken as 0 where prod is 0 (the limits on the box's edges and faces)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(prod == 0, 0.0, prod * np.nan_to_num(val, nan=0.0, posinf=0.0, neginf=0.0))


def _atan_term(u, v, w, r):
    """atan(v w / (u r)), taken as 0 where u = 0 (it is then multiplied by u)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(u == 0, 0.0, np.arctan(v * w / (u * r)))


def box_field(x, lo, hi, rho=1.0, G=1.0):
    """Acceleration [n,3] and potential [n] at points x [n,3] of a uniform box [lo, hi] of
    density rho (Waldvogel's closed form, as a sum over the 8 corners of antiderivatives):
        int dV / r          = sum_corners s F(u, v, w),
        F = u v ln(w + r) + v w ln(u + r) + w u ln(v + r)
            - u^2/2 atan(v w / (u r)) - v^2/2 atan(w u / (v r)) - w^2/2 atan(u v / (w r)),
        int (x' - x)_1 / r^3 dV = - sum_corners s H(u, v, w),
        H = v ln(w + r) + w ln(v + r) - u atan(v w / (u r))   (and cyclically),
    (u, v, w) the corner relative to x, s = +1 / -1 for an even / odd number of lower
    limits.  a = G rho int (x' - x) / r^3 dV, phi = -G rho int dV / r."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    pot = np.zeros(len(x))
    acc = np.zeros((len(x), 3))
    for cx in (0, 1):
        for cy in (0, 1):
            for cz in (0, 1):
                s = (-1.0) ** (3 - cx - cy - cz)
                u = (hi[0] if cx else lo[0]) - x[:, 0]
                v = (hi[1] if cy else lo[1]) - x[:, 1]
                w = (hi[2] if cz else lo[2]) - x[:, 2]
                r = np.sqrt(u * u + v * v + w * w)
                lu, lv, lw = _log_plus_r(u, r), _log_plus_r(v, r), _log_plus_r(w, r)
                F = (_safe(u * v, lw) + _safe(v * w, lu) + _safe(w * u, lv)
                     - 0.5 * u * u * _atan_term(u, v, w, r) - 0.5 * v * v * _atan_term(v, w, u, r)
                     - 0.5 * w * w * _atan_term(w, u, v, r))
                Hx = _safe(v, lw) + _safe(w, lv) - u * _atan_term(u, v, w, r)
                Hy = _safe(w, lu) + _safe(u, lw) - v * _atan_term(v, w, u, r)
                Hz = _safe(u, lv) + _safe(v, lu) - w * _atan_term(w, u, v, r)
                pot += s * F
                acc[:, 0] -= s * Hx
                acc[:, 1] -= s * Hy
                acc[:, 2] -= s * Hz
    return G * rho * acc, -G * rho * pot


def cube_moments(side, p, rho=1.0):
    """Moments about its centre of a uniform cube: rho prod_d int_{-s/2}^{s/2} t^(a_d) dt,
    zero unless every a_d is even; multi_indices(p) order."""
    h = 0.5 * side

    def one(k):
        return 0.0 if k % 2 else 2.0 * h ** (k + 1) / (k + 1)
    return np.array([rho * one(a[0]) * one(a[1]) * one(a[2]) for a in multi_indices(p)])


_GL = {}


def cube_radial_moment(n, nodes=48):
    """I_n = int over the unit cube [-1/2, 1/2]^3 of |x|^n dV, by Gauss-Legendre product
    quadrature over the octant [0, 1/2]^3 (times 8), whose integrand is smooth but at the
    corner (|x|^n with n >= 1 is n - 1 times differentiable there)."""
    key = (n, nodes)
    if key not in _GL:
        t, w = np.polynomial.legendre.leggauss(nodes)
        t = 0.25 * (t + 1.0)
        w = 0.25 * w
        X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
        W = w[:, None, None] * w[None, :, None] * w[None, None, :]
        _GL[key] = 8.0 * float(np.sum(W * (X * X + Y * Y + Z * Z) ** (0.5 * n)))
    return _GL[key]


# ---- the tree code with the background subtracted ----

def _cell_geometry(key, level, lo, L):
    """Centre and side of the cube of a cell key (leading placeholder bit, 3 bits per level,
    x highest in each triplet)."""
    ix = iy = iz = 0
    k = int(key)
    for lv in range(int(level)):
        t = (k >> (3 * (int(level) - 1 - lv))) & 7
        ix = (ix << 1) | ((t >> 2) & 1)
        iy = (iy << 1) | ((t >> 1) & 1)
        iz = (iz << 1) | (t & 1)
    s = L / (1 << int(level))
    return lo + s * (np.array([ix, iy, iz], dtype=np.float64) + 0.5), s


class BackgroundTree:
    """The tree code on the density contrast (readings above).  force() returns the
    accelerations, potentials and interaction counts."""

    def __init__(self, pos, mass, p=4, leaf_max=64, group_max=128, up=2):
        self.pos = np.ascontiguousarray(pos, dtype=np.float64)
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.p, self.up = int(p), int(up)
        t = Tree(self.pos, self.mass, leaf_max, group_max)
        t.moments(self.p)
        self.tree = t
        self.lo, self.L = t.frame()
        self.rho = float(self.mass.sum()) / self.L ** 3
        cl = t.cells()
        self.key, self.level = cl["key"], cl["level"]
        self.begin, self.count = cl["begin"], cl["count"]
        self.parent, self.nchild = cl["parent"], cl["nchild"]
        nc = len(self.key)
        self.children = [[] for _ in range(nc)]
        for c in range(1, nc):
            self.children[self.parent[c]].append(c)
        # pre-order: a subtree is the range [c, cend[c])
        self.cend = np.arange(1, nc + 1)
        for c in range(nc - 1, 0, -1):
            self.cend[self.parent[c]] = max(self.cend[self.parent[c]], self.cend[c])
        _, self.perm = t.keys()
        mo = t.get_moments()
        self.com, self.mom, self.bmax, self.B1, self.B2 = mo["com"], mo["mom"], mo["bmax"], mo["B1"], mo["B2"]
        gr = t.groups()
        self.gcell, self.gcen, self.gdmax = gr["cell"], gr["centre"], gr["dmax"]
        # cube geometry and contrast expansions of every cell
        p = self.p
        self.centre = np.zeros((nc, 3))
        self.side = np.zeros(nc)
        self.cmom = np.zeros((nc, len(multi_indices(p))))
        self.cQ = np.zeros((nc, 2))
        for c in range(nc):
            z, s = _cell_geometry(self.key[c], self.level[c], self.lo, self.L)
            self.centre[c], self.side[c] = z, s
            idx = self.particles(c)
            x, m = self.pos[idx], self.mass[idx]
            self.cmom[c] = moments(x, m, z, p) - cube_moments(s, p, self.rho)
            self.cQ[c] = self._omitted(moments(x, m, z, p + 2) - cube_moments(s, p + 2, self.rho))

    def _omitted(self, M):
        """(Q_{p+1}, Q_{p+2}) of moments M given to order p + 2."""
        q = np.zeros(2)
        for k, a in enumerate(multi_indices(self.p + 2)):
            n = sum(a)
            if n > self.p:
                f = math.factorial(n) / (math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2]))
                q[n - self.p - 1] += f * M[k] ** 2
        return np.sqrt(q)

    def particles(self, c):
        return self.perm[self.begin[c]:self.begin[c] + self.count[c]]

    def _octant_cube(self, c, o):
        s = 0.5 * self.side[c]
        off = np.array([(o >> 2) & 1, (o >> 1) & 1, o & 1], dtype=np.float64)
        lo = self.centre[c] - self.side[c] * 0.5 + s * off
        return lo + 0.5 * s, s

    def force(self, tol, G=1.0, eps=0.0, record=False):
        """With record=True, self.lists holds per group the set of its interactions:
        ("m", c) matter expansion, ("c", c) contrast expansion, ("e", c, o) empty octant o
        of cell c expanded, ("p", c) leaf c particle by particle, ("b", c) leaf c's cube,
        ("be", c, o) empty octant o of c as a cube; and self.surround[g] the cell of S."""
        p, rho = self.p, self.rho
        self.lists = [] if record else None
        self.surround = np.zeros(len(self.gcell), dtype=np.int64)
        n = len(self.mass)
        acc = np.zeros((n, 3))
        pot = np.zeros(n)
        cnt = dict(m2p_matter=0, m2p_contrast=0, m2p_empty=0, p2p_pairs=0, cube_fields=0)
        sq3 = math.sqrt(3.0)
        e2 = eps * eps
        for g in range(len(self.gcell)):
            gc = int(self.gcell[g])
            gcen, dmax = self.gcen[g], self.gdmax[g]
            sinks = self.particles(gc)
            xs = self.pos[sinks]
            a = np.zeros((len(sinks), 3))
            ph = np.zeros(len(sinks))
            S = gc
            for _ in range(self.up):
                if S > 0:
                    S = int(self.parent[S])
            self.surround[g] = S
            rec = set()
            if record:
                self.lists.append(rec)

            def cube_field(z, s):
                fa, fp = box_field(xs, z - 0.5 * s, z + 0.5 * s, -rho, G)
                cnt["cube_fields"] += len(sinks)
                return fa, fp

            def expand(M, z):
                ai, pi = m2p_points(p, M, z, xs, G, eps)
                a[:] += ai
                ph[:] += pi

            def p2p(c):
                src = self.particles(c)
                d = self.pos[src][None, :, :] - xs[:, None, :]
                r2 = np.sum(d * d, axis=-1) + e2
                same = sinks[:, None] == src[None, :]
                with np.errstate(divide="ignore"):
                    inv = np.where(same | (r2 == 0), 0.0, 1.0 / np.sqrt(r2))
                a[:] += G * np.einsum("ij,ijd,j->id", inv ** 3, d, self.mass[src])
                ph[:] -= G * (inv @ self.mass[src])
                cnt["p2p_pairs"] += int(np.sum(~same))

            def contrast_ok(z, s, Q):
                d = float(np.linalg.norm(z - gcen)) - dmax
                b = 0.5 * sq3 * s
                if not d > b:
                    return False
                E = G / (1.0 - b / d) ** 2 * ((p + 2) * Q[0] / d ** (p + 3) + (p + 3) * Q[1] / d ** (p + 4))
                return E <= tol

            def empty_octants(c):
                have = {int(self.key[k]) & 7 for k in self.children[c]}
                for o in range(8):
                    if o in have:
                        continue
                    z, s = self._octant_cube(c, o)
                    if contrast_ok(z, s, self._omitted(-cube_moments(s, p + 2, rho))):
                        expand(-cube_moments(s, p, rho), z)
                        cnt["m2p_empty"] += len(sinks)
                        rec.add(("e", int(c), o))
                    else:
                        rec.add(("be", int(c), o))
                        fa, fp = cube_field(z, s)
                        a[:] += fa
                        ph[:] += fp

            stack = [0]
            while stack:
                c = stack.pop()
                leaf = self.nchild[c] == 0
                inside = S <= c < self.cend[S]
                if c <= gc < self.cend[c]:  # the group's cell or an ancestor: open
                    if leaf:
                        p2p(c)
                        rec.add(("p", int(c)))
                    else:
                        stack.extend(self.children[c])
                        if not inside:
                            empty_octants(c)
                    continue
                if gc < c < self.cend[gc]:  # inside the group's cell: d <= 0, never expanded
                    if leaf:
                        p2p(c)
                        rec.add(("p", int(c)))
                    else:
                        stack.extend(self.children[c])
                    continue
                if inside:  # the plain method: matter about the centre of mass
                    d = float(np.linalg.norm(self.com[c] - gcen)) - dmax
                    b = self.bmax[c]
                    if d > b and mac_bound(d, b, self.B1[c], self.B2[c], p, G) <= tol:
                        expand(self.mom[c], self.com[c])
                        cnt["m2p_matter"] += len(sinks)
                        rec.add(("m", int(c)))
                    elif leaf:
                        p2p(c)
                        rec.add(("p", int(c)))
                    else:
                        stack.extend(self.children[c])
                    continue
                z, s = self.centre[c], self.side[c]
                if contrast_ok(z, s, self.cQ[c]):
                    expand(self.cmom[c], z)
                    cnt["m2p_contrast"] += len(sinks)
                    rec.add(("c", int(c)))
                elif leaf:
                    p2p(c)
                    rec.add(("p", int(c)))
                    rec.add(("b", int(c)))
                    fa, fp = cube_field(z, s)
                    a[:] += fa
                    ph[:] += fp
                else:
                    stack.extend(self.children[c])
                    empty_octants(c)
            # the surrounding cube's background
            fa, fp = cube_field(self.centre[S], self.side[S])
            a += fa
            ph += fp
            acc[sinks] = a
            pot[sinks] = ph
        return acc, pot, cnt

    def exact(self, G=1.0, eps=0.0):
        """The quantity itself: the direct sum minus the root cube's analytic field."""
        a, ph = direct(self.pos, self.mass, G, eps)
        fa, fp = box_field(self.pos, self.lo, self.lo + self.L, -self.rho, G)
        return a + fa, ph + fp
