"""Periodic boundaries for the CPU oracle (Sec. "Boundary Conditions").

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU legs may
use it; the CUDA path never does, and it shares no code with the CUDA library.

The paper treats a periodic cube of side L by the lattice-sum approach (Nijboer and De
Wette, in the Cartesian form of Challacombe et al.): the images within ws cubes of the
central one (ws = 2: the central cube and its 124 neighbours) interact through the tree,
and every farther image through one local expansion about the centre of the cube, whose
coefficients -- lattice sums of the derivatives of the Green's function, the same for
every replica -- are computed once.  The paper uses p = 8 and ws = 2.

Conventions (not stated in the paper; those of Ewald summation): a uniform neutralising
background (the mean density is subtracted, so that the lattice sum converges) and a
conducting (tin-foil) boundary at infinity.  With V = L^3 and any splitting parameter
alpha > 0, the periodic Green's function is

    psi(r) = sum_n erfc(alpha |r + nL|) / |r + nL|
             + (4 pi / V) sum_{k != 0} exp(-k^2 / 4 alpha^2) / k^2 cos(k . r) - pi / (alpha^2 V),

k = 2 pi m / L; it does not depend on alpha.  Accelerations and potentials:

    a_i   = G sum_j m_j grad psi(x_i - x_j)           (the j = i term vanishes)
    phi_i = -G [ sum_{j != i} m_j psi(x_i - x_j) + m_i psi_self ],
    psi_self = lim_{r -> 0} (psi(r) - 1/r).

The far part psi_far(r) = psi(r) - sum_{|n|_inf <= ws} 1/|r + nL| is smooth where the
method evaluates it (|r_d| < L) and is expanded about 0:

    phi_far,i = -G sum_beta (x_i - c)^beta / beta! * L_beta,
    L_beta    = sum_alpha (-1)^|alpha| / alpha! M_alpha(c) D^(alpha + beta) psi_far(0),

with M_alpha(c) the moments of all particles about the centre c of the cube.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc, gammainc, gammaincc

from . import multi_indices


def _images(nmax):
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    return n


def _kvectors(L, kmax):
    m = _images(kmax)
    m = m[np.any(m != 0, axis=1)]
    return 2.0 * math.pi * m / L


def ewald(pos, mass, L, G=1.0, alpha=None, nreal=3, kmax=12):
    """Exact periodic accelerations [N,3] and potentials [N] (definitions above) by direct
    Ewald summation: real-space images |n|_inf <= nreal, reciprocal vectors |m|_inf <= kmax.
    Positions are taken modulo L (their frame does not matter)."""
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    n = len(mass)
    V = L ** 3
    if alpha is None:
        alpha = 3.5 / L
    acc = np.zeros((n, 3))
    pot = np.zeros(n)
    # real space: all pairs (i, j) and images; the i == j, n == 0 term is the self term
    for s in _images(nreal) * L:
        d = pos[:, None, :] - pos[None, :, :] + s  # x_i - x_j + nL
        r = np.sqrt(np.sum(d * d, axis=-1))
        with np.errstate(divide="ignore", invalid="ignore"):
            ec = erfc(alpha * r) / r
            g = ec / (r * r) + 2.0 * alpha / math.sqrt(math.pi) * np.exp(-(alpha * r) ** 2) / (r * r)
        if not np.any(s):
            np.fill_diagonal(ec, 0.0)
            np.fill_diagonal(g, 0.0)
        pot -= G * (ec @ mass)
        # grad of erfc(alpha r)/r = -d g
        acc -= G * np.einsum("ij,ijd,j->id", g, d, mass)
    # self term: lim (erfc(alpha r) - 1)/r = -2 alpha / sqrt(pi)
    pot -= G * mass * (-2.0 * alpha / math.sqrt(math.pi))
    # reciprocal space
    k = _kvectors(L, kmax)
    k2 = np.sum(k * k, axis=1)
    w = 4.0 * math.pi / V * np.exp(-k2 / (4.0 * alpha * alpha)) / k2
    ph = pos @ k.T                                 # [N, K]
    c, sn = np.cos(ph), np.sin(ph)
    S_c, S_s = mass @ c, mass @ sn                 # structure factor: sum_j m_j e^{i k x_j}
    # sum_j m_j cos(k (x_i - x_j)) = c_i S_c + s_i S_s ; sum_j m_j sin(k (x_i - x_j)) = s_i S_c - c_i S_s
    pot -= G * ((c * S_c + sn * S_s) @ w)
    acc -= G * (((sn * S_c - c * S_s) * w) @ k)
    # the constant
    pot -= G * mass.sum() * (-math.pi / (alpha * alpha * V))
    return acc, pot


def _cfac(i, l):
    return math.factorial(i) / (math.factorial(l) * math.factorial(i - 2 * l))


def _radial_derivs(F, R, order):
    """d^g F(|r|^2) at r = R for every multi-index g, |g| <= order, summed over a set of
    points R [K,3], given F [order+1, K] with F[m] = F^(m)(|R|^2):
        d^g F = sum_l prod_d c(g_d, l_d) (2 R_d)^(g_d - 2 l_d) F^(|g| - |l|)."""
    P = [[(2.0 * R[:, d]) ** e for e in range(order + 1)] for d in range(3)]
    out = {}
    for g in multi_indices(order):
        t = 0.0
        for l0 in range(g[0] // 2 + 1):
            for l1 in range(g[1] // 2 + 1):
                for l2 in range(g[2] // 2 + 1):
                    m = g[0] + g[1] + g[2] - (l0 + l1 + l2)
                    cf = _cfac(g[0], l0) * _cfac(g[1], l1) * _cfac(g[2], l2)
                    t += cf * float(np.sum(P[0][g[0] - 2 * l0] * P[1][g[1] - 2 * l1] * P[2][g[2] - 2 * l2] * F[m]))
        out[g] = t
    return out


def _radial_split(s, alpha, order):
    """(-1/s d/ds)^m of erfc(alpha s)/s and of erf(alpha s)/s, m = 0..order (s an array):
    (2m - 1)!! s^-(2m+1) times the regularised upper, resp. lower, incomplete gamma
    function of (m + 1/2, alpha^2 s^2) -- no difference of nearly equal terms, which the
    recurrence from erfc(alpha s)/s or 1/s - erfc(alpha s)/s would take at high m."""
    x = (alpha * s) ** 2
    up, lo = [], []
    for m in range(order + 1):
        base = _dfact(2 * m - 1) / s ** (2 * m + 1)
        up.append(base * gammaincc(m + 0.5, x))
        lo.append(base * gammainc(m + 0.5, x))
    return np.array(up), np.array(lo)


def _dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def lattice_coefficients(L, order, ws=2, alpha=None, nreal=6, kmax=4):
    """D^g psi_far(0) for every |g| <= order (dict keyed by multi-index), psi_far = psi minus
    the images within ws, by Ewald splitting:
        psi_far = - sum_{|n|<=ws} erf(alpha |r+nL|)/|r+nL| + sum_{|n|>ws} erfc(alpha |r+nL|)/|r+nL|
                  + reciprocal sum + constant,
    each radial term differentiated through F^(m)(u) = (-1/2)^m (-1/s d/ds)^m f(s) with the
    incomplete-gamma forms of _radial_split; the n = 0 erf term from its Taylor series,
    erf(alpha s)/s = (2 alpha/sqrt(pi)) sum_m (-1)^m alpha^(2m) s^(2m) / (m! (2m+1)).
    alpha = 1/L by default: the split terms then stay of the size of the result even at
    order 17 (a large alpha makes them grow like alpha^(2m+1) and cancel); the real-space
    sum runs to |n|_inf <= nreal (erfc(6) ~ 2e-17), the reciprocal one to |m|_inf <= kmax."""
    if alpha is None:
        alpha = 1.0 / L
    V = L ** 3
    D = {g: 0.0 for g in multi_indices(order)}
    # n = 0: - erf(alpha s)/s, only even g contribute
    F0 = [-(2 * alpha / math.sqrt(math.pi)) * (-1) ** m * alpha ** (2 * m) / (2 * m + 1) for m in range(order + 1)]
    for g in D:
        if all(x % 2 == 0 for x in g):
            D[g] += _cfac(g[0], g[0] // 2) * _cfac(g[1], g[1] // 2) * _cfac(g[2], g[2] // 2) * F0[(g[0] + g[1] + g[2]) // 2]
    n = _images(nreal)
    n = n[np.any(n != 0, axis=1)]
    R = n * L
    s = np.sqrt(np.sum(R * R, axis=1))
    up, lo = _radial_split(s, alpha, order)
    near = np.max(np.abs(n), axis=1) <= ws
    F = np.array([(-0.5) ** m * np.where(near, -lo[m], up[m]) for m in range(order + 1)])
    for g, v in _radial_derivs(F, R, order).items():
        D[g] += v
    # reciprocal space: d^g cos(k.r) at 0 = (-1)^(|g|/2) k^g for even |g|, 0 for odd
    k = _kvectors(L, kmax)
    k2 = np.sum(k * k, axis=1)
    w = 4.0 * math.pi / V * np.exp(-k2 / (4.0 * alpha * alpha)) / k2
    for g in D:
        ng = g[0] + g[1] + g[2]
        if ng % 2 == 0:
            D[g] += (-1) ** (ng // 2) * float(np.sum(w * k[:, 0] ** g[0] * k[:, 1] ** g[1] * k[:, 2] ** g[2]))
    D[(0, 0, 0)] += -math.pi / (alpha * alpha * V)
    return D


def near_images_direct(pos, mass, L, G=1.0, ws=2):
    """Plain 1/r sum over the images within ws of every particle (its own images included,
    the n = 0 self pair excluded): the part of the periodic force the tree approximates."""
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    n = len(mass)
    acc = np.zeros((n, 3))
    pot = np.zeros(n)
    for s in _images(ws) * L:
        d = pos[None, :, :] + s - pos[:, None, :]   # x_j + nL - x_i
        r2 = np.sum(d * d, axis=-1)
        if not np.any(s):
            np.fill_diagonal(r2, np.inf)
        inv = 1.0 / np.sqrt(r2)
        pot -= G * (inv @ mass)
        acc += G * np.einsum("ij,ijd,j->id", inv ** 3, d, mass)
    return acc, pot


def far_field(pos, mass, L, lo, p=8, ws=2, G=1.0, D=None):
    """The local expansion of every image farther than ws, at every particle: moments of
    all particles about the cube's centre c = lo + L/2 to order p, the local coefficients
    L_beta to order p + 1 (so that the acceleration is of order p), D from
    lattice_coefficients(L, 2p + 1, ws).  Returns (acc [N,3], pot [N])."""
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    c = np.asarray(lo, dtype=np.float64) + 0.5 * L
    if D is None:
        D = lattice_coefficients(L, 2 * p + 1, ws)
    y = pos - c
    fac = math.factorial
    M = {a: float(np.sum(mass * y[:, 0] ** a[0] * y[:, 1] ** a[1] * y[:, 2] ** a[2])) for a in multi_indices(p)}
    Lb = {}
    for b in multi_indices(p + 1):
        t = 0.0
        for a, Ma in M.items():
            t += (-1) ** (a[0] + a[1] + a[2]) / (fac(a[0]) * fac(a[1]) * fac(a[2])) * Ma * D[(a[0] + b[0], a[1] + b[1], a[2] + b[2])]
        Lb[b] = t
    pot = np.zeros(len(mass))
    acc = np.zeros((len(mass), 3))
    for b, v in Lb.items():
        bf = fac(b[0]) * fac(b[1]) * fac(b[2])
        pot -= G * v * y[:, 0] ** b[0] * y[:, 1] ** b[1] * y[:, 2] ** b[2] / bf
        for d in range(3):
            if b[d] == 0:
                continue
            e = list(b)
            e[d] -= 1
            ef = fac(e[0]) * fac(e[1]) * fac(e[2])
            acc[:, d] += G * v * y[:, 0] ** e[0] * y[:, 1] ** e[1] * y[:, 2] ** e[2] / ef
    return acc, pot


def tree_force(pos, mass, L, lo, p=8, tol=1e-6, ws=2, p_far=8, G=1.0, eps=0.0, D=None,
               leaf_max=64, group_max=128):
    """The paper's periodic force: the tree over the central cube and its images within ws
    (open-boundary tree code with the images as further sources), plus the far images
    through the local expansion of order p_far.  Positions inside [lo, lo + L)^3."""
    from . import Tree
    t = Tree(pos, mass, leaf_max, group_max)
    t.periodic(L, ws)
    t.moments(p)
    t.traverse(tol, G)
    an, pn = t.force(G, eps)
    af, pf = far_field(pos, mass, L, lo, p=p_far, ws=ws, G=G, D=D)
    return an + af, pn + pf
