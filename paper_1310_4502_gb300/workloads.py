"""Seeded synthetic particle sets for the tree-force path.

This module only draws inputs (positions, masses, loss weights).  It holds
none of the force method's arithmetic, so both the CPU oracle and the CUDA
path can consume its arrays without sharing any code with each other.

All generators use numpy's PCG64 (``numpy.random.default_rng``) and return
float64 arrays: positions ``[N, 3]`` (row-major), masses ``[N]``.

Recipes (the paper's cosmological initial conditions and production runs are
not available, so these stand in for them):

* ``plummer``: a Plummer sphere (total mass 1, scale radius a), radii
  truncated at ``rmax * a``.  The enclosed-mass fraction X is drawn uniform in
  ``[0, X(rmax)]`` and inverted, ``r = a (X^{-2/3} - 1)^{-1/2}``; directions
  are isotropic.
* ``clustered``: 64 Plummer spheres holding half the particles (centres
  uniform in the unit cube, scale radii log-uniform in [0.005, 0.05], each
  truncated at 20 scale radii) plus a uniform background in the unit cube;
  the concatenation is randomly permuted.
* ``zeldovich``: a regular lattice ``q = (i + 1/2)/n`` displaced by a Gaussian
  random field with power spectrum P(k) ~ k^-2 (amplitude ~ k^-1), cut at the
  lattice Nyquist wavenumber ``pi n``, k=0 removed, displacement
  ``psi_k = i k delta_k / k^2``, rescaled so that the rms |psi| is 0.2 lattice
  spacings.  No periodic wrap is applied.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Workload",
    "plummer",
    "clustered",
    "zeldovich",
    "loss_weights",
    "make",
    "WORKLOADS",
]


@dataclass
class Workload:
    name: str
    pos: np.ndarray   # [N, 3] float64
    mass: np.ndarray  # [N] float64
    eps: float        # Plummer softening length
    p: int            # multipole order used with this workload
    tol: float        # absolute acceleration tolerance of the acceptance test

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def plummer_xmax(rmax: float) -> float:
    """Enclosed-mass fraction of an untruncated Plummer sphere inside rmax (in units of a)."""
    return rmax ** 3 / (rmax * rmax + 1.0) ** 1.5


def plummer(n: int, seed: int = 0, a: float = 1.0, rmax: float = 20.0,
            rng: np.random.Generator | None = None) -> np.ndarray:
    """Positions of an n-particle Plummer sphere of scale radius ``a`` centred at 0."""
    if rng is None:
        rng = np.random.default_rng(seed)
    xmax = plummer_xmax(rmax)
    x = rng.uniform(0.0, xmax, n)
    x = np.maximum(x, np.finfo(np.float64).tiny)
    r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    return r[:, None] * _isotropic(rng, n)


def clustered(n: int, seed: int = 0, nsphere: int = 64) -> np.ndarray:
    """Clustered box: ``nsphere`` Plummer spheres hold n/2 particles, n/2 uniform background."""
    rng = np.random.default_rng(seed)
    n_cl = n // 2
    per = n_cl // nsphere
    centres = rng.uniform(0.0, 1.0, (nsphere, 3))
    radii = np.exp(rng.uniform(math.log(0.005), math.log(0.05), nsphere))
    parts = []
    for s in range(nsphere):
        cnt = per if s < nsphere - 1 else n_cl - per * (nsphere - 1)
        parts.append(centres[s] + plummer(cnt, a=radii[s], rmax=20.0, rng=rng))
    parts.append(rng.uniform(0.0, 1.0, (n - n_cl, 3)))
    pos = np.concatenate(parts, axis=0)
    return pos[rng.permutation(n)]


def zeldovich(ngrid: int, seed: int = 0, rms_disp: float = 0.2) -> np.ndarray:
    """Lattice of ngrid^3 particles in the unit cube with a k^-2 Zel'dovich displacement."""
    rng = np.random.default_rng(seed)
    n = ngrid
    dx = 1.0 / n
    noise = rng.standard_normal((n, n, n))
    nk = np.fft.rfftn(noise)
    del noise
    kf = 2.0 * math.pi * np.fft.fftfreq(n, d=dx)
    kr = 2.0 * math.pi * np.fft.rfftfreq(n, d=dx)
    kx = kf[:, None, None]
    ky = kf[None, :, None]
    kz = kr[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    kmag = np.sqrt(k2)
    amp = 1.0 / kmag                      # delta_k ~ k^-1  <=>  P(k) ~ k^-2
    amp[kmag > math.pi * n] = 0.0         # spherical cut at the lattice Nyquist wavenumber
    amp[0, 0, 0] = 0.0
    delta = nk * amp
    del nk, amp
    psi = np.empty((n, n, n, 3))
    for d, kd in enumerate((kx, ky, kz)):
        psi[..., d] = np.fft.irfftn(1j * kd * delta / k2, s=(n, n, n))
    del delta
    rms = math.sqrt(float(np.mean(np.sum(psi * psi, axis=-1))))
    psi *= (rms_disp * dx) / rms
    q = (np.arange(n) + 0.5) * dx
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    pos = np.stack([qx, qy, qz], axis=-1) + psi
    return np.ascontiguousarray(pos.reshape(-1, 3))


def loss_weights(n: int, seed: int = 1) -> np.ndarray:
    """Weights w_i ~ N(0,1)^3 of the loss L = sum_i w_i . a_i."""
    return np.random.default_rng(seed).standard_normal((n, 3))


def make(name: str) -> Workload:
    """Named workloads (sizes and parameters as in the benchmark table of the design notes)."""
    if name == "plummer4096":
        n = 4096
        return Workload(name, plummer(n, seed=0), np.full(n, 1.0 / n), 0.01, 4, 1e-4)
    if name.startswith("clustered"):
        # clustered<log2 N>, e.g. clustered20 -> N = 2^20
        n = 1 << int(name[len("clustered"):])
        return Workload(name, clustered(n, seed=0), np.full(n, 1.0 / n), 1e-4, 4, 1e-4)
    if name.startswith("zeldovich"):
        g = int(name[len("zeldovich"):])
        n = g ** 3
        return Workload(name, zeldovich(g, seed=0), np.full(n, 1.0 / n), 0.02 / g, 6, 1e-4)
    raise KeyError(name)


WORKLOADS = ("plummer4096", "clustered20", "zeldovich128", "clustered18", "zeldovich256")
