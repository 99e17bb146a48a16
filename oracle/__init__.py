"""CPU FP64 oracle for the hashed oct-tree gravity path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and it imports nothing from there.

The arithmetic lives in ``hot_oracle.c`` (plain C, OpenMP over independent
sinks, built with ``-O2 -ffp-contract=off``); this module only marshals numpy
arrays through ctypes.  Every function cites the part of the paper it follows
in the C source.

Parity pins (tests/test_oracle.py) tie each function to something other than
itself: closed forms (two-body, uniform-sphere interior, truncated Plummer
profile), invariants (third law, translation invariance, linearity in mass),
brute force on tiny inputs, and convergence of the tree towards the direct
sum as p grows and the tolerance tightens.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hot_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
            "-fPIC", "-shared", _SRC, "-o", tmp, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_nthreads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_direct.argtypes = [C.c_int64, _d, _d, C.c_double, C.c_double, C.c_int, C.c_int64,
                                 C.c_void_p, _d, C.c_void_p]
        L.orc_direct_grad.argtypes = [C.c_int64, _d, _d, C.c_double, C.c_double, C.c_int, _d,
                                      C.c_void_p, _d, _d]
        L.orc_soft_eval.restype = C.c_int
        L.orc_soft_eval.argtypes = [C.c_int, C.c_double, C.c_double, _d]
        L.orc_tree_softening.restype = C.c_int
        L.orc_tree_softening.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.orc_tree_order_range.restype = C.c_int
        L.orc_tree_order_range.argtypes = [C.c_void_p, C.c_int]
        L.orc_tree_list_orders.argtypes = [C.c_void_p, _i32]
        L.orc_tree_periodic.restype = C.c_int
        L.orc_tree_periodic.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.orc_tree_list_images.argtypes = [C.c_void_p, _i32, _i32]
        L.orc_bbox.argtypes = [C.c_int64, _d, _d, C.POINTER(C.c_double)]
        L.orc_keys.argtypes = [C.c_int64, _d, _d, C.c_double, _u64]
        L.orc_sort.argtypes = [C.c_int64, _u64, _i64]
        L.orc_m2p.argtypes = [C.c_int, _d, _d, C.c_double, C.c_double, _d,
                              C.POINTER(C.c_double)]
        L.orc_m2p_points.argtypes = [C.c_int, _d, _d, C.c_int64, _d, C.c_double, C.c_double, _d, _d]
        L.orc_moments.argtypes = [C.c_int64, _d, _d, _d, C.c_int, _d]
        L.orc_mac_bound.restype = C.c_double
        L.orc_mac_bound.argtypes = [C.c_double] * 4 + [C.c_int, C.c_double]
        L.orc_tree_new.restype = C.c_void_p
        L.orc_tree_new.argtypes = [C.c_int64, _d, _d, C.c_int, C.c_int]
        L.orc_tree_free.argtypes = [C.c_void_p]
        L.orc_tree_info.argtypes = [C.c_void_p, _i64]
        L.orc_tree_frame.argtypes = [C.c_void_p, _d, C.POINTER(C.c_double)]
        L.orc_tree_keys.argtypes = [C.c_void_p, _u64, _i64]
        L.orc_tree_cells.argtypes = [C.c_void_p, _u64, _i32, _i64, _i64, _i32, _i32]
        L.orc_tree_groups.argtypes = [C.c_void_p, _i32, _d, _d]
        L.orc_tree_moments.restype = C.c_int
        L.orc_tree_moments.argtypes = [C.c_void_p, C.c_int]
        L.orc_tree_get_moments.argtypes = [C.c_void_p, _d, _d, _d, _d, _d, _d]
        L.orc_tree_traverse.restype = C.c_int
        L.orc_tree_traverse.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.orc_tree_traverse_groups.restype = C.c_int
        L.orc_tree_traverse_groups.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int64,
                                               _i64]
        L.orc_tree_list_sizes.argtypes = [C.c_void_p, _i64]
        L.orc_tree_lists.argtypes = [C.c_void_p, _i32, _i32, _i32]
        L.orc_tree_force.restype = C.c_int
        L.orc_tree_force.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int64,
                                     C.c_void_p, _d, C.c_void_p]
        L.orc_frozen_force.restype = C.c_int
        L.orc_frozen_force.argtypes = [C.c_void_p, _d, _d, C.c_double, C.c_double, _d, C.c_void_p]
        L.orc_frozen_loss.restype = C.c_double
        L.orc_frozen_loss.argtypes = [C.c_void_p, _d, _d, C.c_double, C.c_double, _d,
                                      C.c_void_p, C.c_int64]
        _lib = L
    return _lib


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def nthreads() -> int:
    return int(lib().orc_nthreads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def ncomp(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def multi_indices(p: int) -> list[tuple[int, int, int]]:
    """Moment component order: degree ascending, then i descending, then j descending."""
    out = []
    for n in range(p + 1):
        for i in range(n, -1, -1):
            for j in range(n - i, -1, -1):
                out.append((i, j, n - i - j))
    return out


# Force smoothing kinds (Sec. "Force Smoothing"): Plummer, or the K1 compensating kernel
# of support eps (its density is a stated reading; see hot_oracle.c).
SOFT = {"plummer": 0, "k1": 1, "spline": 2}


def soft_kernel(soft, eps, r):
    """(f, f2, psi) of one pair at separation r: a = G m f d, phi = -G m psi, f2 = 2 df/d(r^2);
    None for a skipped pair."""
    out = np.zeros(3)
    if not lib().orc_soft_eval(SOFT[soft], float(eps), float(r), out):
        return None
    return tuple(out)


def direct(pos, mass, G=1.0, eps=0.0, sinks=None, soft="plummer"):
    """O(N^2) softened direct sum; returns (acc [n,3], pot [n]) for the sinks (default all)."""
    pos, mass = _c(pos), _c(mass)
    n = len(mass) if sinks is None else len(sinks)
    sk = None if sinks is None else _c(sinks, np.int64)
    acc = np.zeros((n, 3))
    pot = np.zeros(n)
    lib().orc_direct(len(mass), pos, mass, G, eps, SOFT[soft], n, _ptr(sk), acc, _ptr(pot))
    return acc, pot


def direct_grad(pos, mass, w, v=None, G=1.0, eps=0.0, soft="plummer"):
    """Analytic gradient of L = sum w.a + sum v phi of the direct sum: (dL/dx [N,3], dL/dm [N])."""
    pos, mass, w = _c(pos), _c(mass), _c(w)
    vv = None if v is None else _c(v)
    gx = np.zeros_like(pos)
    gm = np.zeros_like(mass)
    lib().orc_direct_grad(len(mass), pos, mass, G, eps, SOFT[soft], w, _ptr(vv), gx, gm)
    return gx, gm


def bbox(pos):
    pos = _c(pos)
    lo = np.zeros(3)
    L = C.c_double()
    lib().orc_bbox(len(pos), pos, lo, C.byref(L))
    return lo, L.value


def keys(pos, lo, L):
    pos = _c(pos)
    out = np.zeros(len(pos), dtype=np.uint64)
    lib().orc_keys(len(pos), pos, _c(lo), float(L), out)
    return out


def sort(keys_):
    keys_ = _c(keys_, np.uint64)
    perm = np.zeros(len(keys_), dtype=np.int64)
    lib().orc_sort(len(keys_), keys_, perm)
    return perm


def m2p(p, M, R, G=1.0, eps=0.0):
    acc = np.zeros(3)
    pot = C.c_double()
    lib().orc_m2p(int(p), _c(M), _c(R), G, eps, acc, C.byref(pot))
    return acc, pot.value


def m2p_points(p, M, z, x, G=1.0, eps=0.0):
    """m2p at every point of x [n,3] (R = x - z): (acc [n,3], pot [n])."""
    x = _c(x)
    acc = np.zeros((len(x), 3))
    pot = np.zeros(len(x))
    lib().orc_m2p_points(int(p), _c(M), _c(z), len(x), x, G, eps, acc, pot)
    return acc, pot


def moments(pos, mass, z, p):
    M = np.zeros(ncomp(p))
    lib().orc_moments(len(mass), _c(pos), _c(mass), _c(z), int(p), M)
    return M


def mac_bound(d, b, B1, B2, p, G=1.0):
    return float(lib().orc_mac_bound(d, b, B1, B2, int(p), G))


class Tree:
    """Oracle tree: keys, stable sort, pre-order cells, groups, moments, lists, forces."""

    def __init__(self, pos, mass, leaf_max=64, group_max=128):
        self.pos = _c(pos)
        self.mass = _c(mass)
        self.leaf_max, self.group_max = leaf_max, group_max
        self._h = lib().orc_tree_new(len(self.mass), self.pos, self.mass, leaf_max, group_max)
        if not self._h:
            raise ValueError("orc_tree_new rejected its arguments")
        self.p = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_tree_free(h)
            self._h = None

    def info(self):
        out = np.zeros(6, dtype=np.int64)
        lib().orc_tree_info(self._h, out)
        return dict(N=int(out[0]), ncell=int(out[1]), ngroup=int(out[2]), nleaf=int(out[3]),
                    maxlevel=int(out[4]), p=int(out[5]))

    def frame(self):
        lo = np.zeros(3)
        L = C.c_double()
        lib().orc_tree_frame(self._h, lo, C.byref(L))
        return lo, L.value

    def keys(self):
        n = len(self.mass)
        k = np.zeros(n, dtype=np.uint64)
        p = np.zeros(n, dtype=np.int64)
        lib().orc_tree_keys(self._h, k, p)
        return k, p

    def cells(self):
        nc = self.info()["ncell"]
        key = np.zeros(nc, dtype=np.uint64)
        level = np.zeros(nc, dtype=np.int32)
        begin = np.zeros(nc, dtype=np.int64)
        count = np.zeros(nc, dtype=np.int64)
        parent = np.zeros(nc, dtype=np.int32)
        nchild = np.zeros(nc, dtype=np.int32)
        lib().orc_tree_cells(self._h, key, level, begin, count, parent, nchild)
        return dict(key=key, level=level, begin=begin, count=count, parent=parent, nchild=nchild)

    def groups(self):
        ng = self.info()["ngroup"]
        cell = np.zeros(ng, dtype=np.int32)
        cen = np.zeros((ng, 3))
        dmax = np.zeros(ng)
        lib().orc_tree_groups(self._h, cell, cen, dmax)
        return dict(cell=cell, centre=cen, dmax=dmax)

    def moments(self, p):
        if lib().orc_tree_moments(self._h, int(p)) != 0:
            raise ValueError("bad order")
        self.p = int(p)

    def get_moments(self):
        nc = self.info()["ncell"]
        k = ncomp(self.p)
        out = dict(mass=np.zeros(nc), com=np.zeros((nc, 3)), mom=np.zeros((nc, k)),
                   bmax=np.zeros(nc), B1=np.zeros(nc), B2=np.zeros(nc))
        lib().orc_tree_get_moments(self._h, out["mass"], out["com"], out["mom"], out["bmax"],
                                   out["B1"], out["B2"])
        return out

    def softening(self, soft, eps):
        """Force smoothing of the lists and forces ("plummer" default, or "k1" / "spline" with
        support eps: the lists then accept a cell only if d >= b_max + eps); set before
        traverse."""
        if lib().orc_tree_softening(self._h, SOFT[soft], float(eps)) != 0:
            raise ValueError("bad softening")

    def order_range(self, p_lo):
        """Per-interaction order selection (after moments(p)): every accepted cell is
        evaluated at the lowest order in [p_lo, p] whose error bound meets the tolerance;
        p_lo=None restores the fixed order p."""
        if lib().orc_tree_order_range(self._h, -1 if p_lo is None else int(p_lo)) != 0:
            raise ValueError("bad order range")

    def periodic(self, L, ws=2):
        """Periodic images (Sec. "Boundary Conditions"): every group also traverses the tree
        shifted by n L, |n|_inf <= ws; the forces are then the near field of the periodic
        problem (oracle.periodic adds the far field).  L = 0 restores open boundaries."""
        if lib().orc_tree_periodic(self._h, float(L), int(ws)) != 0:
            raise ValueError("bad periodic box")

    def traverse(self, tol, G=1.0, groups=None):
        if groups is None:
            r = lib().orc_tree_traverse(self._h, float(tol), float(G))
        else:
            gs = _c(groups, np.int64)
            r = lib().orc_tree_traverse_groups(self._h, float(tol), float(G), len(gs), gs)
        if r != 0:
            raise ValueError("traverse needs moments and tol > 0")

    def lists(self):
        """CSR lists per group: dict(m2p=(offsets, cells), p2p=(offsets, leaves), border=...)."""
        ng = self.info()["ngroup"]
        sz = np.zeros((ng, 3), dtype=np.int64)
        lib().orc_tree_list_sizes(self._h, sz.reshape(-1))
        off = np.zeros((ng + 1, 3), dtype=np.int64)
        off[1:] = np.cumsum(sz, axis=0)
        m2p = np.zeros(off[-1, 0], dtype=np.int32)
        p2p = np.zeros(off[-1, 1], dtype=np.int32)
        bor = np.zeros(off[-1, 2], dtype=np.int32)
        lib().orc_tree_lists(self._h, m2p, p2p, bor)
        order = np.zeros(off[-1, 0], dtype=np.int32)
        lib().orc_tree_list_orders(self._h, order)
        mimg = np.zeros(off[-1, 0], dtype=np.int32)
        pimg = np.zeros(off[-1, 1], dtype=np.int32)
        lib().orc_tree_list_images(self._h, mimg, pimg)
        return dict(m2p=(off[:, 0].copy(), m2p), p2p=(off[:, 1].copy(), p2p),
                    border=(off[:, 2].copy(), bor), m2p_order=order, m2p_image=mimg, p2p_image=pimg)

    def force(self, G=1.0, eps=0.0, groups=None):
        n = len(self.mass)
        acc = np.zeros((n, 3))
        pot = np.zeros(n)
        gs = None if groups is None else _c(groups, np.int64)
        r = lib().orc_tree_force(self._h, G, eps, 0 if gs is None else len(gs), _ptr(gs), acc,
                                 _ptr(pot))
        if r == -2:
            raise ValueError("K1 forces need the eps the lists were built with")
        if r != 0:
            raise ValueError("force needs lists")
        return acc, pot

    def frozen_force(self, pos, mass, G=1.0, eps=0.0):
        """Force with this tree's lists and centres frozen, moments from the given particles."""
        n = len(self.mass)
        acc = np.zeros((n, 3))
        pot = np.zeros(n)
        r = lib().orc_frozen_force(self._h, _c(pos), _c(mass), G, eps, acc, _ptr(pot))
        if r == -2:
            raise ValueError("K1 forces need the eps the lists were built with")
        if r != 0:
            raise ValueError("frozen_force needs lists")
        return acc, pot

    def frozen_loss(self, pos, mass, w, v=None, G=1.0, eps=0.0, k=-1):
        vv = None if v is None else _c(v)
        return float(lib().orc_frozen_loss(self._h, _c(pos), _c(mass), G, eps, _c(w), _ptr(vv),
                                           int(k)))


def frozen_leapfrog(trees, x0, v0, mass, dt, G=1.0, eps=0.0):
    """Kick-drift-kick leapfrog (Sec. "Time Integration": v += dt/2 a; x += dt v;
    v += dt/2 a) whose force at step point k uses trees[k] frozen (its lists and
    centres), moments recomputed from the current particles.  len(trees) = steps + 1."""
    x = np.array(x0, dtype=np.float64, copy=True)
    v = np.array(v0, dtype=np.float64, copy=True)
    a, _ = trees[0].frozen_force(x, mass, G, eps)
    for k in range(1, len(trees)):
        v += 0.5 * dt * a
        x += dt * v
        a, _ = trees[k].frozen_force(x, mass, G, eps)
        v += 0.5 * dt * a
    return x, v


def tree_force(pos, mass, p=4, tol=1e-4, eps=0.0, G=1.0, leaf_max=64, group_max=128, soft="plummer"):
    t = Tree(pos, mass, leaf_max, group_max)
    t.softening(soft, eps)
    t.moments(p)
    t.traverse(tol, G)
    return t.force(G, eps)
