"""Thin ctypes binding of libhot.so, the C ABI declared in include/hot.h.

Argument marshalling only: every stage of the force path runs in the CUDA
kernels of libhot.so.  There is no fallback; if the library is missing or fails
to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HOT_OK, HOT_EINVAL, HOT_ESTATE, HOT_ENOMEM, HOT_EOVERFLOW, HOT_ECUDA, HOT_EINPUT, HOT_ETIMEOUT = (
    0, -1, -2, -3, -4, -5, -6, -7)
HOT_FP32_MIXED, HOT_FP64 = 0, 1
HOT_SOFT_PLUMMER, HOT_SOFT_K1, HOT_SOFT_SPLINE = 0, 1, 2
HOT_DBGSET_FRONTIER_CAP, HOT_DBGSET_SLOT_CAP, HOT_DBGSET_WAIT_POLLS, HOT_DBGSET_WAIT_PROBE = 0, 1, 2, 3

DBG = dict(FRAME=0, SORTED_KEYS=1, PERM=2, CELL_KEY=3, CELL_LEVEL=4, CELL_BEGIN=5, CELL_COUNT=6,
           CELL_PARENT=7, CELL_NCHILD=8, GROUP_CELL=9, GROUP_CENTRE=10, GROUP_DMAX=11, CELL_MASS=12,
           CELL_COM=13, MOMENTS=14, CELL_BMAX=15, CELL_B1=16, CELL_B2=17, M2P_OFFSETS=18, M2P_CELLS=19,
           P2P_OFFSETS=20, P2P_CELLS=21, M2P_ORDERS=22, M2P_IMAGES=23, P2P_IMAGES=24, BG_CUBE_OFFSETS=25,
           BG_CUBES=26, BG_GROUP_S=27, BG_EMPTY_PARENT=28, BG_EMPTY_OCTANT=29)

EXPORTS = ("hot_create", "hot_set_params", "hot_build_tree", "hot_compute_moments", "hot_traverse",
           "hot_evaluate_forces", "hot_adjoint", "hot_stage_times", "hot_sizes", "hot_debug_get",
           "hot_lookup", "hot_fma_peak", "hot_strerror", "hot_destroy", "hot_key_frame_noalloc", "hot_axpy",
           "hot_memory_stats", "hot_synchronize", "hot_debug_set", "hot_lattice_sums", "hot_bg_sizes")


class hot_params(C.Structure):
    _fields_ = [("p", C.c_int), ("tol", C.c_double), ("eps", C.c_double), ("G", C.c_double),
                ("leaf_max", C.c_int), ("group_max", C.c_int), ("precision", C.c_int),
                ("softening", C.c_int), ("p_min", C.c_int), ("box", C.c_double), ("ws", C.c_int),
                ("box_lo", C.c_double * 3), ("background", C.c_int), ("bg_up", C.c_int)]


class HotError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libhot.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library missing: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.hot_create.argtypes = [C.POINTER(vp), C.POINTER(hot_params), vp]
    L.hot_set_params.argtypes = [vp, C.POINTER(hot_params)]
    L.hot_build_tree.argtypes = [vp, vp, vp, C.c_int64]
    L.hot_compute_moments.argtypes = [vp, C.c_int]
    L.hot_traverse.argtypes = [vp, C.c_double]
    L.hot_evaluate_forces.argtypes = [vp, vp, vp]
    L.hot_adjoint.argtypes = [vp, vp, vp, vp, vp]
    L.hot_stage_times.argtypes = [vp, C.POINTER(C.c_float)]
    L.hot_sizes.argtypes = [vp, C.POINTER(C.c_int64)]
    L.hot_debug_get.argtypes = [vp, C.c_int, vp, C.c_size_t]
    L.hot_lookup.argtypes = [vp, vp, C.c_int64, vp]
    L.hot_fma_peak.argtypes = [vp, C.c_int, C.POINTER(C.c_double)]
    L.hot_strerror.restype = C.c_char_p
    L.hot_strerror.argtypes = [C.c_int]
    L.hot_destroy.argtypes = [vp]
    L.hot_destroy.restype = None
    L.hot_key_frame_noalloc.argtypes = [vp, vp, C.c_int64, vp, vp]
    L.hot_axpy.argtypes = [vp, vp, vp, C.c_double, C.c_int64]
    L.hot_memory_stats.argtypes = [C.POINTER(C.c_int64), C.c_int]
    L.hot_synchronize.argtypes = [vp]
    L.hot_debug_set.argtypes = [vp, C.c_int, C.c_int64]
    L.hot_lattice_sums.argtypes = [C.c_double, C.c_int, C.c_int, vp]
    L.hot_bg_sizes.argtypes = [vp, C.POINTER(C.c_int64)]
    for name in ("hot_create", "hot_set_params", "hot_build_tree", "hot_compute_moments", "hot_traverse",
                 "hot_evaluate_forces", "hot_adjoint", "hot_stage_times", "hot_sizes", "hot_debug_get",
                 "hot_lookup", "hot_fma_peak", "hot_key_frame_noalloc", "hot_axpy",
                 "hot_memory_stats", "hot_synchronize", "hot_debug_set", "hot_lattice_sums", "hot_bg_sizes"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    return load().hot_strerror(int(code)).decode()


def _ck(code, what):
    if code != HOT_OK:
        raise HotError(code, what)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _need(t, shape_last=None):
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t


def make_params(p=4, tol=1e-4, eps=0.0, G=1.0, leaf_max=64, group_max=128, precision="mixed",
                softening="plummer", p_min=None, box=0.0, ws=2, box_lo=(0.0, 0.0, 0.0), background=False,
                bg_up=2):
    prec = HOT_FP64 if precision in ("fp64", "f64", HOT_FP64) else HOT_FP32_MIXED
    kinds = {"plummer": HOT_SOFT_PLUMMER, "k1": HOT_SOFT_K1, "spline": HOT_SOFT_SPLINE,
             HOT_SOFT_PLUMMER: HOT_SOFT_PLUMMER, HOT_SOFT_K1: HOT_SOFT_K1, HOT_SOFT_SPLINE: HOT_SOFT_SPLINE}
    if softening not in kinds:
        raise ValueError(f"unknown softening {softening!r}: plummer, k1 or spline")
    soft = kinds[softening]
    return hot_params(int(p), float(tol), float(eps), float(G), int(leaf_max), int(group_max), prec, soft,
                      -1 if p_min is None else int(p_min), float(box), int(ws),
                      (C.c_double * 3)(*[float(v) for v in box_lo]), 1 if background else 0, int(bg_up))


class Hot:
    """One library context: its tree, moments and lists live on the device."""

    def __init__(self, stream=None, **kw):
        import torch
        L = load()
        self.params = make_params(**kw)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        _ck(L.hot_create(C.byref(h), C.byref(self.params), C.c_void_p(stream.cuda_stream)), "hot_create")
        self._h = h
        self.N = 0
        self.generation = 0  # bumped by every build_tree: names the tree the context holds

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hot_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_params(self, **kw):
        self.params = make_params(**kw)
        _ck(load().hot_set_params(self._h, C.byref(self.params)), "hot_set_params")

    def build_tree(self, pos, mass):
        _need(pos)
        _need(mass)
        self.N = int(mass.shape[0])
        self.generation += 1
        _ck(load().hot_build_tree(self._h, _ptr(pos), _ptr(mass), self.N), "hot_build_tree")

    def compute_moments(self, p=None):
        p = self.params.p if p is None else p
        _ck(load().hot_compute_moments(self._h, int(p)), "hot_compute_moments")

    def traverse(self, tol=None):
        tol = self.params.tol if tol is None else tol
        _ck(load().hot_traverse(self._h, float(tol)), "hot_traverse")

    def evaluate_forces(self, acc, pot=None):
        _need(acc)
        if pot is not None:
            _need(pot)
        _ck(load().hot_evaluate_forces(self._h, _ptr(acc), _ptr(pot)), "hot_evaluate_forces")

    def force(self, pos, mass, acc, pot=None):
        """The whole forward path at this context's parameters: build, moments,
        traversal, interactions into the given device tensors."""
        self.build_tree(pos, mass)
        self.compute_moments(self.params.p)
        self.traverse(self.params.tol)
        self.evaluate_forces(acc, pot)

    def adjoint(self, g_acc, g_pot, g_pos, g_mass):
        for t in (g_acc, g_pos, g_mass):
            _need(t)
        if g_pot is not None:
            _need(g_pot)
        _ck(load().hot_adjoint(self._h, _ptr(g_acc), _ptr(g_pot), _ptr(g_pos), _ptr(g_mass)), "hot_adjoint")

    def stage_times(self):
        ms = (C.c_float * 6)()
        _ck(load().hot_stage_times(self._h, ms), "hot_stage_times")
        return dict(zip(("sort", "build", "moments", "traverse", "interact", "adjoint"), list(ms)))

    def sizes(self):
        out = (C.c_int64 * 10)()
        _ck(load().hot_sizes(self._h, out), "hot_sizes")
        return dict(zip(("N", "ncell", "ngroup", "nleaf", "maxlevel", "n_m2p", "n_p2p", "n_pairs", "n_m2p_int",
                         "launches"), list(out)))

    def bg_sizes(self):
        """Background subtraction's sizes (see hot_bg_sizes in include/hot.h)."""
        out = (C.c_int64 * 6)()
        _ck(load().hot_bg_sizes(self._h, out), "hot_bg_sizes")
        return dict(zip(("n_empty", "n_cube_entries", "cube_evals", "m2p_contrast", "m2p_empty", "m2p_matter"),
                        list(out)))

    def debug_get(self, what):
        s = self.sizes()
        N, nc, ng = s["N"], s["ncell"], s["ngroup"]
        bg = self.bg_sizes() if self.params.background else {"n_empty": 0, "n_cube_entries": 0}
        ncomp = (self.params.p + 1) * (self.params.p + 2) * (self.params.p + 3) // 6
        spec = {
            "FRAME": (np.float64, (4,)), "SORTED_KEYS": (np.uint64, (N,)), "PERM": (np.int32, (N,)),
            "CELL_KEY": (np.uint64, (nc,)), "CELL_LEVEL": (np.int32, (nc,)), "CELL_BEGIN": (np.int32, (nc,)),
            "CELL_COUNT": (np.int32, (nc,)), "CELL_PARENT": (np.int32, (nc,)), "CELL_NCHILD": (np.int32, (nc,)),
            "GROUP_CELL": (np.int32, (ng,)), "GROUP_CENTRE": (np.float64, (ng, 3)),
            "GROUP_DMAX": (np.float64, (ng,)), "CELL_MASS": (np.float64, (nc,)), "CELL_COM": (np.float64, (nc, 3)),
            "MOMENTS": (np.float64, (nc, ncomp)), "CELL_BMAX": (np.float64, (nc,)), "CELL_B1": (np.float64, (nc,)),
            "CELL_B2": (np.float64, (nc,)), "M2P_OFFSETS": (np.int64, (ng + 1,)), "M2P_CELLS": (np.int32, (s["n_m2p"],)),
            "P2P_OFFSETS": (np.int64, (ng + 1,)), "P2P_CELLS": (np.int32, (s["n_p2p"],)),
            "M2P_ORDERS": (np.int32, (s["n_m2p"],)), "M2P_IMAGES": (np.int32, (s["n_m2p"],)),
            "P2P_IMAGES": (np.int32, (s["n_p2p"],)), "BG_CUBE_OFFSETS": (np.int64, (ng + 1,)),
            "BG_CUBES": (np.int32, (bg["n_cube_entries"],)), "BG_GROUP_S": (np.int32, (ng,)),
            "BG_EMPTY_PARENT": (np.int32, (bg["n_empty"],)), "BG_EMPTY_OCTANT": (np.int32, (bg["n_empty"],)),
        }[what]
        out = np.zeros(spec[1], dtype=spec[0])
        _ck(load().hot_debug_get(self._h, DBG[what], out.ctypes.data_as(C.c_void_p), out.nbytes),
            f"hot_debug_get({what})")
        return out

    def lookup(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.zeros(len(keys), dtype=np.int32)
        _ck(load().hot_lookup(self._h, keys.ctypes.data_as(C.c_void_p), len(keys),
                              out.ctypes.data_as(C.c_void_p)), "hot_lookup")
        return out

    def axpy(self, y, x, alpha):
        """y += alpha * x on the device (float64 CUDA tensors of equal size)."""
        _need(y)
        _need(x)
        if y.numel() != x.numel():
            raise ValueError("size mismatch")
        _ck(load().hot_axpy(self._h, _ptr(y), _ptr(x), float(alpha), int(y.numel())), "hot_axpy")

    def synchronize(self):
        """Wait for the context stream; raises HotError for a device-side status (for the
        asynchronous calls: moments, forces, adjoint)."""
        _ck(load().hot_synchronize(self._h), "hot_synchronize")

    def debug_set(self, what, value):
        """Test knobs: HOT_DBGSET_FRONTIER_CAP, HOT_DBGSET_SLOT_CAP, HOT_DBGSET_WAIT_POLLS,
        HOT_DBGSET_WAIT_PROBE (see include/hot.h)."""
        _ck(load().hot_debug_set(self._h, int(what), int(value)), "hot_debug_set")

    def fma_peak(self, dbl=False):
        v = C.c_double()
        _ck(load().hot_fma_peak(self._h, 1 if dbl else 0, C.byref(v)), "hot_fma_peak")
        return v.value


def lattice_sums(L, ws=2, order=17):
    """D^g psi_far(0), |g| <= order, of a periodic cube of side L less the images within ws
    (host computation): a numpy array in graded order (by |g|, then descending g_x, then
    descending g_y)."""
    import numpy as np
    n = (order + 1) * (order + 2) * (order + 3) // 6 if order >= 0 else 0
    out = np.zeros(max(n, 1))
    _ck(load().hot_lattice_sums(float(L), int(ws), int(order), out.ctypes.data_as(C.c_void_p)), "hot_lattice_sums")
    return out[:n]


def memory_stats(reset_peak=False):
    """(bytes the library holds on the device now, peak bytes since load or last reset)."""
    out = (C.c_int64 * 2)()
    _ck(load().hot_memory_stats(out, 1 if reset_peak else 0), "hot_memory_stats")
    return int(out[0]), int(out[1])


def key_frame_noalloc(pos, mass, frame, stream=None):
    """Allocation-free key frame (lo_x, lo_y, lo_z, L) of device tensors into the device
    tensor frame[4]; see hot_key_frame_noalloc in include/hot.h."""
    import torch
    _need(pos)
    _need(mass)
    _need(frame)
    if pos.dim() != 2 or pos.shape[1] != 3 or mass.dim() != 1 or pos.shape[0] != mass.shape[0]:
        raise ValueError("key_frame_noalloc: pos must be [N,3] and mass [N] with the same N")
    if frame.numel() < 4:
        raise ValueError("key_frame_noalloc: frame needs at least 4 float64 elements")
    if not (pos.device == mass.device == frame.device):
        raise ValueError("key_frame_noalloc: pos, mass and frame must be on one device")
    st = stream or torch.cuda.current_stream()
    _ck(load().hot_key_frame_noalloc(_ptr(pos), _ptr(mass), int(mass.shape[0]), _ptr(frame),
                                     C.c_void_p(st.cuda_stream)), "hot_key_frame_noalloc")
    return frame


def tree_force(pos, mass, p=4, tol=1e-4, eps=0.0, G=1.0, leaf_max=64, group_max=128, precision="mixed",
               ctx: Hot | None = None, want_pot=True, softening="plummer", p_min=None, box=0.0, ws=2,
               box_lo=(0.0, 0.0, 0.0), background=False, bg_up=2):
    """Tree-code acceleration (and potential) of float64 CUDA tensors pos [N,3], mass [N];
    box > 0: periodic cube [box_lo, box_lo + box) with the images within ws served by the tree."""
    import torch
    h = ctx or Hot(p=p, tol=tol, eps=eps, G=G, leaf_max=leaf_max, group_max=group_max, precision=precision,
                   softening=softening, p_min=p_min, box=box, ws=ws, box_lo=box_lo, background=background,
                   bg_up=bg_up)
    h.build_tree(pos, mass)
    h.compute_moments(p)
    h.traverse(tol)
    acc = torch.empty_like(pos)
    pot = torch.empty_like(mass) if want_pot else None
    h.evaluate_forces(acc, pot)
    return acc, pot


def tree_force_host(pos_h, mass_h, acc_h, pot_h=None, ctx: Hot | None = None, p=4, tol=1e-4, **kw):
    """Tree force of host (preferably pinned) float64 tensors: copies the inputs to the
    device, runs the whole path on the context's stream and copies acc (and pot) back
    into the given host tensors.  Returns after the results are on the host."""
    import torch
    h = ctx or Hot(p=p, tol=tol, **kw)
    st = h.stream
    with torch.cuda.stream(st):
        P = pos_h.to("cuda", non_blocking=True)
        M = mass_h.to("cuda", non_blocking=True)
        h.build_tree(P, M)
        h.compute_moments(p)
        h.traverse(tol)
        acc = torch.empty_like(P)
        pot = torch.empty_like(M) if pot_h is not None else None
        h.evaluate_forces(acc, pot)
        acc_h.copy_(acc, non_blocking=True)
        if pot_h is not None:
            pot_h.copy_(pot, non_blocking=True)
    st.synchronize()
    return acc_h, pot_h
