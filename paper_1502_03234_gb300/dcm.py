"""Thin ctypes binding of libdcm.so (include/dcm.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  The functions keep the C names (``dcm_create``, ``dcm_step``, ...);
``System`` wraps a handle for convenience.  Loading fails loudly when the
library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdcm.so")

DCM_OK = 0
DCM_ERR_ARG, DCM_ERR_OOM, DCM_ERR_CUDA, DCM_ERR_BOX_TOO_SMALL = 1, 2, 3, 4
DCM_ERR_NOT_CONVERGED, DCM_ERR_DEVICE_CHECK, DCM_ERR_CANCELLED, DCM_ERR_STATE = 5, 6, 7, 8
DCM_FP64, DCM_MIXED = 0, 1
DCM_HOST, DCM_DEVICE = 0, 1
DCM_CUTOFF_EXP, DCM_CUTOFF_LINEAR = 0, 1
DCM_MAX_CLASSES = 8
DCM_WALK_WARP, DCM_WALK_LANES = 0, 1
DCM_SEG_KMEANS, DCM_SEG_MUMFORD_SHAH = 0, 1
# limits of the allocation-free cell sort (include/dcm.h)
DCM_NOALLOC_MAX_PARTICLES, DCM_NOALLOC_MAX_CELLS = 1 << 19, 1 << 20
DCM_GRAPH_BRANCHED, DCM_GRAPH_FLAT = 0, 1

#: every entry point include/dcm.h declares (checked by the ABI test)
EXPORTS = [
    "dcm_default_params", "dcm_create", "dcm_destroy", "dcm_set_state", "dcm_get_state",
    "dcm_update_state",
    "dcm_set_step", "dcm_set_cutoffs", "dcm_detect_interface", "dcm_compute_forces",
    "dcm_step", "dcm_energy_virial", "dcm_get_grid", "dcm_get_cutoffs", "dcm_get_cells",
    "dcm_get_pair_counts", "dcm_get_stats", "dcm_set_tuning", "dcm_get_tuning", "dcm_sync",
    "dcm_device_bytes", "dcm_estimate_bytes", "dcm_last_error", "dcm_version",
    "dcm_set_timing", "dcm_get_phase_times", "dcm_ensemble_create", "dcm_system_count",
    "dcm_system_range", "dcm_ensemble_set_state", "dcm_ensemble_get_state",
    "dcm_ensemble_energy_virial", "dcm_check_bounded_wait", "dcm_cell_sort_noalloc",
    "dcm_remove_small_components", "dcm_ms_segment", "dcm_set_allocator", "dcm_fp32_peak",
]
DCM_NUM_PHASES = 5
PHASES = ("kick_drift", "detect", "bin", "force", "kick")


class DcmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libdcm error {code}: {msg}")
        self.code = code


class dcm_box(C.Structure):
    _fields_ = [("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double)]


class dcm_params(C.Structure):
    _fields_ = [("rc_min", C.c_double), ("rc_max", C.c_double), ("alpha", C.c_double),
                ("dt", C.c_double), ("mass", C.c_double), ("eps", C.c_double),
                ("sigma", C.c_double), ("voxel", C.c_double), ("smooth_order", C.c_int32),
                ("detect_every", C.c_int32), ("kmeans_max_iter", C.c_int32),
                ("cfsm_iter_max", C.c_int32), ("cfsm_eps", C.c_double),
                ("precision", C.c_int32), ("n_classes", C.c_int32), ("cell_min", C.c_double),
                ("skin", C.c_double), ("list_density", C.c_float),
                ("list_margin", C.c_float), ("skin_time", C.c_float),
                ("skin_floor", C.c_float), ("min_component_voxels", C.c_int32),
                ("cutoff_fn", C.c_int32), ("segmentation", C.c_int32), ("ms_iters", C.c_int32),
                ("ms_outer", C.c_int32), ("ms_nu", C.c_double)]


class dcm_tuning(C.Structure):
    _fields_ = [("lanes", C.c_int32 * DCM_MAX_CLASSES), ("block", C.c_int32),
                ("walk", C.c_int32), ("list_lanes", C.c_int32), ("step_graph", C.c_int32),
                ("list_lanes_class", C.c_int32 * DCM_MAX_CLASSES), ("reserved", C.c_int32 * 4)]


class dcm_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("pairs", C.c_int64), ("kmeans_iters", C.c_int32),
                ("cfsm_iters", C.c_int32), ("class_count", C.c_int32 * DCM_MAX_CLASSES),
                ("grid", C.c_int32 * 3), ("cells", C.c_int32 * 3), ("c_liquid", C.c_double),
                ("c_vapor", C.c_double), ("guard_rechecks", C.c_int64),
                ("kernels_plain", C.c_int32), ("kernels_detect", C.c_int32),
                ("list_builds", C.c_int64), ("list_entries", C.c_int64),
                ("kernels_plain_reuse", C.c_int32), ("kernels_detect_reuse", C.c_int32),
                ("cc_flipped", C.c_int64), ("refined", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    """Load libdcm.so (build it first with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libdcm.so not built at {LIB_PATH}; run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p
    P = C.POINTER
    sig = {
        "dcm_default_params": (None, [P(dcm_params)]),
        "dcm_create": (C.c_int, [P(dcm_box), i64, P(dcm_params), vp, P(vp)]),
        "dcm_destroy": (C.c_int, [vp]),
        "dcm_set_allocator": (C.c_int, [vp, vp, vp]),
        "dcm_fp32_peak": (C.c_int, [i32, P(C.c_double), P(C.c_double)]),
        "dcm_set_state": (C.c_int, [vp, dp, dp, C.c_int]),
        "dcm_update_state": (C.c_int, [vp, dp, dp, C.c_int]),
        "dcm_get_state": (C.c_int, [vp, dp, dp, dp, C.c_int]),
        "dcm_set_step": (C.c_int, [vp, i64]),
        "dcm_set_cutoffs": (C.c_int, [vp, dp, C.c_int]),
        "dcm_detect_interface": (C.c_int, [vp]),
        "dcm_compute_forces": (C.c_int, [vp]),
        "dcm_step": (C.c_int, [vp, i64]),
        "dcm_energy_virial": (C.c_int, [vp, dp, dp, dp]),
        "dcm_get_grid": (C.c_int, [vp, dp, dp, dp, dp, dp]),
        "dcm_remove_small_components": (C.c_int, [vp, dp, i32, C.c_int, P(i64)]),
        "dcm_ms_segment": (C.c_int, [vp, dp, C.c_double, C.c_double, C.c_double, i32, dp, dp,
                                     C.c_int]),
        "dcm_get_cutoffs": (C.c_int, [vp, dp, dp, dp]),
        "dcm_get_cells": (C.c_int, [vp, dp, dp, dp]),
        "dcm_get_pair_counts": (C.c_int, [vp, dp]),
        "dcm_get_stats": (C.c_int, [vp, P(dcm_stats)]),
        "dcm_set_tuning": (C.c_int, [vp, P(dcm_tuning)]),
        "dcm_get_tuning": (C.c_int, [vp, P(dcm_tuning)]),
        "dcm_sync": (C.c_int, [vp]),
        "dcm_device_bytes": (i64, [vp]),
        "dcm_estimate_bytes": (i64, [P(dcm_box), i64, P(dcm_params)]),
        "dcm_last_error": (C.c_char_p, []),
        "dcm_set_timing": (C.c_int, [vp, C.c_int]),
        "dcm_ensemble_create": (C.c_int, [C.c_int, P(dcm_box), P(i64), P(dcm_params), vp,
                                          P(vp)]),
        "dcm_system_count": (C.c_int, [vp]),
        "dcm_check_bounded_wait": (C.c_int, [vp]),
        "dcm_cell_sort_noalloc": (C.c_int, [dp, i64, P(dcm_box), dp, dp, dp, vp]),
        "dcm_system_range": (C.c_int, [vp, C.c_int, P(i64), P(i64)]),
        "dcm_ensemble_set_state": (C.c_int, [vp, C.c_int, dp, dp, C.c_int]),
        "dcm_ensemble_get_state": (C.c_int, [vp, C.c_int, dp, dp, dp, C.c_int]),
        "dcm_ensemble_energy_virial": (C.c_int, [vp, C.c_int, dp, dp, dp]),
        "dcm_get_phase_times": (C.c_int, [vp, dp]),
        "dcm_version": (C.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(code: int) -> None:
    if code != DCM_OK:
        raise DcmError(code, lib().dcm_last_error().decode(errors="replace"))


def _ptr(a):
    """(pointer, mem) for a numpy array or a torch CUDA tensor."""
    if a is None:
        return None, DCM_HOST
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        return C.c_void_p(a.data_ptr()), DCM_DEVICE
    return a.ctypes.data_as(C.c_void_p), DCM_HOST


def default_params(**over) -> dcm_params:
    p = dcm_params()
    lib().dcm_default_params(C.byref(p))
    for k, v in over.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# ---- the C names ------------------------------------------------------------
def dcm_create(box, n: int, params: dcm_params | None = None, stream=None):
    h = C.c_void_p()
    b = dcm_box(*box)
    p = params if params is not None else default_params()
    s = C.c_void_p(stream) if stream else None
    check(lib().dcm_create(C.byref(b), int(n), C.byref(p), s, C.byref(h)))
    return h


def dcm_destroy(h) -> None:
    check(lib().dcm_destroy(h))


def dcm_fp32_peak(iters: int = 100000) -> tuple:
    """(TFLOP/s, ms) of an FP32 FMA chain on every SM of the current device"""
    t, ms = C.c_double(), C.c_double()
    check(lib().dcm_fp32_peak(int(iters), C.byref(t), C.byref(ms)))
    return t.value, ms.value


_ALLOCATOR = None          # the callbacks handed to the library, kept alive


def dcm_set_allocator(alloc=None, release=None, ctx=None) -> None:
    """The device allocator handles created from now on use (both None:
    cudaMallocAsync / cudaFreeAsync on the handle's stream)."""
    def addr(f):
        return None if f is None else C.cast(f, C.c_void_p)
    check(lib().dcm_set_allocator(addr(alloc), addr(release), ctx))


def use_torch_allocator() -> None:
    """Handles created from now on take their device memory from PyTorch's
    caching allocator, on the handle's stream (the allocator's memory then
    shows in torch.cuda.memory_allocated and is cached across handles)."""
    import torch

    alloc_t = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    release_t = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except RuntimeError:           # out of memory: the library reports DCM_ERR_OOM
            return None

    def _release(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    global _ALLOCATOR
    _ALLOCATOR = (alloc_t(_alloc), release_t(_release))
    dcm_set_allocator(*_ALLOCATOR)


def use_default_allocator() -> None:
    global _ALLOCATOR
    dcm_set_allocator(None, None)
    _ALLOCATOR = None


def dcm_set_state(h, x, v=None) -> None:
    px, mx = _ptr(x)
    pv, mv = _ptr(v)
    if v is not None and mv != mx:
        raise ValueError("x and v must live in the same memory space")
    check(lib().dcm_set_state(h, px, pv, mx))


def dcm_update_state(h, x, v=None) -> None:
    """replace the state of a running system, keeping its step counter,
    cutoffs and Verlet lists (the reuse test decides on a rebuild)"""
    px, mx = _ptr(x)
    pv, mv = _ptr(v)
    if v is not None and mv != mx:
        raise ValueError("x and v must live in the same memory space")
    check(lib().dcm_update_state(h, px, pv, mx))


def dcm_get_state(h, n: int):
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    f = np.empty((n, 3))
    check(lib().dcm_get_state(h, _ptr(x)[0], _ptr(v)[0], _ptr(f)[0], DCM_HOST))
    return x, v, f


def dcm_set_step(h, step: int) -> None:
    check(lib().dcm_set_step(h, int(step)))


def dcm_set_cutoffs(h, rc) -> None:
    p, m = _ptr(rc)
    check(lib().dcm_set_cutoffs(h, p, m))


def dcm_detect_interface(h) -> None:
    check(lib().dcm_detect_interface(h))


def dcm_compute_forces(h) -> None:
    check(lib().dcm_compute_forces(h))


def dcm_step(h, nsteps: int) -> None:
    check(lib().dcm_step(h, int(nsteps)))


def dcm_energy_virial(h):
    pe, ke = C.c_double(), C.c_double()
    w = (C.c_double * 6)()
    check(lib().dcm_energy_virial(h, C.byref(pe), C.byref(ke), w))
    return pe.value, ke.value, np.array(list(w))


def dcm_get_grid(h):
    dims = np.zeros(3, np.int32)
    check(lib().dcm_get_grid(h, _ptr(dims)[0], None, None, None, None))
    nv = int(np.prod(dims))
    counts = np.empty(nv, np.int32)
    sm = np.empty(nv)
    lab = np.empty(nv, np.uint8)
    dist = np.empty(nv)
    check(lib().dcm_get_grid(h, _ptr(dims)[0], _ptr(counts)[0], _ptr(sm)[0], _ptr(lab)[0],
                             _ptr(dist)[0]))
    return tuple(int(q) for q in dims), counts, sm, lab, dist


def dcm_remove_small_components(h, labels, min_voxels: int):
    """Section 4.2 on a label grid of system 0 (numpy uint8, or a CUDA
    tensor rewritten in place); returns (labels, voxels changed)."""
    dims = np.zeros(3, np.int32)
    check(lib().dcm_get_grid(h, _ptr(dims)[0], None, None, None, None))
    if not (hasattr(labels, "data_ptr") and getattr(labels, "is_cuda", False)):
        labels = np.array(np.ascontiguousarray(labels, dtype=np.uint8).ravel())
        size = labels.size
    else:
        if labels.dtype.itemsize != 1 or not labels.is_contiguous():
            raise ValueError("labels must be a contiguous uint8 tensor")
        size = labels.numel()
    if size != int(np.prod(dims)):
        raise ValueError(f"labels hold {size} voxels, the grid {int(np.prod(dims))}")
    p, mem = _ptr(labels)
    fl = C.c_int64(0)
    check(lib().dcm_remove_small_components(h, p, int(min_voxels), mem, C.byref(fl)))
    return labels, int(fl.value)


def dcm_ms_segment(h, rho, c_l: float, c_v: float, nu: float, iters: int):
    """Eq. 13 with fixed densities on an image of system 0's grid (numpy);
    returns (labels, relaxed u)"""
    dims = np.zeros(3, np.int32)
    check(lib().dcm_get_grid(h, _ptr(dims)[0], None, None, None, None))
    nv = int(np.prod(dims))
    rho = np.ascontiguousarray(rho, dtype=np.float64).ravel()
    if rho.size != nv:
        raise ValueError(f"image holds {rho.size} voxels, the grid {nv}")
    lab = np.empty(nv, np.uint8)
    u = np.empty(nv)
    check(lib().dcm_ms_segment(h, _ptr(rho)[0], float(c_l), float(c_v), float(nu), int(iters),
                               _ptr(lab)[0], _ptr(u)[0], DCM_HOST))
    return lab, u


def dcm_get_cutoffs(h, n: int):
    d = np.empty(n)
    rc = np.empty(n)
    cls = np.empty(n, np.uint8)
    check(lib().dcm_get_cutoffs(h, _ptr(d)[0], _ptr(rc)[0], _ptr(cls)[0]))
    return d, rc, cls


def dcm_get_cells(h, n: int):
    nc = np.zeros(3, np.int32)
    check(lib().dcm_get_cells(h, _ptr(nc)[0], None, None))
    ncell = int(np.prod(nc))
    start = np.empty(ncell + 1, np.int32)
    sid = np.empty(n, np.int32)
    check(lib().dcm_get_cells(h, _ptr(nc)[0], _ptr(start)[0], _ptr(sid)[0]))
    return tuple(int(q) for q in nc), start, sid


def dcm_get_pair_counts(h, n: int):
    out = np.empty(n, np.int32)
    check(lib().dcm_get_pair_counts(h, _ptr(out)[0]))
    return out


def dcm_get_stats(h) -> dcm_stats:
    s = dcm_stats()
    check(lib().dcm_get_stats(h, C.byref(s)))
    return s


def dcm_set_tuning(h, lanes, block: int = 256, walk: int = None, list_lanes: int = 8,
                   list_lanes_class=None) -> None:
    """lanes/block: the FP64 lanes walk; list_lanes: lanes per particle of
    the mixed-precision list force; list_lanes_class: per cutoff class
    instead (the class-ordered list force; None: list_lanes for all); walk
    None keeps the handle's walk"""
    cur = dcm_get_tuning(h)
    t = dcm_tuning()
    for q in range(DCM_MAX_CLASSES):
        t.lanes[q] = int(lanes[min(q, len(lanes) - 1)])
    t.block = int(block)
    t.walk = cur.walk if walk is None else int(walk)
    t.list_lanes = int(list_lanes)
    t.step_graph = cur.step_graph          # kept (see set_step_graph)
    if list_lanes_class is not None:
        for q in range(DCM_MAX_CLASSES):
            t.list_lanes_class[q] = int(list_lanes_class[min(q, len(list_lanes_class) - 1)])
    check(lib().dcm_set_tuning(h, C.byref(t)))


def dcm_get_tuning(h) -> dcm_tuning:
    t = dcm_tuning()
    check(lib().dcm_get_tuning(h, C.byref(t)))
    return t


def dcm_set_timing(h, on: bool) -> None:
    check(lib().dcm_set_timing(h, 1 if on else 0))


def dcm_get_phase_times(h) -> dict:
    ms = np.zeros(DCM_NUM_PHASES, np.float32)
    check(lib().dcm_get_phase_times(h, ms.ctypes.data_as(C.c_void_p)))
    return {k: float(v) for k, v in zip(PHASES, ms)}


def dcm_sync(h) -> None:
    check(lib().dcm_sync(h))


def dcm_device_bytes(h) -> int:
    return int(lib().dcm_device_bytes(h))


def dcm_estimate_bytes(box, n: int, params: dcm_params | None = None) -> int:
    b = dcm_box(*box)
    p = params if params is not None else default_params()
    return int(lib().dcm_estimate_bytes(C.byref(b), int(n), C.byref(p)))


def _check_device_tensor(t, name: str, dtype: str, count: int) -> None:
    # the C side sees only pointers: a buffer of the wrong type, place or
    # length would be written out of bounds on the GPU
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype}":
        raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < count:
        raise ValueError(f"{name} holds {t.numel()} elements, needs at least {count}")


def dcm_cell_sort_noalloc(x_dev, n: int, box, nc, cell_start_dev, sorted_id_dev,
                          stream=None) -> None:
    """Allocation-free link-cell sort on device buffers (torch CUDA tensors:
    x float64 [n, 3], cell_start int32 [ncell + 1], sorted_id int32 [n])."""
    n = int(n)
    if len(nc) != 3 or min(int(q) for q in nc) < 1:
        raise ValueError("nc must be three positive cell counts")
    ncell = int(np.prod([int(q) for q in nc], dtype=object))
    if 1 <= n <= DCM_NOALLOC_MAX_PARTICLES and ncell <= DCM_NOALLOC_MAX_CELLS:
        # (sizes beyond the scratch limits are left to the library, which
        # rejects them before any launch)
        _check_device_tensor(x_dev, "x", "float64", 3 * n)
        _check_device_tensor(cell_start_dev, "cell_start", "int32", ncell + 1)
        _check_device_tensor(sorted_id_dev, "sorted_id", "int32", n)
    b = dcm_box(*box)
    ncv = (C.c_int32 * 3)(*[int(q) for q in nc])
    s = C.c_void_p(stream) if stream else None
    check(lib().dcm_cell_sort_noalloc(C.c_void_p(x_dev.data_ptr()), int(n), C.byref(b), ncv,
                                      C.c_void_p(cell_start_dev.data_ptr()),
                                      C.c_void_p(sorted_id_dev.data_ptr()), s))


def dcm_ensemble_create(boxes, ns, params_list, stream=None):
    m = len(ns)
    B = (dcm_box * m)(*[dcm_box(*b) for b in boxes])
    Nn = (C.c_int64 * m)(*[int(x) for x in ns])
    Pp = (dcm_params * m)(*params_list)
    h = C.c_void_p()
    s = C.c_void_p(stream) if stream else None
    check(lib().dcm_ensemble_create(m, B, Nn, Pp, s, C.byref(h)))
    return h


def dcm_system_count(h) -> int:
    return int(lib().dcm_system_count(h))


def dcm_system_range(h, k: int):
    a, b = C.c_int64(), C.c_int64()
    check(lib().dcm_system_range(h, int(k), C.byref(a), C.byref(b)))
    return a.value, b.value


def dcm_ensemble_set_state(h, k: int, x, v=None) -> None:
    px, mx = _ptr(x)
    pv, _ = _ptr(v)
    check(lib().dcm_ensemble_set_state(h, int(k), px, pv, mx))


def dcm_ensemble_get_state(h, k: int, n: int):
    x, v, f = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
    check(lib().dcm_ensemble_get_state(h, int(k), _ptr(x)[0], _ptr(v)[0], _ptr(f)[0], DCM_HOST))
    return x, v, f


def dcm_ensemble_energy_virial(h, k: int):
    pe, ke = C.c_double(), C.c_double()
    w = (C.c_double * 6)()
    check(lib().dcm_ensemble_energy_virial(h, int(k), C.byref(pe), C.byref(ke), w))
    return pe.value, ke.value, np.array(list(w))


# ---- convenience wrapper ------------------------------------------------------
class System:
    """One DCM system on the GPU (a dcm_handle)."""

    def __init__(self, box, n: int, params: dcm_params | None = None, stream=None, **over):
        if params is None:
            params = default_params(**over)
        else:
            for k, v in over.items():
                setattr(params, k, v)
        self.box = tuple(float(b) for b in box)
        self.n = int(n)
        self.params = params
        self.h = dcm_create(self.box, self.n, params, stream)

    def close(self):
        if self.h:
            dcm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, x, v=None):
        if not (hasattr(x, "is_cuda") and x.is_cuda):
            x = np.ascontiguousarray(x, np.float64)
            v = None if v is None else np.ascontiguousarray(v, np.float64)
        dcm_set_state(self.h, x, v)

    def update_state(self, x, v=None):
        """the state of the running system replaced (step counter, cutoffs
        and lists kept; forces recomputed before the next step)"""
        if not (hasattr(x, "is_cuda") and x.is_cuda):
            x = np.ascontiguousarray(x, np.float64)
            v = None if v is None else np.ascontiguousarray(v, np.float64)
        dcm_update_state(self.h, x, v)

    def get_state(self):
        return dcm_get_state(self.h, self.n)

    def set_cutoffs(self, rc):
        dcm_set_cutoffs(self.h, np.ascontiguousarray(rc, np.float64))

    def detect_interface(self):
        dcm_detect_interface(self.h)

    def compute_forces(self):
        dcm_compute_forces(self.h)

    def step(self, nsteps: int):
        dcm_step(self.h, nsteps)

    def energy_virial(self):
        return dcm_energy_virial(self.h)

    def grid(self):
        return dcm_get_grid(self.h)

    def remove_small_components(self, labels, min_voxels: int):
        return dcm_remove_small_components(self.h, labels, min_voxels)

    def ms_segment(self, rho, c_l, c_v, nu, iters):
        return dcm_ms_segment(self.h, rho, c_l, c_v, nu, iters)

    def cutoffs(self):
        return dcm_get_cutoffs(self.h, self.n)

    def cells(self):
        return dcm_get_cells(self.h, self.n)

    def pair_counts(self):
        return dcm_get_pair_counts(self.h, self.n)

    def stats(self) -> dcm_stats:
        return dcm_get_stats(self.h)

    def set_tuning(self, lanes, block=256, walk=None, list_lanes=8, list_lanes_class=None):
        """lanes/block: the FP64 lanes walk (lanes per particle per cutoff
        class, threads per block); list_lanes: lanes per particle of the
        mixed-precision Verlet-list force, or list_lanes_class per cutoff
        class; walk None keeps the current walk (DCM_MIXED always runs the
        warp kernels)"""
        dcm_set_tuning(self.h, lanes, block, walk, list_lanes, list_lanes_class)

    def set_step(self, step: int):
        """the global step counter (detection runs on steps divisible by
        detect_every): continue a resumed run on its original cadence"""
        dcm_set_step(self.h, step)

    def set_step_graph(self, shape: int):
        """DCM_GRAPH_BRANCHED (default) or DCM_GRAPH_FLAT"""
        t = dcm_get_tuning(self.h)
        t.step_graph = int(shape)
        check(lib().dcm_set_tuning(self.h, C.byref(t)))

    def sync(self):
        dcm_sync(self.h)

    def set_timing(self, on: bool = True):
        dcm_set_timing(self.h, on)

    def phase_times(self) -> dict:
        return dcm_get_phase_times(self.h)

    def device_bytes(self) -> int:
        return dcm_device_bytes(self.h)


class Ensemble(System):
    """Many independent systems in one handle: one set of kernels and one
    persistent force launch per step for all of them."""

    def __init__(self, boxes, ns, params_list, stream=None):
        self.boxes = [tuple(float(q) for q in b) for b in boxes]
        self.ns = [int(q) for q in ns]
        self.n = sum(self.ns)
        self.params = params_list[0]
        self.h = dcm_ensemble_create(self.boxes, self.ns, params_list, stream)
        self.ranges = [dcm_system_range(self.h, k) for k in range(len(self.ns))]

    def set_system_state(self, k, x, v=None):
        dcm_ensemble_set_state(self.h, k, np.ascontiguousarray(x, np.float64),
                               None if v is None else np.ascontiguousarray(v, np.float64))

    def get_system_state(self, k):
        return dcm_ensemble_get_state(self.h, k, self.ns[k])

    def system_energy(self, k):
        return dcm_ensemble_energy_virial(self.h, k)
