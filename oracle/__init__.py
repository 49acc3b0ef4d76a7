"""FP64 CPU oracle of the dynamic cutoff method (DCM) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python binding
never import it, and it imports nothing from them.

Every function is a thin ctypes wrapper over ``dcm_oracle.c``; the arithmetic
lives there, written from Springer's thesis (arxiv 1502.03234), each routine
citing its equation or algorithm.  ``build()`` compiles the shared library
with gcc (``-ffp-contract=off``, optional OpenMP for the Algorithm 5.1
``schedule(dynamic,20)`` loop over particles).
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dcm_oracle.c")
_HDR = os.path.join(_HERE, "dcm_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None


_CMD = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]


def _fingerprint() -> str:
    # content of the sources, the flags and the machine: a library built from
    # other sources or on another machine is never reused
    h = hashlib.sha256()
    for f in (_SRC, _HDR):
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(_CMD).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources (quick: one C file)."""
    fp = _fingerprint()
    stamp = _LIB + ".fingerprint"
    if not force and os.path.exists(_LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == fp:
                return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(_CMD + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    with open(stamp + f".tmp{os.getpid()}", "w") as fh:
        fh.write(fp)
    os.replace(stamp + f".tmp{os.getpid()}", stamp)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    d, i32, i64, vp = C.c_double, C.c_int32, C.c_int64, C.c_void_p
    sig = {
        "orc_set_threads": (C.c_int, [C.c_int]),
        "orc_get_threads": (C.c_int, []),
        "orc_lj": (None, [d, d, d, vp, vp]),
        "orc_cutoff": (d, [d, d, d, d]),
        "orc_class_thresholds": (None, [d, d, d, C.c_int, vp]),
        "orc_cutoff_class": (C.c_int, [d, d, C.c_int, vp]),
        "orc_cutoff_linear": (d, [d, d, d]),
        "orc_class_thresholds_linear": (None, [d, d, C.c_int, vp]),
        "orc_grid_dims": (None, [vp, d, vp]),
        "orc_cell_dims": (None, [vp, d, vp]),
        "orc_bin_index": (C.c_int, [d, C.c_int, d]),
        "orc_wrap": (d, [d, d]),
        "orc_cell_list": (None, [i64, vp, vp, vp, vp, vp, vp]),
        "orc_forces": (C.c_int, [i64, vp, vp, vp, vp, d, d, vp, vp, vp, vp]),
        "orc_forces_brute": (C.c_int, [i64, vp, vp, vp, d, d, vp, vp, vp, vp]),
        "orc_forces_static_half": (C.c_int, [i64, vp, d, vp, d, d, vp, vp]),
        "orc_density": (None, [i64, vp, vp, vp, vp]),
        "orc_smooth": (None, [vp, vp, C.c_int, vp]),
        "orc_kmeans": (C.c_int, [i64, vp, C.c_int, vp, vp, vp]),
        "orc_ms_energy": (d, [vp, vp, d, d, d, vp]),
        "orc_ms_segment": (None, [vp, vp, d, d, d, C.c_int, vp, vp]),
        "orc_ms_alternate": (C.c_int, [vp, vp, d, C.c_int, C.c_int, vp, vp, vp]),
        "orc_ms_detect": (C.c_int, [vp, vp, d, d, C.c_int, C.c_int, vp]),
        "orc_label_components": (i64, [vp, vp, C.c_int, vp]),
        "orc_remove_small_components": (i64, [vp, vp, C.c_int]),
        "orc_godunov": (d, [vp, vp]),
        "orc_fsm": (C.c_int, [vp, vp, vp, d, vp]),
        "orc_cfsm": (C.c_int, [vp, vp, vp, d, C.c_int, d, vp]),
        "orc_particle_distance": (None, [i64, vp, vp, vp, vp, vp]),
        "orc_detect": (C.c_int, [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "orc_run": (C.c_int, [i64, vp, vp, vp, vp, i64, i64, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def set_threads(n: int) -> int:
    return _load().orc_set_threads(int(n))


def get_threads() -> int:
    return _load().orc_get_threads()


# ---- Eq. 4 -----------------------------------------------------------------
def lj(r: float, eps: float = 1.0, sigma: float = 1.0) -> tuple[float, float]:
    """(V(r), fr) with F_i<-j = fr * (x_i - x_j)."""
    V, fr = C.c_double(), C.c_double()
    _load().orc_lj(float(r), float(eps), float(sigma), C.byref(V), C.byref(fr))
    return V.value, fr.value


# ---- Eq. 7-8 ---------------------------------------------------------------
def cutoff(d: float, rc_min: float, rc_max: float, alpha: float = -0.5) -> float:
    return _load().orc_cutoff(float(d), float(rc_min), float(rc_max), float(alpha))


def class_thresholds(rc_min, rc_max, alpha, K) -> np.ndarray:
    thr = np.zeros(max(K - 2, 1), np.float64)
    _load().orc_class_thresholds(float(rc_min), float(rc_max), float(alpha), int(K), _p(thr))
    return thr[: max(K - 2, 0)]


def cutoff_linear(d: float, rc_min: float, rc_max: float) -> float:
    return _load().orc_cutoff_linear(float(d), float(rc_min), float(rc_max))


def class_thresholds_linear(rc_min, rc_max, K) -> np.ndarray:
    thr = np.zeros(max(K - 2, 1), np.float64)
    _load().orc_class_thresholds_linear(float(rc_min), float(rc_max), int(K), _p(thr))
    return thr[: max(K - 2, 0)]


def cutoff_class(d, rc_max, K, thr) -> int:
    thr = _f64(thr if len(thr) else np.zeros(1))
    return _load().orc_cutoff_class(float(d), float(rc_max), int(K), _p(thr))


# ---- bins ------------------------------------------------------------------
def grid_dims(L, b) -> tuple[int, int, int]:
    L = _f64(L)
    dims = np.zeros(3, np.int32)
    _load().orc_grid_dims(_p(L), float(b), _p(dims))
    return tuple(int(v) for v in dims)


def cell_dims(L, c) -> tuple[int, int, int]:
    L = _f64(L)
    nc = np.zeros(3, np.int32)
    _load().orc_cell_dims(_p(L), float(c), _p(nc))
    return tuple(int(v) for v in nc)


def bin_index(x: float, n: int, L: float) -> int:
    return _load().orc_bin_index(float(x), int(n), float(L))


def wrap(x: float, L: float) -> float:
    return _load().orc_wrap(float(x), float(L))


def cell_list(x, L, nc):
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    L = _f64(L)
    nc_a = _i32(nc)
    ncell = int(np.prod(nc_a))
    cell_of = np.zeros(max(n, 1), np.int32)
    start = np.zeros(ncell + 1, np.int32)
    sid = np.zeros(max(n, 1), np.int32)
    _load().orc_cell_list(n, _p(x), _p(L), _p(nc_a), _p(cell_of), _p(start), _p(sid))
    return cell_of[:n], start, sid[:n]


# ---- Algorithms 3.2 / 2.1 -------------------------------------------------
@dataclass
class ForceResult:
    f: np.ndarray       # (N, 3)
    pe: np.ndarray      # (N,)  1/2 sum_j V
    vir: np.ndarray     # (6,)  xx yy zz xy xz yz
    npair: np.ndarray   # (N,)  contributing neighbours


def forces(x, rc, L, nc, eps=1.0, sigma=1.0, brute=False) -> ForceResult:
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    rc = _f64(np.broadcast_to(rc, (n,)))
    L = _f64(L)
    f = np.zeros((max(n, 1), 3))
    pe = np.zeros(max(n, 1))
    vir = np.zeros(6)
    npair = np.zeros(max(n, 1), np.int32)
    lib = _load()
    if brute:
        rcode = lib.orc_forces_brute(n, _p(x), _p(rc), _p(L), eps, sigma, _p(f), _p(pe),
                                     _p(vir), _p(npair))
    else:
        nc_a = _i32(nc)
        rcode = lib.orc_forces(n, _p(x), _p(rc), _p(L), _p(nc_a), eps, sigma, _p(f), _p(pe),
                               _p(vir), _p(npair))
    if rcode != 0:
        raise ValueError("oracle: cutoff not below half the shortest box edge")
    return ForceResult(f[:n], pe[:n], vir, npair[:n])


def forces_static_half(x, rc, L, eps=1.0, sigma=1.0):
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    L = _f64(L)
    f = np.zeros((max(n, 1), 3))
    pe = np.zeros(max(n, 1))
    if _load().orc_forces_static_half(n, _p(x), float(rc), _p(L), eps, sigma, _p(f), _p(pe)):
        raise ValueError("oracle: cutoff not below half the shortest box edge")
    return f[:n], pe[:n]


# ---- Section 4 ---------------------------------------------------------------
def density(x, L, dims) -> np.ndarray:
    x = _f64(x).reshape(-1, 3)
    L = _f64(L)
    d = _i32(dims)
    B = np.zeros(int(np.prod(d)), np.int32)
    _load().orc_density(x.shape[0], _p(x), _p(L), _p(d), _p(B))
    return B


def smooth(dims, B, order=8) -> np.ndarray:
    d = _i32(dims)
    B = _i32(B).ravel()
    Bs = np.zeros(B.size)
    _load().orc_smooth(_p(d), _p(B), int(order), _p(Bs))
    return Bs


def kmeans(Bs, max_iter=100):
    Bs = _f64(Bs).ravel()
    S = np.zeros(Bs.size, np.uint8)
    cl, cv = C.c_double(), C.c_double()
    it = _load().orc_kmeans(Bs.size, _p(Bs), int(max_iter), _p(S), C.byref(cl), C.byref(cv))
    return S, cl.value, cv.value, it


def ms_energy(dims, rho, c_l, c_v, nu, S) -> float:
    """Eq. 13 of labels S with fixed densities (perimeter = liquid/vapor faces)"""
    d = _i32(dims)
    rho = _f64(rho).ravel()
    S = np.ascontiguousarray(S, dtype=np.uint8).ravel()
    return _load().orc_ms_energy(_p(d), _p(rho), float(c_l), float(c_v), float(nu), _p(S))


def ms_segment(dims, rho, c_l, c_v, nu, iters):
    """Eq. 13 minimised by the convex relaxation; returns (labels, relaxed u)"""
    d = _i32(dims)
    rho = _f64(rho).ravel()
    S = np.zeros(rho.size, np.uint8)
    u = np.zeros(rho.size)
    _load().orc_ms_segment(_p(d), _p(rho), float(c_l), float(c_v), float(nu), int(iters),
                           _p(S), _p(u))
    return S, u


def ms_alternate(dims, rho, nu, iters, max_outer, c_l, c_v):
    """Eq. 13 over sets and densities; returns (labels, c_l, c_v, rounds)"""
    d = _i32(dims)
    rho = _f64(rho).ravel()
    S = np.zeros(rho.size, np.uint8)
    cl = C.c_double(c_l)
    cv = C.c_double(c_v)
    rounds = _load().orc_ms_alternate(_p(d), _p(rho), float(nu), int(iters), int(max_outer),
                                      _p(S), C.byref(cl), C.byref(cv))
    return S, cl.value, cv.value, rounds


def ms_detect(dims, Bs, inv_scale, nu, iters, max_outer, S):
    """Eq. 13 as the detection's segmentation step from labels S on
    rho = Bs * inv_scale; returns (labels, rounds)"""
    d = _i32(dims)
    Bs = _f64(Bs).ravel()
    S = np.ascontiguousarray(S, dtype=np.uint8).ravel().copy()
    rounds = _load().orc_ms_detect(_p(d), _p(Bs), float(inv_scale), float(nu), int(iters),
                                   int(max_outer), _p(S))
    return S, rounds


def label_components(dims, S, phase):
    """Section 4.2 / Algorithm 4.1: (labels, count) of the phase's components."""
    d = _i32(dims)
    S = np.ascontiguousarray(S, dtype=np.uint8).ravel()
    lab = np.zeros(max(S.size, 1), np.int32)
    nc = _load().orc_label_components(_p(d), _p(S), int(phase), _p(lab))
    return lab[: S.size], int(nc)


def remove_small_components(dims, S, min_voxels):
    """Section 4.2: (new labels, voxels changed) after removing the small
    liquid, then vapor components."""
    d = _i32(dims)
    out = np.array(np.ascontiguousarray(S, dtype=np.uint8).ravel())
    flipped = _load().orc_remove_small_components(_p(d), _p(out), int(min_voxels))
    return out, int(flipped)


def godunov(a, h) -> float:
    a = _f64(a)
    h = _f64(h)
    return _load().orc_godunov(_p(a), _p(h))


def fsm(dims, h, S, cap=0.0):
    d = _i32(dims)
    h = _f64(h)
    S = np.ascontiguousarray(S, dtype=np.uint8).ravel()
    D = np.zeros(S.size)
    rounds = _load().orc_fsm(_p(d), _p(h), _p(S), float(cap), _p(D))
    return D, rounds


def cfsm(dims, h, S, r_grid, iter_max=0, eps=0.0):
    d = _i32(dims)
    h = _f64(h)
    S = np.ascontiguousarray(S, dtype=np.uint8).ravel()
    D = np.zeros(S.size)
    if iter_max <= 0:
        iter_max = 4 * int(max(dims))
    it = _load().orc_cfsm(_p(d), _p(h), _p(S), float(r_grid), int(iter_max), float(eps), _p(D))
    return D, it


def particle_distance(x, L, dims, D) -> np.ndarray:
    x = _f64(x).reshape(-1, 3)
    L = _f64(L)
    d = _i32(dims)
    D = _f64(D).ravel()
    out = np.zeros(max(x.shape[0], 1))
    _load().orc_particle_distance(x.shape[0], _p(x), _p(L), _p(d), _p(D), _p(out))
    return out[: x.shape[0]]


class _DetectParams(C.Structure):
    _fields_ = [("rc_min", C.c_double), ("rc_max", C.c_double), ("alpha", C.c_double),
                ("voxel", C.c_double), ("smooth_order", C.c_int),
                ("kmeans_max_iter", C.c_int), ("cfsm_iter_max", C.c_int),
                ("cfsm_eps", C.c_double), ("n_classes", C.c_int),
                ("min_component_voxels", C.c_int), ("cutoff_fn", C.c_int),
                ("segmentation", C.c_int), ("ms_iters", C.c_int), ("ms_outer", C.c_int),
                ("ms_nu", C.c_double)]


class _RunParams(C.Structure):
    _fields_ = [("det", _DetectParams), ("dt", C.c_double), ("mass", C.c_double),
                ("eps", C.c_double), ("sigma", C.c_double), ("cell_min", C.c_double),
                ("detect_every", C.c_int)]


@dataclass
class DetectParams:
    rc_min: float = 3.0
    rc_max: float = 6.0
    alpha: float = -0.5
    voxel: float = 1.0
    smooth_order: int = 8
    kmeans_max_iter: int = 100
    cfsm_iter_max: int = 0
    cfsm_eps: float = 0.0
    n_classes: int = 4
    min_component_voxels: int = 0
    cutoff_fn: int = 0
    segmentation: int = 0
    ms_iters: int = 50
    ms_outer: int = 1
    ms_nu: float = 0.005

    def _c(self) -> _DetectParams:
        return _DetectParams(self.rc_min, self.rc_max, self.alpha, self.voxel,
                             self.smooth_order, self.kmeans_max_iter, self.cfsm_iter_max,
                             self.cfsm_eps, self.n_classes, self.min_component_voxels,
                             self.cutoff_fn, self.segmentation, self.ms_iters, self.ms_outer,
                             self.ms_nu)


@dataclass
class Detection:
    dims: tuple
    B: np.ndarray
    Bs: np.ndarray
    S: np.ndarray
    D: np.ndarray
    d: np.ndarray
    rc: np.ndarray
    cls: np.ndarray
    cfsm_iters: int


def detect(x, L, p: DetectParams) -> Detection:
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    L = _f64(L)
    dims = grid_dims(L, p.voxel)
    nv = int(np.prod(dims))
    dims_a = np.zeros(3, np.int32)
    B = np.zeros(nv, np.int32)
    Bs = np.zeros(nv)
    S = np.zeros(nv, np.uint8)
    D = np.zeros(nv)
    d = np.zeros(max(n, 1))
    rc = np.zeros(max(n, 1))
    cls = np.zeros(max(n, 1), np.uint8)
    cp = p._c()
    it = _load().orc_detect(n, _p(x), _p(L), C.byref(cp), _p(dims_a), _p(B), _p(Bs), _p(S),
                            _p(D), _p(d), _p(rc), _p(cls))
    return Detection(tuple(int(v) for v in dims_a), B, Bs, S, D, d[:n], rc[:n], cls[:n], it)


@dataclass
class RunParams:
    det: DetectParams
    dt: float = 0.005
    mass: float = 1.0
    eps: float = 1.0
    sigma: float = 1.0
    cell_min: float = 1.5
    detect_every: int = 2


def run(x, v, L, p: RunParams, nsteps: int, step0: int = 0):
    """Velocity Verlet with the DCM cadence; returns (x, v, f, rc, epot, ekin)."""
    x = _f64(x).reshape(-1, 3).copy()
    v = _f64(v).reshape(-1, 3).copy()
    n = x.shape[0]
    L = _f64(L)
    f = np.zeros((max(n, 1), 3))
    rc = np.zeros(max(n, 1))
    epot = np.zeros(nsteps + 1)
    ekin = np.zeros(nsteps + 1)
    cp = _RunParams(p.det._c(), p.dt, p.mass, p.eps, p.sigma, p.cell_min, p.detect_every)
    rcode = _load().orc_run(n, _p(x), _p(v), _p(L), C.byref(cp), int(step0), int(nsteps),
                            _p(f), _p(rc), _p(epot), _p(ekin))
    if rcode != 0:
        raise ValueError("oracle: cutoff not below half the shortest box edge")
    return x, v, f[:n], rc[:n], epot, ekin
