"""Seeded synthetic inputs shaped like the thesis's workloads.

This module holds none of the method's arithmetic: it only places particles
and draws velocities.  Both the CUDA path (tests, bench) and the CPU oracle
(tests) take their inputs from here, so neither side generates data for the
other.

Workload shapes (Springer, arxiv 1502.03234, Section 6 and Fig. 1/32): a
Lennard-Jones liquid slab of density 0.8 across the centre of an elongated
periodic box (L_z = 4 L_x), vapor of density ~0.005 elsewhere, Maxwell
velocities at T* = 0.7.  The box edge is derived from N so that N, the two
densities and the aspect ratio hold together:
    L_x = (N / (0.8 * 4/3 + 0.005 * 8/3))^(1/3) = (N / 1.08)^(1/3),
rounded to a whole number of FCC cells of edge a = (4/0.8)^(1/3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

RHO_L = 0.8
RHO_V = 0.005


@dataclass
class Slab:
    x: np.ndarray          # (N, 3) float64, wrapped into [0, L)
    v: np.ndarray          # (N, 3) float64
    box: tuple             # (Lx, Ly, Lz)
    n_liquid: int
    z_planes: tuple        # nominal liquid extent (z_lo, z_hi) of the flat slab
    temperature: float
    seed: int


def fcc_edge(rho: float = RHO_L) -> float:
    return (4.0 / rho) ** (1.0 / 3.0)


def box_for(n: int, rho_l: float = RHO_L, rho_v: float = RHO_V,
            min_edge: float | None = None) -> tuple[int, tuple]:
    """(n_x FCC cells, (Lx, Ly, Lz)) for an N-particle slab.  min_edge raises
    the lateral edge for small N (the slab then gets thinner), so that a
    cutoff of about (min_edge - a few cells)/2 still fits the minimum image."""
    a = fcc_edge(rho_l)
    lx_target = (n / (rho_l * 4.0 / 3.0 + rho_v * 8.0 / 3.0)) ** (1.0 / 3.0)
    nx = max(1, int(round(lx_target / a)))
    if min_edge:
        nx = max(nx, int(math.ceil(min_edge / a)))
    L = nx * a
    return nx, (L, L, 4.0 * L)


def _fcc_sites(nx: int, ny: int, nz: int, a: float, z0: float) -> np.ndarray:
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    basis = (basis + 0.25) * a
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    corners = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) * a
    sites = (corners[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    sites[:, 2] += z0
    return sites


def _wrap(x: np.ndarray, box) -> np.ndarray:
    L = np.asarray(box, np.float64)
    x = x - np.floor(x / L) * L
    x[x >= L] -= np.broadcast_to(L, x.shape)[x >= L]
    x[x < 0] = 0.0
    return x


def _capillary(xy: np.ndarray, box, phases: np.ndarray, amp: float) -> np.ndarray:
    """sum of three sinusoidal modes (1,0), (0,1), (1,1) with amplitude amp/3"""
    modes = ((1, 0), (0, 1), (1, 1))
    h = np.zeros(xy.shape[0])
    for (mx, my), ph in zip(modes, phases):
        h += np.sin(2 * np.pi * (mx * xy[:, 0] / box[0] + my * xy[:, 1] / box[1]) + ph)
    return h * (amp / 3.0)


def _place_vapor(rng, count, box, occupied, inside_liquid, min_sep):
    """uniform vapor, redrawn when inside the liquid or within min_sep of any
    particle already placed"""
    if count <= 0:
        return np.zeros((0, 3))
    from scipy.spatial import cKDTree

    L = np.asarray(box, np.float64)
    tree = cKDTree(_wrap(occupied.copy(), box), boxsize=L) if len(occupied) else None
    accepted = np.zeros((0, 3))
    for _ in range(10000):
        need = count - accepted.shape[0]
        if need <= 0:
            break
        cand = rng.random((max(2 * need, 64), 3)) * L
        cand = cand[~inside_liquid(cand)]
        if tree is not None and len(cand):
            cand = cand[tree.query(cand, k=1)[0] >= min_sep]
        if accepted.shape[0] and len(cand):
            acc_tree = cKDTree(accepted, boxsize=L)
            cand = cand[acc_tree.query(cand, k=1)[0] >= min_sep]
        if len(cand) > 1:
            # greedy: drop the later candidate of every close pair in the batch
            pairs = cKDTree(cand, boxsize=L).query_pairs(min_sep, output_type="ndarray")
            drop = np.zeros(len(cand), bool)
            for i, j in sorted(map(tuple, pairs)):
                if not drop[i]:
                    drop[j] = True
            cand = cand[~drop]
        accepted = np.vstack([accepted, cand[:need]])
    if accepted.shape[0] < count:
        raise RuntimeError("vapor placement did not converge")
    return accepted


def maxwell(rng, n: int, temperature: float, mass: float = 1.0) -> np.ndarray:
    """Maxwell velocities, centre-of-mass motion removed, rescaled to exactly
    T with 3N-3 degrees of freedom."""
    if n == 0:
        return np.zeros((0, 3))
    v = rng.normal(0.0, math.sqrt(temperature / mass), size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0)
        ke2 = mass * float(np.sum(v * v))
        v *= math.sqrt((3 * n - 3) * temperature / ke2)
    return v


def make_slab(n: int, temperature: float = 0.7, seed: int = 0, *, rho_l: float = RHO_L,
              rho_v: float = RHO_V, jitter: float = 0.05, min_sep: float = 0.8,
              capillary_amp: float = 0.0, mass: float = 1.0,
              min_edge: float | None = None) -> Slab:
    """Jittered-FCC liquid slab across the box centre plus uniform vapor.

    capillary_amp > 0 perturbs both liquid/vapor planes by three sinusoidal
    modes with independent random phases (|h| <= capillary_amp)."""
    rng = np.random.default_rng(seed)
    a = fcc_edge(rho_l)
    nx, box = box_for(n, rho_l, rho_v, min_edge)
    Lx, Ly, Lz = box
    denom = 4 * nx * nx - rho_v * Lx * Ly * a
    nz = int(math.floor((n - rho_v * Lx * Ly * Lz) / denom))
    nz = max(1, min(nz, int(Lz / a) - 2))
    while 4 * nx * nx * nz > n and nz > 1:
        nz -= 1
    t = nz * a
    z0 = 0.5 * (Lz - t)
    target_liquid = 4 * nx * nx * nz
    if capillary_amp > 0.0:
        extra = int(math.ceil(capillary_amp / a)) + 1
        sites = _fcc_sites(nx, nx, nz + 2 * extra, a, z0 - extra * a)
        ph_lo = rng.uniform(0, 2 * np.pi, 3)
        ph_hi = rng.uniform(0, 2 * np.pi, 3)
        z_lo = z0 + _capillary(sites[:, :2], box, ph_lo, capillary_amp)
        z_hi = z0 + t + _capillary(sites[:, :2], box, ph_hi, capillary_amp)
        sites = sites[(sites[:, 2] >= z_lo) & (sites[:, 2] < z_hi)]
        if sites.shape[0] > target_liquid:
            drop = rng.choice(sites.shape[0], sites.shape[0] - target_liquid, replace=False)
            sites = np.delete(sites, drop, axis=0)

        def inside(c):
            lo = z0 + _capillary(c[:, :2], box, ph_lo, capillary_amp)
            hi = z0 + t + _capillary(c[:, :2], box, ph_hi, capillary_amp)
            return (c[:, 2] >= lo - 0.5 * a) & (c[:, 2] < hi + 0.5 * a)
    else:
        sites = _fcc_sites(nx, nx, nz, a, z0)

        def inside(c):
            return (c[:, 2] >= z0 - 0.25 * a) & (c[:, 2] < z0 + t + 0.25 * a)

    liquid = sites + rng.uniform(-jitter, jitter, size=sites.shape)
    n_vap = n - liquid.shape[0]
    vapor = _place_vapor(rng, n_vap, box, liquid, inside, min_sep)
    x = _wrap(np.vstack([liquid, vapor]), box)
    v = maxwell(rng, n, temperature, mass)
    return Slab(x=np.ascontiguousarray(x), v=np.ascontiguousarray(v), box=box,
                n_liquid=int(liquid.shape[0]), z_planes=(z0, z0 + t),
                temperature=temperature, seed=seed)


def make_gas(n: int, box, seed: int = 0, temperature: float = 0.7, min_sep: float = 0.85,
             mass: float = 1.0):
    """Uniform random particles with a minimum separation (small tests)."""
    rng = np.random.default_rng(seed)
    x = _place_vapor(rng, n, box, np.zeros((0, 3)), lambda c: np.zeros(len(c), bool), min_sep)
    return np.ascontiguousarray(x), maxwell(rng, n, temperature, mass)


@dataclass
class EnsembleMember:
    slab: Slab
    n: int
    temperature: float


def make_ensemble(count: int = 64, n_min: int = 4096, n_max: int = 131072,
                  t_min: float = 0.65, t_max: float = 0.85, seed: int = 0):
    """Independent slabs with N log-uniform in [n_min, n_max] and T uniform."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        temp = float(rng.uniform(t_min, t_max))
        out.append(EnsembleMember(make_slab(n, temp, seed=seed * 100003 + k + 1), n, temp))
    return out


@dataclass
class Request:
    rid: int
    arrival_s: float
    n: int
    nsteps: int
    seed: int
    temperature: float


def make_trace(count: int = 400, rate_per_s: float = 20.0, n_min: int = 2048,
               n_max: int = 524288, steps_min: int = 100, steps_max: int = 2000,
               temperature: float = 0.7, seed: int = 0):
    """Poisson arrival stream of slab requests (finite, seeded)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        steps = int(rng.integers(steps_min, steps_max + 1))
        out.append(Request(k, t, n, steps, seed * 7919 + k + 1, temperature))
    return out
