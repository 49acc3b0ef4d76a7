"""Autotuner of the DCM force kernel's launch shape.

The thesis balances its force loop with OpenMP's schedule(dynamic,20)
(Section 5.1, Algorithm 5.1); here the work queue of the force kernels does
that, and what is left to choose is the shape the kernels run with.  It is
tuned on the live system and depends on the precision:

* DCM_MIXED runs the warp kernels.  Without Verlet lists the direct warp walk
  has no shape parameter; with lists, list_lanes sets how many lanes share
  one particle of the list force (4, 8, 16 or 32): few lanes suit the short
  lists of bulk particles (r_c,min), many lanes the long lists of
  interfacial ones (up to r_c,max, 8-13x the pairs).  After the uniform
  choice, list_lanes_class tries lanes per cutoff class (the class-ordered
  list force), by coordinate descent from the heaviest class.
* DCM_FP64 runs the lanes walk: per cutoff class the number of lanes that
  share one particle (1..32), searched by coordinate descent heaviest class
  first, and the threads per block.

tune() also searches the link-cell edge (a fraction of r_c,min: smaller
cells trim the candidate volume towards the cutoff sphere, larger ones cut
per-row overhead), which is fixed when a handle is created; tune_live()
chooses among launch shapes on an existing handle (a System or an Ensemble,
whose one persistent force launch covers every member).  Every candidate is
timed with the library's per-phase CUDA events (the force phase of real
steps).  Results are cached per (N bucket, r_c,min, r_c,max, precision, skin)
in a JSON file, so systems of similar size reuse the choice without
re-tuning.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from dataclasses import asdict, dataclass, field

from . import dcm

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning_cache.json")
LANES = (1, 2, 4, 8, 16, 32)
LIST_LANES = (4, 8, 16, 32)
CELL_FRACTIONS = (1.0 / 3.0, 0.4, 0.5, 2.0 / 3.0)
BLOCKS = (128, 256)


@dataclass
class Tuning:
    cell_min: float
    block: int
    lanes: list = field(default_factory=lambda: [4, 8, 8, 8, 8, 8, 8, 8])
    force_ms: float = float("nan")
    walk: int = dcm.DCM_WALK_WARP
    list_lanes: int = 8
    list_lanes_class: list = None      # per cutoff class (class-ordered list force), or None


def key(n: int, rc_min: float, rc_max: float, precision: int, skin: float = 0.0) -> str:
    return f"v4|n2^{round(math.log2(max(n, 1)))}|rc{rc_min:g}/{rc_max:g}|p{precision}|s{skin:g}"


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = CACHE) -> None:
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def force_ms(sy: dcm.System, reps: int = 5) -> float:
    """median device time of the force phase over reps steps"""
    sy.set_timing(True)
    sy.step(1)
    out = []
    for _ in range(reps):
        sy.step(1)
        out.append(sy.phase_times()["force"])
    return statistics.median(out)


def _system(box, x, v, params: dcm.dcm_params, cell_min: float, stream=None) -> dcm.System:
    p = dcm.dcm_params.from_buffer_copy(params)
    p.cell_min = cell_min
    sy = dcm.System(box, len(x), p, stream=stream)
    sy.set_state(x, v)
    sy.compute_forces()
    return sy


PER_CLASS_MARGIN = 0.03   # a per-class shape must beat the uniform one by this much


def _tune_list_classes(sy, K: int, G0: int, t0: float, reps: int, list_lanes, log=None):
    """lanes per cutoff class of the class-ordered list force: coordinate
    descent from G0 everywhere, heaviest class first.  Returns (lanes per
    class, force ms), or (None, t0) unless the best per-class shape beats t0
    by PER_CLASS_MARGIN: the class-ordered queue gives up the slot order's L1
    sharing, which a system tuned early (a lattice start) but run long gets
    back (measured: 1.5 % ahead at tuning, 1 % behind over 1000 steps)."""
    cur = [G0] * dcm.DCM_MAX_CLASSES
    sy.set_tuning([1], 128, dcm.DCM_WALK_WARP, G0, cur)
    t_cur = force_ms(sy, reps)
    if log:
        log(f"list lanes per class {cur[:K]}: force {t_cur:.4f} ms")
    for q in reversed(range(K)):
        for G in list_lanes:
            if G == cur[q]:
                continue
            trial = list(cur)
            trial[q] = G
            sy.set_tuning([1], 128, dcm.DCM_WALK_WARP, G0, trial)
            t = force_ms(sy, reps)
            if log:
                log(f"list lanes per class {trial[:K]}: force {t:.4f} ms")
            if t < t_cur:
                cur, t_cur = trial, t
    return (cur, t_cur) if t_cur < (1.0 - PER_CLASS_MARGIN) * t0 else (None, t0)


def _tune_mixed(sy: dcm.System, params, reps, list_lanes, log, cell):
    """the warp kernels: list_lanes with Verlet lists (uniform, then per
    cutoff class), nothing without"""
    best = None
    shapes = list_lanes if params.skin > 0 else (8,)
    for G in shapes:
        sy.set_tuning([1], 128, dcm.DCM_WALK_WARP, G)
        t = force_ms(sy, reps)
        if log:
            log(f"cell {cell:.3f} warp kernels, list lanes {G}: force {t:.4f} ms")
        if best is None or t < best.force_ms:
            best = Tuning(cell_min=cell, block=128, lanes=[1] * dcm.DCM_MAX_CLASSES,
                          force_ms=t, walk=dcm.DCM_WALK_WARP, list_lanes=G)
    if params.skin > 0 and params.n_classes > 1:
        cls, t = _tune_list_classes(sy, params.n_classes, best.list_lanes, best.force_ms, reps,
                                    list_lanes, log)
        if cls is not None:
            best.list_lanes_class, best.force_ms = cls, t
    return best


def _tune_fp64(sy: dcm.System, params, reps, blocks, lanes, log, cell):
    """the lanes walk: lanes per cutoff class (coordinate descent, heaviest
    class first) for each block size"""
    K = params.n_classes
    best = None
    for block in blocks:
        cur = [4] + [8] * (dcm.DCM_MAX_CLASSES - 1)
        sy.set_tuning(cur, block, dcm.DCM_WALK_LANES)
        t_cur = force_ms(sy, reps)
        for q in reversed(range(K)):
            for G in lanes:
                if G == cur[q]:
                    continue
                trial = list(cur)
                trial[q] = G
                sy.set_tuning(trial, block, dcm.DCM_WALK_LANES)
                t = force_ms(sy, reps)
                if t < t_cur:
                    cur, t_cur = trial, t
        if log:
            log(f"cell {cell:.3f} block {block} lanes {cur[:K]} force {t_cur:.4f} ms")
        if best is None or t_cur < best.force_ms:
            best = Tuning(cell_min=cell, block=block, lanes=cur, force_ms=t_cur,
                          walk=dcm.DCM_WALK_LANES)
    return best


def tune(box, x, v, params: dcm.dcm_params, *, reps: int = 5, stream=None,
         fractions=CELL_FRACTIONS, blocks=BLOCKS, lanes=LANES, list_lanes=LIST_LANES,
         log=None) -> Tuning:
    """Search the link-cell edge and the launch shape of this precision on
    this system's state; returns the fastest."""
    best: Tuning | None = None
    for frac in fractions:
        cell = frac * params.rc_min
        try:
            sy = _system(box, x, v, params, cell, stream)
        except dcm.DcmError:
            continue
        try:
            if params.precision == dcm.DCM_MIXED:
                t = _tune_mixed(sy, params, reps, list_lanes, log, cell)
            else:
                t = _tune_fp64(sy, params, reps, blocks, lanes, log, cell)
        finally:
            sy.close()
        if best is None or t.force_ms < best.force_ms:
            best = t
    if best is None:
        raise RuntimeError("autotune: no cell size fits this box")
    return best


def live_candidates(precision: int) -> tuple:
    """launch shapes tried on a live handle (the cell edge is fixed at
    creation)"""
    if precision == dcm.DCM_MIXED:
        return tuple({"walk": dcm.DCM_WALK_WARP, "lanes": [1], "block": 128, "list_lanes": G}
                     for G in LIST_LANES)
    return ({"walk": dcm.DCM_WALK_LANES, "lanes": [4, 4, 8, 8], "block": 128},
            {"walk": dcm.DCM_WALK_LANES, "lanes": [8, 8, 16, 16], "block": 128},
            {"walk": dcm.DCM_WALK_LANES, "lanes": [16, 16, 32, 32], "block": 128},
            {"walk": dcm.DCM_WALK_LANES, "lanes": [32, 32, 32, 32], "block": 256})


def tune_live(sy: dcm.System, *, reps: int = 5, candidates=None, per_class: bool = True,
              log=None) -> dict:
    """Time each launch shape on a live handle (a System or an Ensemble: the
    ensemble's one persistent force launch covers every member), keep the
    fastest and leave it set.  With DCM_MIXED Verlet lists and per_class,
    lanes per cutoff class are tried after the uniform shapes.  Returns the
    choice with its force time."""
    if candidates is None:
        candidates = live_candidates(sy.params.precision)
    best = None
    for c in candidates:
        try:
            sy.set_tuning(c["lanes"], c["block"], c["walk"], c.get("list_lanes", 8))
        except dcm.DcmError:
            continue
        t = force_ms(sy, reps)
        if log:
            log(f"walk {c['walk']} lanes {c['lanes']} block {c['block']} list lanes "
                f"{c.get('list_lanes', 8)}: force {t:.4f} ms")
        if best is None or t < best["force_ms"]:
            best = dict(c, force_ms=t)
    p = sy.params
    if (per_class and p.precision == dcm.DCM_MIXED and p.skin > 0 and p.n_classes > 1
            and "list_lanes" in best):
        cls, t = _tune_list_classes(sy, p.n_classes, best["list_lanes"], best["force_ms"], reps,
                                    LIST_LANES, log)
        if cls is not None:
            best = dict(best, list_lanes_class=cls, force_ms=t)
    sy.set_tuning(best["lanes"], best["block"], best["walk"], best.get("list_lanes", 8),
                  best.get("list_lanes_class"))
    return best


def tuned_system(box, x, v, params: dcm.dcm_params, *, stream=None, cache_path: str = CACHE,
                 retune: bool = False, log=None) -> tuple[dcm.System, Tuning]:
    """A system built with the cached (or freshly tuned) launch shape."""
    cache = load_cache(cache_path)
    k = key(len(x), params.rc_min, params.rc_max, params.precision, params.skin)
    if retune or k not in cache:
        t = tune(box, x, v, params, stream=stream, log=log)
        cache[k] = asdict(t)
        save_cache(cache, cache_path)
    t = Tuning(**cache[k])
    sy = _system(box, x, v, params, t.cell_min, stream)
    sy.set_tuning(t.lanes, t.block, t.walk, t.list_lanes, t.list_lanes_class)
    return sy, t
