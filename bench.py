#!/usr/bin/env python3
"""Benchmark of the DCM hot path: atom-steps/s of the full DCM step
(velocity Verlet + interface detection every other step + link-cell sort +
dynamic-cutoff LJ forces) on a synthetic LJ liquid/vapor slab.

Workload (the N = 262,144 slab): density-0.8 jittered-FCC liquid across the
centre of an L x L x 4L periodic box, vapor elsewhere, T* = 0.7,
r_c,min = 3, r_c,max = 6 (exponential Eq. 7, alpha = -0.5), 1-sigma voxels,
detection every 2 steps, dt = 0.005.  The timed arm is the mixed-precision
path (FP32 pair / FP64 state); the plain FP64 GPU path is measured on the
same system and reported beside it.

One JSON line on stdout (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on the host cores, on a bounded sample of the workload.

Other workloads (one GPU, one JSON line each; not the default):
  --workload wavy      N = 2,097,152 slab whose two interfaces carry
                       capillary-wave-like sinusoidal z offsets (amplitude
                       1 sigma, random phases), r_c 3/7, mixed precision,
                       200 steps, plus a weak-scaling sweep in N (--sweep)
  --workload ensemble  64 independent slabs, N log-uniform in [4096, 131072],
                       T* uniform in [0.65, 0.85], one handle (one persistent
                       force launch per step, the step a CUDA graph), launch
                       shape tuned on the live ensemble, 500 steps
  --workload serving   Poisson request stream (20 req/s), N log-uniform in
                       [2048, 524288], nsteps uniform in [100, 2000], HBM
                       budget 120 GB, continuous batching: p50/p99 latency
                       and aggregate atom-steps/s
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "atom-steps/s of DCM step (forces+interface) vs plain FP64 GPU path; p50/p99 latency"
UNIT = "atom-steps/s"
N_DEFAULT = 262144
FP32_LANES_PER_SM = 128          # Blackwell SM: 4 sub-partitions x 32 FP32 lanes


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0                # fallback figure when the measured file is absent


HBM_PEAK_GBS = _hbm_peak()
FLOPS_PER_PAIR = 24              # 8 (distance test) + 16 (LJ force), per in-cutoff pair
FLOPS_PER_CHECK = 8              # per candidate distance check (a Verlet-list entry)
FLOPS_PER_FORCE = 16             # per in-cutoff pair: rcp, (s/r)^6, the scalar, 3 FMA
# DRAM bytes (read + write) per force launch of the direct walk (skin 0) from the committed
# ncu capture of that kernel on this workload; None: not captured
FORCE_TRAFFIC = {"mixed": None, "fp64": None}
# DRAM bytes (read + write) per launch of the Verlet-list force kernel
# (k_force_list_warp, N = 262,144, skin 0.7, skin_time 0.06, skin_floor 0.07) from the
# committed ncu capture of that kernel on this workload, with the list entries in
# use at the captured launches; the reported traffic scales it by the algorithmic bytes
LIST_TRAFFIC = {"k_force_list_warp": {"bytes": 205.36e6 + 4.49e6, "entries": 39320880}}
LIST_TRAFFIC_CONFIG = (0.7, 0.06, 0.07, 1.0)    # skin, skin_time, skin_floor, list_margin
# bytes the list kernel must move per particle besides its list entries: own
# position, cutoff constants, id/cell, list start and count, queue slot, the
# force written and the pair count
LIST_BYTES_PER_PARTICLE = 16 + 16 + 16 + 4 + 4 + 4 + 24 + 4
LIST_BYTES_PER_ENTRY = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 1000; wavy 200; ensemble 500)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="dcm", choices=["dcm", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--ens-steps", type=int, default=50,
                    help="steps of the 64-slab ensemble comparison, batched mixed against "
                         "per-system FP64 (0: skip)")
    ap.add_argument("--wavy-steps", type=int, default=30,
                    help="steps of the 2.1M-atom capillary-wave slab leg of the default line "
                         "(0: skip)")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the serving leg of the default line (nsteps up to 500; "
                         "0: skip)")
    ap.add_argument("--seg-steps", type=int, default=20,
                    help="steps of the detection-with-Eq.-13 comparison (0: skip)")
    ap.add_argument("--skin", type=float, default=0.7,
                    help="Verlet-list skin in sigma (0: direct link-cell walk every step)")
    ap.add_argument("--cell-min", type=float, default=0.0,
                    help="link-cell edge target in sigma (0: the library's, r_c,min / 2)")
    ap.add_argument("--list-lanes", type=int, default=0, choices=[0, 4, 8, 16, 32],
                    help="lanes per particle of the Verlet-list force (0: tuned on a scratch "
                         "copy of the system before the timed run, see --no-tune)")
    ap.add_argument("--list-lanes-class", default=None,
                    help="with --list-lanes: lanes per cutoff class, comma-separated (the "
                         "class-ordered list force), e.g. 8,8,16,16")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default launch shape instead of tuning it")
    ap.add_argument("--step-graph", default="branched", choices=["branched", "flat"],
                    help="flat: no conditional nodes in the step graph (for per-kernel profiling)")
    ap.add_argument("--skin-time", type=float, default=0.06,
                    help="adaptive skin shares: share = clamp(skin_time |v| + skin_time^2 |F| / 2m, "
                         "skin_floor, skin/2); 0: skin/2 for every particle")
    ap.add_argument("--skin-floor", type=float, default=0.07)
    ap.add_argument("--min-component", type=int, default=0,
                    help="small-component removal (Section 4.2): components of either phase "
                         "below this many voxels change phase; 0: off")
    ap.add_argument("--list-margin", type=float, default=1.0,
                    help="interface-distance margin of the Verlet-list radius in sigma")
    ap.add_argument("--workload", default="slab",
                    choices=["slab", "wavy", "ensemble", "serving", "accuracy"])
    ap.add_argument("--sweep", default="131072,262144,524288,1048576",
                    help="wavy: further N of the weak-scaling sweep")
    ap.add_argument("--sweep-steps", type=int, default=40)
    ap.add_argument("--requests", type=int, default=120, help="serving: trace length")
    a = ap.parse_args()
    if a.list_lanes_class:
        a.list_lanes_class = [int(g) for g in a.list_lanes_class.split(",")]
    if a.steps is None:
        a.steps = {"slab": 1000, "wavy": 200, "ensemble": 500, "serving": 0, "accuracy": 0}[a.workload]
    return a


def workload_config(n, precision):
    return {"workload": f"LJ liquid/vapor slab N={n}, L x L x 4L periodic, rho_l=0.8, T*=0.7, "
                        f"DCM r_c 3/6 (Eq. 7, alpha=-0.5), 1-sigma voxels, detection every 2 steps",
            "n": n, "rc_min": 3.0, "rc_max": 6.0, "detect_every": 2, "dt": 0.005,
            "precision": precision,
            "l2": L2_NOTE + "; each step timed alone"}


def force_kernel_name(dcm, sy, prec, skin):
    if prec != dcm.DCM_MIXED:
        return "k_force (fp64)"
    return "k_force_list_warp + k_force_warp (mixed, Verlet lists)" if skin > 0 else "k_force_warp (mixed)"


# ---- clocks sampled during the timed region ------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        # raw samples: $DCM_CLOCKS_DIR (default: the temp directory)
        out = os.environ.get("DCM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None or not os.path.exists(self.path):
            out["reasons"] = ["nvidia-smi unavailable"]
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(smax)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


# ---- reference arm: the FP64 CPU oracle ----------------------------------------------
def oracle_rate(n_sample: int, target_s: float, max_steps: int = 2000, seed: int = 1,
                min_component: int = 0, threads: int = 0):
    """atom-steps/s of the FP64 oracle (all host cores, or `threads`) on an
    n_sample slab with the same densities, cutoffs and cadence."""
    import oracle
    from paper_1502_03234_gb300 import slabgen

    cores = threads if threads > 0 else (os.cpu_count() or 1)
    cores = oracle.set_threads(cores)
    s = slabgen.make_slab(n_sample, seed=seed)
    p = oracle.RunParams(det=oracle.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0,
                                                 min_component_voxels=min_component),
                         dt=0.005, cell_min=1.5, detect_every=2)
    t0 = time.perf_counter()
    oracle.run(s.x, s.v, s.box, p, 2)                  # setup + 2 steps: calibration
    t_cal = time.perf_counter() - t0
    steps = int(max(2, min(max_steps, 2 * round(target_s / max(t_cal, 1e-3)))))
    t0 = time.perf_counter()
    oracle.run(s.x, s.v, s.box, p, steps)
    dt = time.perf_counter() - t0
    return n_sample * steps / dt, cores, steps, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1502_03234_gb300 import slabgen

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n_sample = 16384
    s = slabgen.make_slab(n_sample, seed=1)
    p = oracle.RunParams(det=oracle.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0,
                                                 min_component_voxels=args.min_component),
                         dt=0.005, cell_min=1.5, detect_every=2)
    x, v = s.x, s.v
    if args.warmup > 0:
        x, v, *_ = oracle.run(x, v, s.box, p, args.warmup)
    # one call for all timed steps: its setup (one detection + one force
    # evaluation) is the only work beyond the K steps
    t0 = time.perf_counter()
    oracle.run(x, v, s.box, p, args.steps, step0=args.warmup)
    total = time.perf_counter() - t0
    value = n_sample * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.n, "fp64 CPU oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"N={n_sample} slab of the same shape and cutoffs "
                                       f"(atom-steps/s is size-independent for this linear-time "
                                       f"method); K oracle steps in one run after W warm-up steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0



# ---- further workloads (one GPU) -------------------------------------------------------
class L2Flush:
    """Evicts the timed program's data from the 129 MB L2 before a step: a
    256 MiB write, then a 256 MiB read, so that the write's dirty lines are
    written back here rather than inside the next timed step."""

    def __init__(self, torch):
        self.w = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        self.r = torch.zeros(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def __call__(self):
        self.w.zero_()
        self.s = self.r.amax()


L2_NOTE = ("flushed before every timed step (256 MiB write, then a 256 MiB read that "
           "drains the write's dirty lines)")


def _launches(st, kinds):
    """kernels the timed steps launched: each step is one CUDA graph whose
    kernel count depends on detection and, with Verlet lists, on whether the
    step rebuilt them (the rebuild-only kernels sit in conditional nodes)"""
    n = 0
    for det, rebuilt in kinds:
        if det:
            n += st.kernels_detect if rebuilt else st.kernels_detect_reuse
        else:
            n += st.kernels_plain if rebuilt else st.kernels_plain_reuse
    return n


def _kind(sy, builds_before):
    """(detected, rebuilt) of the step just run, the list builds so far and
    the entries of the lists in use"""
    st = sy.stats()
    every = sy.params.detect_every
    return ((every > 0 and st.step % every == 0, st.list_builds != builds_before), st.list_builds,
            int(st.list_entries))


def _timed(sy, stream, flush, k, warm):
    """per-step device times (ms) with L2 flushed before each step, and the
    per-phase sums of the library's own step events; the steps' kinds go to
    _timed.kinds"""
    import torch

    def run(nsteps, phases):
        sy.set_timing(phases)
        for _ in range(warm):
            with torch.cuda.stream(stream):
                flush()
            sy.step(1)
        sy.sync()
        out, phase, kinds = [], {}, []
        builds = sy.stats().list_builds
        for _ in range(nsteps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush()
                e0.record(stream)
            sy.step(1)
            with torch.cuda.stream(stream):
                e1.record(stream)
            if phases:
                for key, val in sy.phase_times().items():
                    phase[key] = phase.get(key, 0.0) + val / nsteps
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
            kind, builds, _ = _kind(sy, builds)
            kinds.append(kind)
        return out, phase, kinds

    # timed without the per-phase events; the phases over the next steps
    out, _, kinds = run(k, False)
    _, phase, _ = run(min(k, 100), True)
    _timed.kinds = kinds
    return out, phase


def _pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))]


def max_over_ranks(v, dist, device):
    """the largest v over the ranks (v itself without a process group)"""
    if dist is None:
        return float(v)
    import torch

    t = torch.tensor([float(v)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, n, steps, t_max_ms):
    """atom-steps/s of the whole job: every rank steps its own n atoms, and the
    slowest rank's time bounds the job"""
    return world * n * steps / (t_max_ms * 1e-3)


def force_error(f, ref):
    """Eq. 20 as printed, sqrt(mean_i (|F_i - F_i^ref| / |F_i^ref|)^2), and the
    norm ratio sqrt(sum |F_i - F_i^ref|^2 / sum |F_i^ref|^2)"""
    import numpy as np

    d = np.linalg.norm(f - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    return float(np.sqrt(np.mean((d / r) ** 2))), float(np.sqrt((d * d).sum() / (r * r).sum()))


ACCURACY_GRID = [(3.0, 4.5), (3.0, 5.0), (3.0, 5.5), (3.0, 6.0), (3.0, 7.0), (3.0, 8.0),
                 (4.0, 6.0), (4.0, 7.0), (4.0, 8.0), (4.5, 9.0)]
ACCURACY_REF_RC = 12.0


def accuracy_study(dcm, slabgen, stream, np, torch, n=262144):
    """Section 6.1.1 (Fig. 34, 36): force error of DCM against a large static
    cutoff (r_c = 12 sigma, FP64, standing in for the thesis's Ewald sums) on
    the benchmark slab, for the exponential (Eq. 7) and linear (Fig. 12)
    cutoff functions over a grid of (r_c,min, r_c,max); FP64 forces, one
    force evaluation per setting at the same positions"""
    s = slabgen.make_slab(n, seed=1)

    def forces(rc_min, rc_max, fn, prec=dcm.DCM_FP64):
        sy = dcm.System(s.box, n, precision=prec, rc_min=rc_min, rc_max=rc_max, cutoff_fn=fn,
                        stream=stream.cuda_stream)
        sy.set_state(s.x, s.v)
        sy.detect_interface()
        sy.compute_forces()                                  # warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sy.compute_forces()
        e1.record(stream)
        e1.synchronize()
        _, _, f = sy.get_state()
        st = sy.stats()
        sy.close()
        return f, st.pairs / n, e0.elapsed_time(e1)

    ref, ref_pairs, ref_ms = forces(ACCURACY_REF_RC, ACCURACY_REF_RC, dcm.DCM_CUTOFF_EXP)
    rows = []
    for fn, name in ((dcm.DCM_CUTOFF_EXP, "exponential"), (dcm.DCM_CUTOFF_LINEAR, "linear")):
        for rc_min, rc_max in ACCURACY_GRID:
            f, pairs, ms = forces(rc_min, rc_max, fn)
            e20, enorm = force_error(f, ref)
            rows.append({"cutoff_fn": name, "rc_min": rc_min, "rc_max": rc_max,
                         "eq20_rms_rel": e20, "norm_ratio": enorm,
                         "pairs_per_particle": pairs, "force_ms_fp64": ms})
    static = []
    for rc in (3.0, 4.0, 6.0):
        f, pairs, ms = forces(rc, rc, dcm.DCM_CUTOFF_EXP)
        e20, enorm = force_error(f, ref)
        static.append({"rc": rc, "eq20_rms_rel": e20, "norm_ratio": enorm,
                       "pairs_per_particle": pairs, "force_ms_fp64": ms})
    # the mixed-precision path's own error at the default cutoffs, for scale
    f64, _, _ = forces(3.0, 6.0, dcm.DCM_CUTOFF_EXP)
    fmx, _, _ = forces(3.0, 6.0, dcm.DCM_CUTOFF_EXP, dcm.DCM_MIXED)
    mixed = dict(zip(("eq20_rms_rel", "norm_ratio"), force_error(fmx, f64)))
    default = next(r for r in rows if r["cutoff_fn"] == "exponential" and r["rc_max"] == 6.0
                   and r["rc_min"] == 3.0)
    return {"metric": "RMS relative force error of DCM (Eq. 20) against a static r_c = 12 sigma",
            "value": default["eq20_rms_rel"], "unit": "relative", "higher_is_better": False,
            "dtype": "f64", "steps": None, "ms_per_step": None,
            "config": {"workload": f"LJ liquid/vapor slab N={n}, L x L x 4L periodic, rho_l=0.8, "
                                   f"T*=0.7, synthetic start (jittered FCC liquid), 1-sigma voxels; "
                                   f"reference: static truncated cutoff {ACCURACY_REF_RC} sigma in "
                                   f"FP64 (stand-in for Ewald sums)",
                       "n": n, "reference_pairs_per_particle": ref_pairs,
                       "reference_force_ms_fp64": ref_ms, "dcm": rows, "static": static,
                       "mixed_vs_fp64_at_3_6": mixed,
                       "note": ("value = Eq. 20 for r_c 3/6 with the exponential function; "
                                "norm_ratio = sqrt(sum |dF|^2 / sum |F|^2), which tiny reference "
                                "forces cannot dominate")}}


def wavy_run(dcm, slabgen, np, stream, flush, n, steps, warm, skin, skin_time, skin_floor):
    """the capillary-wave slab (two interfaces with sinusoidal z offsets of
    amplitude 1 sigma), DCM r_c 3/7, timed like the headline: per-step device
    times with L2 flushed before each step"""
    s = slabgen.make_slab(n, seed=3, capillary_amp=1.0)
    sy = dcm.System(s.box, n, precision=dcm.DCM_MIXED, rc_min=3.0, rc_max=7.0, skin=skin,
                    skin_time=skin_time, skin_floor=skin_floor, stream=stream.cuda_stream)
    sy.set_state(s.x, s.v)
    sy.compute_forces()
    ms, ph = _timed(sy, stream, flush, steps, warm)
    st = sy.stats()
    x, _, _ = sy.get_state()
    sy.close()
    if not np.all(np.isfinite(x)):
        raise RuntimeError("non-finite positions")
    return n * steps / (sum(ms) * 1e-3), ms, ph, st


WAVY_N = 2097152


def serving_run(dcm, serving, count, steps_max, skin, skin_time, skin_floor):
    """a Poisson stream of slab requests through the serving loop (HBM-budget
    admission, continuous batching); its summary"""
    rep = serving.serve_trace(count=count, rate=20.0, n_min=2048, n_max=524288, steps_min=100,
                              steps_max=steps_max, budget_gb=120.0, precision=dcm.DCM_MIXED,
                              skin=skin, skin_time=skin_time, skin_floor=skin_floor)
    return rep.summary()


def serving_workload(count, steps_max):
    return (f"Poisson stream of {count} slab requests at 20 req/s, N log-uniform in [2048, "
            f"524288], nsteps uniform in [100, {steps_max}], 120 GB HBM budget, continuous "
            f"batching (up to 16 resident slots, 50-step chunks), mixed precision")


def run_workload(args):
    import numpy as np
    import torch

    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import autotune, dcm, serving, slabgen

    stream = torch.cuda.Stream()
    flush = L2Flush(torch)
    line = {"n_gpus": 1, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-pair/f64-state", "data": "synthetic",
            "unit": UNIT}
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        if args.workload == "wavy":
            def wavy(n, steps, warm):
                return wavy_run(dcm, slabgen, np, stream, flush, n, steps, warm, args.skin,
                                args.skin_time, args.skin_floor)

            n = WAVY_N
            value, ms, ph, st = wavy(n, args.steps, args.warmup)
            sweep = {}
            for nn in [int(q) for q in args.sweep.split(",") if q]:
                sweep[str(nn)] = wavy(nn, args.sweep_steps, 3)[0]
            sweep[str(n)] = value
            line.update({
                "metric": "atom-steps/s of the DCM step, capillary-wave slab", "value": value,
                "steps": args.steps, "ms_per_step": sum(ms) / len(ms),
                "config": {"workload": f"LJ slab N={n}, L x L x 4L periodic, two interfaces "
                                       f"with sinusoidal z offsets (amplitude 1 sigma, random "
                                       f"phases), DCM r_c 3/7, 1-sigma voxels, detection every "
                                       f"2 steps, mixed precision",
                           "n": n, "rc_min": 3.0, "rc_max": 7.0, "skin": args.skin,
                           "skin_time": args.skin_time, "skin_floor": args.skin_floor,
                           "phase_ms_avg": ph,
                           "pairs_per_particle": st.pairs / n,
                           "l2": L2_NOTE},
                "latency_ms": {"p50": _pct(ms, 50), "p99": _pct(ms, 99), "unit": "ms per step"},
                "weak_scaling_in_n": {"unit": UNIT, "steps": args.sweep_steps, "values": sweep}})
        elif args.workload == "accuracy":
            line.update(accuracy_study(dcm, slabgen, stream, np, torch))
        elif args.workload == "ensemble":
            mem = slabgen.make_ensemble(64, 4096, 131072, 0.65, 0.85, seed=0)
            boxes = [m.slab.box for m in mem]
            ns = [m.n for m in mem]
            params = [dcm.default_params(precision=dcm.DCM_MIXED, skin=args.skin,
                                         skin_time=args.skin_time, skin_floor=args.skin_floor)
                      for _ in mem]
            ens = dcm.Ensemble(boxes, ns, params, stream=stream.cuda_stream)
            for k, m in enumerate(mem):
                ens.set_system_state(k, m.slab.x, m.slab.v)
            ens.compute_forces()
            choice = autotune.tune_live(ens)
            ms, ph = _timed(ens, stream, flush, args.steps, args.warmup)
            st = ens.stats()
            kernels = _launches(st, _timed.kinds)
            ens.close()
            ntot = sum(ns)
            value = ntot * args.steps / (sum(ms) * 1e-3)
            line.update({
                "metric": "atom-steps/s of the DCM step, batched ensemble", "value": value,
                "steps": args.steps, "ms_per_step": sum(ms) / len(ms),
                "config": {"workload": "64 independent LJ slabs in one handle, N log-uniform in "
                                       "[4096, 131072], T* uniform in [0.65, 0.85], own boxes, "
                                       "DCM r_c 3/6, mixed precision; one persistent force "
                                       "launch per step, each step one CUDA graph",
                           "systems": len(ns), "n_total": ntot, "n_min": min(ns), "skin": args.skin,
                           "skin_time": args.skin_time, "skin_floor": args.skin_floor,
                           "n_max": max(ns), "phase_ms_avg": ph, "tuning": choice,
                           "l2": L2_NOTE},
                "latency_ms": {"p50": _pct(ms, 50), "p99": _pct(ms, 99), "unit": "ms per step"},
                "gpu_launches": int(kernels)})
        else:
            summ = serving_run(dcm, serving, args.requests, 2000, args.skin, args.skin_time,
                               args.skin_floor)
            line.update({
                "metric": "aggregate atom-steps/s of a served request stream; p50/p99 latency",
                "value": summ["atom_steps_per_s"], "steps": None, "ms_per_step": None,
                "config": {"workload": serving_workload(args.requests, 2000),
                           "requests": args.requests, "skin": args.skin,
                           "skin_time": args.skin_time, "skin_floor": args.skin_floor},
                "latency_s": summ["latency_s"], "serving": summ})
    line["clocks"] = clk.summary()
    print(json.dumps(line), flush=True)
    return 0


def ensemble_compare(dcm, slabgen, autotune, stream, flush, torch, steps, warm, skin, skin_time,
                     skin_floor):
    """The mixed/FP64 comparison on the ensemble workload: 64 independent
    slabs (N log-uniform in [4096, 131072], T* uniform in [0.65, 0.85], own
    boxes), mixed precision batched in one handle (one persistent force
    launch per step, the launch shape tuned on the live ensemble) against
    the plain per-system FP64 path (one handle per system, stepped one after
    the other), the same steps from the same states, L2 flushed before each
    timed step (batched) or system step (per system)"""
    mem = slabgen.make_ensemble(64, 4096, 131072, 0.65, 0.85, seed=0)
    boxes = [m.slab.box for m in mem]
    ns = [m.n for m in mem]
    ntot = sum(ns)
    params = [dcm.default_params(precision=dcm.DCM_MIXED, skin=skin, skin_time=skin_time,
                                 skin_floor=skin_floor) for _ in mem]
    ens = dcm.Ensemble(boxes, ns, params, stream=stream.cuda_stream)
    for k, m in enumerate(mem):
        ens.set_system_state(k, m.slab.x, m.slab.v)
    ens.compute_forces()
    choice = autotune.tune_live(ens, reps=3)
    ms, _ = _timed(ens, stream, flush, steps, warm)
    ens.close()
    mixed = ntot * steps / (sum(ms) * 1e-3)
    # per system, FP64: every system its own handle, warmed, then each system's
    # steps timed with events around them
    t64 = 0.0
    for m in mem:
        sy = dcm.System(m.slab.box, m.n, precision=dcm.DCM_FP64, stream=stream.cuda_stream,
                        skin=skin, skin_time=skin_time, skin_floor=skin_floor)
        sy.set_state(m.slab.x, m.slab.v)
        for _ in range(warm):
            sy.step(1)
        sy.sync()
        with torch.cuda.stream(stream):
            flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sy.step(steps)
        e1.record(stream)
        e1.synchronize()
        t64 += e0.elapsed_time(e1)
        sy.close()
    fp64 = ntot * steps / (t64 * 1e-3)
    return {"systems": len(ns), "n_total": ntot, "n_min": min(ns), "n_max": max(ns),
            "steps": steps, "warmup": warm,
            "mixed_batched": {"value": mixed, "unit": UNIT, "ms_per_step": sum(ms) / len(ms),
                              "tuning": {k: v for k, v in choice.items()
                                         if k in ("list_lanes", "list_lanes_class",
                                                  "force_ms")}},
            "fp64_per_system": {"value": fp64, "unit": UNIT, "ms_per_step_all_systems": t64 / steps},
            "speedup": mixed / fp64,
            "note": "the 64-slab ensemble workload, both arms from the same states"}


# ---- the GPU arm ---------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "slab":
        return run_workload(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist_mod.init_process_group("nccl")
        dist = dist_mod
    # build once per node, then import
    if local == 0:
        import __graft_entry__

        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    from paper_1502_03234_gb300 import dcm, slabgen

    n = args.n
    prec = dcm.DCM_MIXED if args.precision == "mixed" else dcm.DCM_FP64
    slab = slabgen.make_slab(n, seed=1 + rank)
    stream = torch.cuda.Stream()
    flush = L2Flush(torch)

    def make_system(precision):
        sy = dcm.System(slab.box, n, precision=precision, stream=stream.cuda_stream,
                        skin=args.skin, list_margin=args.list_margin, skin_time=args.skin_time,
                        skin_floor=args.skin_floor, cell_min=args.cell_min,
                        min_component_voxels=args.min_component)
        if args.list_lanes and precision == dcm.DCM_MIXED:    # (the list force's lanes)
            t = dcm.dcm_get_tuning(sy.h)
            sy.set_tuning(list(t.lanes), t.block, t.walk, args.list_lanes, args.list_lanes_class)
        if args.step_graph == "flat":
            sy.set_step_graph(dcm.DCM_GRAPH_FLAT)
        sy.set_state(slab.x, slab.v)
        sy.compute_forces()
        return sy

    def timed_steps(sy, k, warm, phases, on_ready=None):
        """per-step device times (ms), L2 flushed before each step; with
        phases, the step graph also records the library's per-phase events
        (force time per step for the roofline), which adds event nodes to
        every step, so the headline pass runs without them.  on_ready runs
        after the warm-up, before the timed steps (outside the timing)"""
        sy.set_timing(phases)
        for _ in range(warm):
            with torch.cuda.stream(stream):
                flush()
            sy.step(1)
        sy.sync()
        if on_ready is not None:
            on_ready()
            sy.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        force_ms, phase_sum, rebuilt, kinds, ents = [], {}, [], [], []
        b_prev = sy.stats().list_builds
        for q in range(k):
            with torch.cuda.stream(stream):
                flush()
                ev[q][0].record(stream)
            sy.step(1)
            with torch.cuda.stream(stream):
                ev[q][1].record(stream)
            if phases:
                ph = sy.phase_times()                   # waits for this step
                force_ms.append(ph["force"])
                for key, val in ph.items():
                    phase_sum[key] = phase_sum.get(key, 0.0) + val
            kind, b_now, e_now = _kind(sy, b_prev)      # (outside the timed events)
            kinds.append(kind)
            rebuilt.append(b_now != b_prev)
            ents.append(e_now)
            b_prev = b_now
        sy.sync()
        timed_steps.rebuilt = rebuilt
        timed_steps.kinds = kinds
        timed_steps.entries = ents
        return [a.elapsed_time(b) for a, b in ev], force_ms, phase_sum

    def total_energy(sy_):
        pe, ke, _ = sy_.energy_virial()
        return pe + ke

    energy = {}
    # the launch shape: tuned on a scratch copy of the system (same start,
    # a few steps in), then used by the timed system
    tuning = None
    if not args.list_lanes and not args.no_tune:
        from paper_1502_03234_gb300 import autotune

        scratch = make_system(prec)
        scratch.step(4)
        choice = autotune.tune_live(scratch, reps=5)
        scratch.close()
        tuning = {k: v for k, v in choice.items() if k in ("walk", "lanes", "block", "list_lanes",
                                                              "list_lanes_class", "force_ms")}
        tuning["how"] = "autotune.tune_live on a scratch copy of the slab, 4 steps in"
        if prec == dcm.DCM_MIXED:
            args.list_lanes = int(choice.get("list_lanes", 8))
            args.list_lanes_class = choice.get("list_lanes_class")
    sy = make_system(prec)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        step_ms, _, _ = timed_steps(sy, args.steps, args.warmup, False,
                                    on_ready=lambda: energy.update(e0=total_energy(sy)))
    head_entries = timed_steps.entries
    torch.cuda.synchronize()
    energy["e1"] = total_energy(sy)
    if dist is not None:
        dist.barrier()
    total_ms = sum(step_ms)
    st = sy.stats()
    kernels = _launches(st, timed_steps.kinds)
    # the same steps again on a second system from the same start (the
    # trajectory is deterministic), this time with the per-phase events:
    # force time per step for the roofline and the phase breakdown; not part
    # of the headline number
    phase_steps = args.steps
    sy_ph = make_system(prec)
    _, force_ms, phase_sum = timed_steps(sy_ph, phase_steps, args.warmup, True)
    st = sy_ph.stats()
    pairs = st.pairs
    sy_ph.close()
    x_end, _, _ = sy.get_state()
    if not np.all(np.isfinite(x_end)):
        raise RuntimeError("non-finite positions after the timed run")
    sy.sync()

    # max over ranks, whole-job throughput
    t_max = max_over_ranks(total_ms, dist, "cuda")
    value = whole_job_rate(world, n, args.steps, t_max)

    # roofline of the dominant kernel
    clocks = clk.summary()
    rebuilt = timed_steps.rebuilt
    f_avg_ms = sum(force_ms) / len(force_ms)
    sm_mhz = clocks.get("sm_mhz") or 1477.0
    fp32_peak = 152 * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    list_steps = [t for t, r in zip(force_ms, rebuilt) if not r]
    if prec == dcm.DCM_MIXED and args.skin > 0 and list_steps:
        # Verlet-list steps: the force phase is k_force_list_warp (plus the
        # empty launch of the rebuild kernel).  It streams each particle's
        # list from HBM (arithmetic intensity ~3 flop/B, under the HBM roof)
        l_ms = sum(list_steps) / len(list_steps)
        # the lists' entries averaged over the timed list steps (they change
        # with every build)
        list_ents = [e for e, r in zip(timed_steps.entries, rebuilt) if not r]
        entries = sum(list_ents) / len(list_ents)
        lkernel = "k_force_list_cls" if args.list_lanes_class else "k_force_list_warp"
        alg_bytes = LIST_BYTES_PER_ENTRY * entries + LIST_BYTES_PER_PARTICLE * n
        achieved_gbs = alg_bytes / (l_ms * 1e-3) / 1e9
        # algorithmic work: 8 flops per distance check (every list entry)
        # and 16 more per in-cutoff pair (rcp, (s/r)^6, the scalar, 3 FMA)
        alg_flops = FLOPS_PER_CHECK * entries + FLOPS_PER_FORCE * pairs
        achieved = alg_flops / (l_ms * 1e-3) / 1e12
        cap = LIST_TRAFFIC.get(lkernel) or {}
        traffic = None
        if (cap.get("bytes") and n == N_DEFAULT and
                (args.skin, args.skin_time, args.skin_floor, args.list_margin) == LIST_TRAFFIC_CONFIG):
            cap_alg = LIST_BYTES_PER_ENTRY * cap["entries"] + LIST_BYTES_PER_PARTICLE * n
            traffic = cap["bytes"] * alg_bytes / cap_alg
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak,
                    "traffic": traffic,
                    "traffic_note": ("ncu DRAM bytes of one captured launch, scaled from that "
                                     "launch's list entries to this run's mean by the algorithmic "
                                     "bytes"),
                    "kernel": f"{lkernel} (mixed, Verlet lists)",
                    "peak_note": ("FP32 FMA peak derived from 152 SMs x 128 lanes x 2 flops x the "
                                  "median SM clock sampled during the timed region"),
                    "algorithmic_flops_per_launch": alg_flops,
                    "flops_convention": "8 per distance check (list entry) + 16 per in-cutoff pair",
                    "list_entries": entries,
                    "launch_ms_avg": l_ms, "launches": len(list_steps),
                    "hbm_view": {"achieved": achieved_gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                 "frac": achieved_gbs / HBM_PEAK_GBS,
                                 "algorithmic_bytes_per_launch": alg_bytes,
                                 "bytes_convention": "4 B per list entry + 88 B per particle",
                                 "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
                    "phase_note": ("with the step graph's single conditional node the force phase "
                                   "of a rebuild step also holds the list build (sort, gather, "
                                   "class lists, capacity scan); the binning phase is empty"),
                    "rebuild_steps": sum(rebuilt),
                    "rebuild_force_ms_avg": (sum(t for t, r in zip(force_ms, rebuilt) if r) /
                                             max(1, sum(rebuilt))),
                    "force_ms_avg_all_steps": f_avg_ms, "pairs_per_launch": pairs}
    else:
        achieved = FLOPS_PER_PAIR * pairs / (f_avg_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak,
                    "traffic": (FORCE_TRAFFIC.get(args.precision)
                                if n == N_DEFAULT and args.skin == 0 else None),
                    "kernel": force_kernel_name(dcm, sy, prec, args.skin),
                    "peak_note": "FP32 FMA peak derived from 152 SMs x 128 lanes x 2 flops x the "
                                 "median SM clock sampled during the timed region",
                    "pairs_per_launch": pairs, "force_ms_avg": f_avg_ms}
    # the FP32 FMA throughput measured on this GPU in this run (an FMA chain
    # on every SM): the derived peak above is the unit-count figure the
    # roofline is quoted against; this is the reachable one beside it
    try:
        ffma, ffma_ms = dcm.dcm_fp32_peak(100000)
        roofline["ffma_measured"] = {
            "value": ffma, "unit": "TFLOP/s", "frac": roofline["achieved"] / ffma,
            "ms": ffma_ms, "note": "dcm_fp32_peak: 8 dependent FMA chains per thread, 64 warps "
                                  "per SM on every SM, timed by CUDA events after the timed steps"}
    except dcm.DcmError as e:
        roofline["ffma_measured"] = {"error": str(e)}

    # detection with Eq. 13 (Section 4.1, DCM_SEG_MUMFORD_SHAH) in place of
    # the K-means labels: per-phase times over a short run of the same slab
    seg_info = None
    if rank == 0 and prec == dcm.DCM_MIXED and args.seg_steps > 0:
        def detect_ms(seg, **ms):
            syx = dcm.System(slab.box, n, precision=prec, stream=stream.cuda_stream,
                             skin=args.skin, list_margin=args.list_margin,
                             skin_time=args.skin_time, skin_floor=args.skin_floor,
                             cell_min=args.cell_min, segmentation=seg, **ms)
            if args.list_lanes:
                t = dcm.dcm_get_tuning(syx.h)
                syx.set_tuning(list(t.lanes), t.block, t.walk, args.list_lanes,
                               args.list_lanes_class)
            syx.set_state(slab.x, slab.v)
            syx.compute_forces()
            ms_, _, ph_ = timed_steps(syx, args.seg_steps, 2, True)
            st_ = syx.stats()
            syx.close()
            det_steps = max(1, args.seg_steps // 2)       # detection every second step
            return {"ms_per_step": sum(ms_) / len(ms_),
                    "detect_ms_per_detection": ph_.get("detect", 0.0) / det_steps,
                    "kernels_detect_step": int(st_.kernels_detect)}
        km = detect_ms(dcm.DCM_SEG_KMEANS)
        mu = detect_ms(dcm.DCM_SEG_MUMFORD_SHAH)                 # the defaults: one round
        mu4 = detect_ms(dcm.DCM_SEG_MUMFORD_SHAH, ms_outer=4)    # densities alternated
        seg_info = {"kmeans": km, "eq13": mu, "eq13_alternating_4_rounds": mu4,
                    "steps": args.seg_steps,
                    "eq13_params": {"nu": 0.005, "iters": 50, "rounds": 1},
                    "segmentation_share_of_detection":
                        1.0 - km["detect_ms_per_detection"] / mu["detect_ms_per_detection"]
                        if mu["detect_ms_per_detection"] > 0 else None,
                    "note": "per-phase CUDA events over a short run from the same start; the "
                            "share is that of the Eq. 13 step in a detection (thesis: 75-80 %)"}

    ens_info = None
    if rank == 0 and prec == dcm.DCM_MIXED and args.ens_steps > 0:
        from paper_1502_03234_gb300 import autotune

        ens_info = ensemble_compare(dcm, slabgen, autotune, stream, flush, torch, args.ens_steps,
                                    3, args.skin, args.skin_time, args.skin_floor)

    # the other workloads of the method, short: the 2.1M-atom capillary-wave
    # slab (timed like the headline) and a served request stream
    wavy_info = None
    if rank == 0 and prec == dcm.DCM_MIXED and args.wavy_steps > 0:
        wv, wms, wph, wst = wavy_run(dcm, slabgen, np, stream, flush, WAVY_N, args.wavy_steps, 3,
                                     args.skin, args.skin_time, args.skin_floor)
        wavy_info = {"value": wv, "unit": UNIT, "n": WAVY_N, "steps": args.wavy_steps,
                     "warmup": 3, "ms_per_step": sum(wms) / len(wms),
                     "latency_ms": {"p50": _pct(wms, 50), "p99": _pct(wms, 99)},
                     "pairs_per_particle": wst.pairs / WAVY_N, "phase_ms_avg": wph,
                     "workload": f"LJ slab N={WAVY_N}, L x L x 4L periodic, two interfaces with "
                                 f"sinusoidal z offsets (amplitude 1 sigma, random phases), DCM "
                                 f"r_c 3/7, detection every 2 steps, mixed precision; L2 flushed "
                                 f"before every timed step"}
    serve_info = None
    if rank == 0 and prec == dcm.DCM_MIXED and args.serve_requests > 0:
        from paper_1502_03234_gb300 import serving

        summ = serving_run(dcm, serving, args.serve_requests, 500, args.skin, args.skin_time,
                           args.skin_floor)
        serve_info = dict(summ)
        serve_info["workload"] = serving_workload(args.serve_requests, 500)

    # the plain FP64 GPU path on the same system (the comparison the metric
    # names), timed exactly like the headline: the same steps and warm-up,
    # no per-phase events, L2 flushed before every step
    fp64_info = None
    accuracy = None
    if not args.no_fp64_compare and prec == dcm.DCM_MIXED and rank == 0:
        sy64 = make_system(dcm.DCM_FP64)
        e64 = {}
        s64, _, _ = timed_steps(sy64, args.steps, args.warmup, False,
                                on_ready=lambda: e64.update(e0=total_energy(sy64)))
        e64["e1"] = total_energy(sy64)
        t64 = sum(s64)
        fp64_info = {"value": n * args.steps / (t64 * 1e-3), "unit": UNIT, "steps": args.steps,
                     "warmup": args.warmup, "ms_per_step": t64 / args.steps,
                     "energy_drift": abs(e64["e1"] - e64["e0"]) / abs(e64["e0"]),
                     "speedup_of_mixed": t64 / total_ms,
                     "kernel": "k_force (FP64 lanes walk over the Verlet lists)"}
        # the mixed path's forces against FP64 forces at its final positions
        # and cutoffs (per particle, the parity bar 1e-6 + 1e-5 |F|)
        x_end, v_end, f_mix = sy.get_state()
        _, rc_end, _ = sy.cutoffs()
        sy64.set_state(x_end, v_end)
        sy64.set_cutoffs(rc_end)
        sy64.compute_forces()
        _, _, f_ref = sy64.get_state()
        err = np.linalg.norm(f_mix - f_ref, axis=1)
        fmag = np.linalg.norm(f_ref, axis=1)
        accuracy = {"max_abs": float(err.max()), "p99_abs": float(np.percentile(err, 99)),
                    "max_err_over_bar": float(np.max(err / (1e-6 + 1e-5 * fmag))),
                    "bar": "|F_mixed - F_fp64| <= 1e-6 + 1e-5 |F_fp64| per particle",
                    "at": f"the final state of the timed run ({args.steps} steps)",
                    "refined_last_step": int(sy.stats().refined)}
        sy64.close()

    # end to end through the public API with host buffers: the host holds
    # the state and hands it back each step (dcm_update_state keeps the
    # run's cutoffs, step counter and lists; the forces are recomputed from
    # the positions handed in), then reads the new state back
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        sy.set_timing(False)
        xs, vs, _ = sy.get_state()                  # the running state (host copy)
        xh = torch.from_numpy(np.ascontiguousarray(xs)).pin_memory()
        vh = torch.from_numpy(np.ascontiguousarray(vs)).pin_memory()
        xo = torch.empty_like(xh).pin_memory()
        vo = torch.empty_like(vh).pin_memory()
        lib = dcm.lib()
        px, pv = xh.data_ptr(), vh.data_ptr()
        pxo, pvo = xo.data_ptr(), vo.data_ptr()
        import ctypes as C

        builds0 = sy.stats().list_builds
        sy.sync()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            dcm.check(lib.dcm_update_state(sy.h, C.c_void_p(px), C.c_void_p(pv), dcm.DCM_HOST))
            dcm.check(lib.dcm_step(sy.h, 1))
            dcm.check(lib.dcm_get_state(sy.h, C.c_void_p(pxo), C.c_void_p(pvo), None, dcm.DCM_HOST))
            px, pxo = pxo, px
            pv, pvo = pvo, pv
        sy.sync()
        dt = time.perf_counter() - t0
        e2e = {"value": n * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": 2 * 24 * n, "d2h_bytes_per_step": 2 * 24 * n,
               "steps": args.e2e_steps,
               "list_builds": int(sy.stats().list_builds - builds0),
               "note": "per step: dcm_update_state (x, v from pinned host) + dcm_step(1) + "
                       "dcm_get_state (x, v to pinned host), from the timed run's final state; "
                       "the update keeps the cutoffs, the step counter and the lists (the reuse "
                       "test rebuilds them when due) and recomputes the forces from the "
                       "positions handed in"}
    sy.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, csteps, cdt = oracle_rate(16384, target_s=12.0,
                                               min_component=args.min_component)
        rate1, _, csteps1, cdt1 = oracle_rate(16384, target_s=5.0, threads=1,
                                              min_component=args.min_component)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"N=16384 slab of the same shape, {csteps} oracle steps "
                         f"({cdt:.1f} s) after a 2-step calibration",
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": f"the same slab, {csteps1} oracle steps ({cdt1:.1f} s)"}}

    if rank == 0:
        sms = sorted(step_ms)
        p50 = sms[len(sms) // 2]
        p99 = sms[min(len(sms) - 1, int(math.ceil(0.99 * len(sms))) - 1)]
        cfg = workload_config(n, args.precision)
        cfg["skin"] = args.skin
        cfg["list_margin"] = args.list_margin
        cfg["cell_min"] = args.cell_min
        cfg["skin_time"] = args.skin_time
        cfg["skin_floor"] = args.skin_floor
        cfg["min_component_voxels"] = args.min_component
        if args.steps <= 64 and args.skin > 0:
            # list entries after each timed step (to match profiler captures
            # of single launches)
            cfg["list_entries_steps"] = head_entries
        cfg["phase_ms_avg"] = {k: v / phase_steps for k, v in phase_sum.items()}
        cfg["phase_note"] = ("per-phase CUDA events inside the step graph, on a second run of the "
                             "same steps from the same start (the timed run records none)")
        cfg["tuning"] = tuning
        cfg["list_lanes"] = args.list_lanes
        cfg["list_lanes_class"] = args.list_lanes_class
        cfg["fp64_gpu_path"] = fp64_info
        cfg["segmentation_eq13"] = seg_info
        cfg["ensemble_vs_fp64"] = ens_info
        cfg["wavy_slab"] = wavy_info
        cfg["serving"] = serve_info
        cfg["energy_drift"] = {"rel": abs(energy["e1"] - energy["e0"]) / abs(energy["e0"]),
                               "steps": args.steps,
                               "note": "|E(K) - E(0)| / |E(0)| over the timed steps (NVE; the "
                                       "potential is truncated and unshifted, and r_c moves)"}
        cfg["mixed_vs_fp64_forces"] = accuracy
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32-pair/f64-state" if prec == dcm.DCM_MIXED else "f64",
                "data": "synthetic", "config": cfg,
                "latency_ms": {"p50": p50, "p99": p99, "unit": "ms per step"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(kernels), "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
