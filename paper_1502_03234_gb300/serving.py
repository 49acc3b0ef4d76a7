"""Continuous-batching server for DCM slab simulations.

Requests (a slab of N particles, a number of steps) arrive over time.  A
request is admitted as soon as a slot is free and its device footprint
(``dcm_estimate_bytes``) fits in the remaining HBM budget; its state then
stays resident on the device until it finishes.  Every admitted request owns
a handle on its own CUDA stream and advances in chunks of steps; chunks of
different requests run concurrently on the GPU, and requests that arrive
while others are running join between chunks -- the batch changes
continuously instead of draining before new work is taken.

Under budget pressure a running request can be evicted (``evict_after``):
when the oldest waiting request has waited that long and does not fit, the
running requests with the most work left stop taking chunks, and once their
chunks have drained each one's state (positions, velocities, step counter)
is read back, its handle is released, and it waits again; re-admitted, it
continues from that state.  Chunks end on even steps, the detection
boundaries, so a request resumed without Verlet lists reproduces the
uninterrupted run bit for bit (with lists, its lists are rebuilt at the
resume and it agrees within the force tolerance).

Latency is measured from arrival to the read-back of the final state; the
report gives p50/p99 latency, queueing delay and aggregate atom-steps/s.

The scheduler talks to a small backend interface, so its admission,
slotting, cancellation and failure handling are testable on the CPU with a
simulated backend; ``DcmBackend`` is the GPU one.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

QUEUED, RUNNING, DONE, FAILED, REJECTED, CANCELLED = (
    "queued", "running", "done", "failed", "rejected", "cancelled")


@dataclass
class Job:
    rid: int
    n: int
    nsteps: int
    box: tuple
    x: np.ndarray | None = None
    v: np.ndarray | None = None
    params: object = None
    arrival: float = 0.0                 # seconds from the start of the run
    status: str = QUEUED
    admitted_at: float | None = None
    finished_at: float | None = None
    steps_done: int = 0
    result: tuple | None = None          # (x, v, f) at the end
    error: str | None = None
    bytes: int = 0
    cancel: bool = False
    resume_step: int = 0                 # step counter of the state in x, v (after an eviction)
    evictions: int = 0
    evicting: bool = False
    since_admit: int = 0                 # chunks completed since the last admission

    @property
    def latency(self) -> float | None:
        if self.finished_at is None:
            return None
        return self.finished_at - self.arrival

    @property
    def queue_delay(self) -> float | None:
        if self.admitted_at is None:
            return None
        return self.admitted_at - self.arrival


class Backend:
    """What the scheduler needs from a device."""

    def estimate(self, job: Job) -> int:
        raise NotImplementedError

    def start(self, job: Job):
        raise NotImplementedError

    def advance(self, slot, nsteps: int) -> None:
        raise NotImplementedError

    def inflight(self, slot) -> int:
        """Number of chunks enqueued on the slot that have not completed."""
        raise NotImplementedError

    def finish(self, slot) -> tuple:
        raise NotImplementedError

    def release(self, slot) -> None:
        raise NotImplementedError

    def checkpoint(self, slot) -> tuple:
        """(x, v) of a slot with no chunk in flight, to resume it later
        through start() with job.x, job.v and job.resume_step."""
        raise NotImplementedError


@dataclass
class Report:
    jobs: list
    makespan: float
    atom_steps: float
    budget_bytes: int
    peak_bytes: int
    max_active: int
    offered_atom_steps_per_s: float = 0.0
    evictions: int = 0

    @property
    def throughput(self) -> float:
        return self.atom_steps / self.makespan if self.makespan > 0 else 0.0

    def latency_percentiles(self, qs=(50, 99)) -> dict:
        lat = sorted(j.latency for j in self.jobs if j.status == DONE)
        if not lat:
            return {f"p{q}": None for q in qs}
        return {f"p{q}": float(np.percentile(lat, q)) for q in qs}

    def summary(self) -> dict:
        done = [j for j in self.jobs if j.status == DONE]
        qd = [j.queue_delay for j in done]
        d = {"requests": len(self.jobs), "done": len(done),
             "failed": sum(j.status == FAILED for j in self.jobs),
             "rejected": sum(j.status == REJECTED for j in self.jobs),
             "cancelled": sum(j.status == CANCELLED for j in self.jobs),
             "makespan_s": self.makespan, "atom_steps_per_s": self.throughput,
             "latency_s": self.latency_percentiles(),
             "queue_delay_s": {"p50": float(np.percentile(qd, 50)) if qd else None,
                               "p99": float(np.percentile(qd, 99)) if qd else None},
             "budget_bytes": self.budget_bytes, "peak_bytes": self.peak_bytes,
             "max_active": self.max_active, "evictions": self.evictions,
             "offered_atom_steps_per_s": self.offered_atom_steps_per_s}
        if self.offered_atom_steps_per_s:
            d["load"] = ("overloaded" if self.offered_atom_steps_per_s > self.throughput * 1.05
                         else "underloaded")
        return d


class Server:
    """Admission by HBM budget, slots, chunked stepping, continuous joining."""

    def __init__(self, backend: Backend, budget_bytes: int, max_slots: int = 16,
                 chunk_steps: int = 50, ahead: int = 2, clock=time.perf_counter,
                 sleep=time.sleep, evict_after: float | None = None, max_evictions: int = 1):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        # chunks end on detection boundaries (detect_every = 2): a resumed
        # request re-detects at the step the uninterrupted run does
        self.chunk = max(2, int(chunk_steps) // 2 * 2)
        self.ahead = int(ahead)
        self.clock = clock
        self.sleep = sleep
        self.evict_after = evict_after        # None: never evict
        self.max_evictions = int(max_evictions)

    def run(self, jobs: list, realtime: bool = True) -> Report:
        """Serve jobs (each with its arrival time); returns when all ended."""
        t0 = self.clock()
        now = lambda: self.clock() - t0  # noqa: E731
        future = deque(sorted(jobs, key=lambda j: j.arrival))
        pending: deque = deque()
        active = {}                     # rid -> (job, slot)
        used = peak = max_active = evictions = 0
        waiting_since = {}              # rid -> time it (re)entered the queue
        while future or pending or active:
            t = now()
            while future and (not realtime or future[0].arrival <= t):
                j = future.popleft()
                if not realtime:
                    j.arrival = t
                j.bytes = self.backend.estimate(j)
                if j.bytes < 0 or j.bytes > self.budget:
                    j.status = REJECTED
                    j.error = "does not fit the HBM budget" if j.bytes >= 0 else "invalid request"
                    j.finished_at = t
                    continue
                pending.append(j)
                waiting_since[j.rid] = t
            progressed = False
            # admission in arrival order; a request that does not fit yet
            # lets later, smaller ones in (first fit) without losing its place
            for j in list(pending):
                if j.cancel:
                    pending.remove(j)
                    j.status = CANCELLED
                    j.finished_at = now()
                    continue
                if len(active) >= self.max_slots:
                    break
                if used + j.bytes > self.budget:
                    continue
                pending.remove(j)
                try:
                    slot = self.backend.start(j)
                except Exception as e:   # allocation or upload failed
                    j.status = FAILED
                    j.error = f"start: {e}"
                    j.finished_at = now()
                    continue
                j.status = RUNNING
                if j.admitted_at is None:
                    j.admitted_at = now()
                j.since_admit = 0
                used += j.bytes
                peak = max(peak, used)
                active[j.rid] = (j, slot)
                max_active = max(max_active, len(active))
                progressed = True
            # eviction under budget pressure: the oldest waiting request has
            # waited evict_after and does not fit; the running requests with
            # the most work left (each evicted at most max_evictions times,
            # and only after a chunk since its admission) stop taking chunks
            if self.evict_after is not None and pending and len(active) > 0:
                h = pending[0]
                deficit = used + h.bytes - self.budget
                if deficit > 0 and now() - waiting_since.get(h.rid, 0.0) >= self.evict_after:
                    already = sum(j.bytes for j, _ in active.values() if j.evicting)
                    cand = sorted((j for j, _ in active.values()
                                   if not j.evicting and j.evictions < self.max_evictions
                                   and j.since_admit > 0 and j.steps_done < j.nsteps),
                                  key=lambda j: (j.nsteps - j.steps_done) * j.n, reverse=True)
                    for j in cand:
                        if already >= deficit:
                            break
                        j.evicting = True
                        already += j.bytes
            # advance: keep up to `ahead` chunks queued per slot
            for rid in list(active):
                j, slot = active[rid]
                if j.cancel:
                    self._end(j, slot, CANCELLED, None, now())
                    used -= j.bytes
                    del active[rid]
                    progressed = True
                    continue
                inflight = self.backend.inflight(slot)
                if j.evicting and inflight == 0:
                    try:
                        j.x, j.v = self.backend.checkpoint(slot)
                        j.resume_step = j.steps_done
                    except Exception as e:
                        self._end(j, slot, FAILED, None, now(), err=f"checkpoint: {e}")
                        used -= j.bytes
                        del active[rid]
                        progressed = True
                        continue
                    try:
                        self.backend.release(slot)
                    except Exception:
                        pass
                    used -= j.bytes
                    del active[rid]
                    j.status = QUEUED
                    j.evicting = False
                    j.evictions += 1
                    evictions += 1
                    pending.append(j)
                    waiting_since[j.rid] = now()
                    progressed = True
                    continue
                if j.evicting:
                    continue
                if j.steps_done >= j.nsteps and inflight == 0:
                    try:
                        res = self.backend.finish(slot)
                        self._end(j, slot, DONE, res, now())
                    except Exception as e:
                        self._end(j, slot, FAILED, None, now(), err=str(e))
                    used -= j.bytes
                    del active[rid]
                    progressed = True
                    continue
                j.since_admit = max(j.since_admit, (j.steps_done - j.resume_step) // self.chunk
                                    - inflight)
                while inflight < self.ahead and j.steps_done < j.nsteps:
                    k = min(self.chunk, j.nsteps - j.steps_done)
                    self.backend.advance(slot, k)
                    j.steps_done += k
                    inflight += 1
                    progressed = True
            if not progressed:
                self.sleep(0.0002)
        makespan = now()
        atom_steps = float(sum(j.n * j.nsteps for j in jobs if j.status == DONE))
        span = max((j.arrival for j in jobs), default=0.0)
        offered = (float(sum(j.n * j.nsteps for j in jobs)) / span) if span > 0 else 0.0
        return Report(jobs=list(jobs), makespan=makespan, atom_steps=atom_steps,
                      budget_bytes=self.budget, peak_bytes=peak, max_active=max_active,
                      offered_atom_steps_per_s=offered, evictions=evictions)

    def _end(self, job, slot, status, result, t, err=None):
        job.status = status
        job.result = result
        job.error = err
        job.finished_at = t
        try:
            self.backend.release(slot)
        except Exception:
            pass


# ---- the GPU backend ------------------------------------------------------------------
class DcmBackend(Backend):
    """One libdcm handle per admitted request, each on its own CUDA stream;
    the state stays on the device between chunks."""

    def __init__(self, precision: int | None = None, tune: dict | None = None,
                 skin: float | None = None, skin_time: float = 0.0, skin_floor: float = 0.0):
        import torch

        from . import dcm

        self.torch = torch
        self.dcm = dcm
        self.precision = dcm.DCM_MIXED if precision is None else precision
        self.tune = tune or {}
        self.skin = skin
        self.skin_time, self.skin_floor = skin_time, skin_floor

    def _params(self, job: Job):
        p = job.params if job.params is not None else self.dcm.default_params()
        p.precision = self.precision
        if self.skin is not None:
            p.skin = self.skin
            p.skin_time = self.skin_time
            p.skin_floor = self.skin_floor
        return p

    def estimate(self, job: Job) -> int:
        return self.dcm.dcm_estimate_bytes(job.box, job.n, self._params(job))

    def start(self, job: Job):
        stream = self.torch.cuda.Stream()
        sy = self.dcm.System(job.box, job.n, self._params(job), stream=stream.cuda_stream)
        if self.tune:
            sy.set_tuning(self.tune.get("lanes", [2, 1, 2, 2]), self.tune.get("block", 128),
                          self.tune.get("walk", self.dcm.DCM_WALK_WARP))
        sy.set_state(job.x, job.v)
        if job.resume_step:
            sy.set_step(job.resume_step)     # the detection cadence continues
        return {"sys": sy, "stream": stream, "events": deque()}

    def advance(self, slot, nsteps: int) -> None:
        slot["sys"].step(nsteps)
        ev = self.torch.cuda.Event()
        ev.record(slot["stream"])
        slot["events"].append(ev)

    def inflight(self, slot) -> int:
        ev = slot["events"]
        while ev and ev[0].query():
            ev.popleft()
        return len(ev)

    def finish(self, slot) -> tuple:
        sy = slot["sys"]
        sy.sync()                      # raises on a device-side check
        return sy.get_state()

    def release(self, slot) -> None:
        slot["sys"].close()

    def checkpoint(self, slot) -> tuple:
        sy = slot["sys"]
        sy.sync()
        x, v, _ = sy.get_state()
        return x, v


def trace_jobs(requests, min_edge: float | None = 17.0) -> list:
    """Jobs for a slabgen request trace (slabs generated up front)."""
    from . import slabgen

    jobs = []
    for r in requests:
        s = slabgen.make_slab(r.n, r.temperature, seed=r.seed, min_edge=min_edge)
        jobs.append(Job(rid=r.rid, n=r.n, nsteps=r.nsteps, box=s.box, x=s.x, v=s.v,
                        arrival=r.arrival_s))
    return jobs


def serve_trace(count=400, rate=20.0, n_min=2048, n_max=524288, steps_min=100, steps_max=2000,
                budget_gb=120.0, max_slots=16, chunk=50, seed=0, precision=None,
                realtime=True, skin=None, skin_time=0.0, skin_floor=0.0) -> Report:
    from . import slabgen

    reqs = slabgen.make_trace(count, rate, n_min, n_max, steps_min, steps_max, seed=seed)
    jobs = trace_jobs(reqs)
    srv = Server(DcmBackend(precision, skin=skin, skin_time=skin_time, skin_floor=skin_floor),
                 int(budget_gb * 2**30), max_slots, chunk)
    return srv.run(jobs, realtime=realtime)


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=400)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--n-max", type=int, default=524288)
    ap.add_argument("--steps-max", type=int, default=2000)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--chunk", type=int, default=50)
    a = ap.parse_args()
    rep = serve_trace(a.count, a.rate, n_max=a.n_max, steps_max=a.steps_max,
                      budget_gb=a.budget_gb, max_slots=a.slots, chunk=a.chunk)
    print(json.dumps(rep.summary()))
