"""Serving scheduler logic on the CPU with a simulated device: admission by
HBM budget, slots, continuous joining, first-fit bypass, cancellation and
failures injected on the host (no GPU involved)."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import serving as sv


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeBackend(sv.Backend):
    """Each slot runs its chunks back to back at `rate` atom-steps/s."""

    def __init__(self, clock, rate=1e8, bytes_per_atom=500, fail_start=(), fail_finish=()):
        self.clock, self.rate, self.bpa = clock, rate, bytes_per_atom
        self.fail_start, self.fail_finish = set(fail_start), set(fail_finish)
        self.live = 0
        self.max_live = 0
        self.released = []

    def estimate(self, job):
        return job.n * self.bpa

    def start(self, job):
        if job.rid in self.fail_start:
            raise MemoryError("injected allocation failure")
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return {"job": job, "done_at": [], "free": self.clock()}

    def advance(self, slot, nsteps):
        t0 = max(self.clock(), slot["free"])
        slot["free"] = t0 + nsteps * slot["job"].n / self.rate
        slot["done_at"].append(slot["free"])

    def inflight(self, slot):
        return sum(t > self.clock() for t in slot["done_at"])

    def finish(self, slot):
        if slot["job"].rid in self.fail_finish:
            raise RuntimeError("device check failed (non-finite position)")
        return ("x", "v", "f")

    def release(self, slot):
        self.live -= 1
        self.released.append(slot["job"].rid)


def _jobs(spec):
    return [sv.Job(rid=i, n=n, nsteps=s, box=(1, 1, 1), arrival=a) for i, (n, s, a) in enumerate(spec)]


def _server(backend, clock, budget, slots=4, chunk=10):
    return sv.Server(backend, budget, slots, chunk, clock=clock, sleep=clock.sleep)


def test_all_complete_with_latency_and_throughput():
    c = Clock()
    b = FakeBackend(c)
    jobs = _jobs([(10000, 100, 0.0), (20000, 200, 0.001), (5000, 50, 0.002)])
    rep = _server(b, c, 10**9).run(jobs)
    assert all(j.status == sv.DONE for j in jobs)
    assert all(j.latency > 0 and j.queue_delay >= 0 for j in jobs)
    assert rep.atom_steps == 10000 * 100 + 20000 * 200 + 5000 * 50
    s = rep.summary()
    assert s["done"] == 3 and s["latency_s"]["p50"] > 0 and s["atom_steps_per_s"] > 0
    assert b.live == 0


def test_budget_limits_concurrency_and_rejects_oversized():
    c = Clock()
    b = FakeBackend(c, bytes_per_atom=1000)
    # budget fits two 40k jobs at once; the 2M job can never fit
    jobs = _jobs([(40000, 50, 0.0)] * 4 + [(2_000_000, 10, 0.0)])
    rep = _server(b, c, budget=90_000_000, slots=8).run(jobs)
    assert jobs[-1].status == sv.REJECTED
    assert all(j.status == sv.DONE for j in jobs[:4])
    assert rep.peak_bytes <= 90_000_000 and b.max_live == 2


def test_slots_limit():
    c = Clock()
    b = FakeBackend(c)
    jobs = _jobs([(1000, 100, 0.0)] * 10)
    rep = _server(b, c, 10**12, slots=3).run(jobs)
    assert rep.max_active == 3 and b.max_live == 3
    assert all(j.status == sv.DONE for j in jobs)


def test_late_arrival_joins_while_others_run():
    # continuous batching: a request arriving mid-run is admitted before the
    # long-running one finishes, and finishes first
    c = Clock()
    b = FakeBackend(c, rate=1e7)
    jobs = _jobs([(100000, 2000, 0.0), (2000, 100, 0.5)])
    _server(b, c, 10**12).run(jobs)
    long, short = jobs
    assert short.admitted_at < long.finished_at
    assert short.finished_at < long.finished_at


def test_first_fit_lets_small_requests_bypass_without_starving():
    c = Clock()
    b = FakeBackend(c, bytes_per_atom=1000)
    # job 1 (80 MB) waits for job 0 (50 MB) to finish; job 2 (10 MB) fits now
    jobs = _jobs([(50000, 400, 0.0), (80000, 10, 0.001), (10000, 10, 0.002)])
    _server(b, c, budget=100_000_000).run(jobs)
    assert jobs[2].admitted_at < jobs[1].admitted_at
    assert jobs[1].status == sv.DONE


def test_cancel_queued_and_running():
    c = Clock()
    b = FakeBackend(c, rate=1e6)
    jobs = _jobs([(100000, 1000, 0.0), (1000, 10, 0.0)])
    jobs[1].cancel = True                       # cancelled while queued
    srv = _server(b, c, 10**12, slots=1)
    orig = b.advance

    def advance(slot, k):                       # cancel the big one mid-run
        orig(slot, k)
        if slot["job"].steps_done >= 200:
            slot["job"].cancel = True
    b.advance = advance
    srv.run(jobs)
    assert jobs[0].status == sv.CANCELLED and jobs[0].steps_done < 1000
    assert jobs[1].status == sv.CANCELLED
    assert b.live == 0


def test_injected_failures_do_not_stop_the_server():
    c = Clock()
    b = FakeBackend(c, fail_start={1}, fail_finish={2})
    jobs = _jobs([(1000, 20, 0.0), (1000, 20, 0.0), (1000, 20, 0.0), (1000, 20, 0.0)])
    rep = _server(b, c, 10**12).run(jobs)
    assert [j.status for j in jobs] == [sv.DONE, sv.FAILED, sv.FAILED, sv.DONE]
    assert "allocation" in jobs[1].error and "non-finite" in jobs[2].error
    assert rep.summary()["failed"] == 2 and b.live == 0


def test_trace_generator_shapes():
    from paper_1502_03234_gb300 import slabgen

    tr = slabgen.make_trace(400, 20.0, 2048, 524288, 100, 2000, seed=0)
    arr = np.array([r.arrival_s for r in tr])
    assert np.all(np.diff(arr) > 0)
    rate = len(tr) / arr[-1]
    assert 15 < rate < 25                                   # Poisson, mean 20/s
    ns = np.array([r.n for r in tr])
    assert ns.min() >= 2048 and ns.max() <= 524288
    lg = np.log(ns)
    assert abs(lg.mean() - 0.5 * (np.log(2048) + np.log(524288))) < 0.3   # log-uniform


class ResumableBackend(FakeBackend):
    """FakeBackend whose state is the number of steps a request has run:
    checkpoint() reads it back, start() resumes from job.x."""

    def start(self, job):
        slot = super().start(job)
        slot["steps"] = job.x if isinstance(job.x, int) else 0
        assert slot["steps"] == job.resume_step
        slot["resumed"] = job.resume_step > 0
        return slot

    def advance(self, slot, nsteps):
        super().advance(slot, nsteps)
        slot["steps"] += nsteps

    def checkpoint(self, slot):
        assert self.inflight(slot) == 0          # never while chunks run
        return slot["steps"], None

    def finish(self, slot):
        return (slot["steps"], slot["resumed"], None)


def test_eviction_frees_the_budget_and_resumes_the_victim():
    # a long request holds the budget; a later one that does not fit waits
    # evict_after, the long one is checkpointed at a chunk boundary and
    # requeued, and finishes from its state once the other is done
    c = Clock()
    b = ResumableBackend(c, rate=1e7)
    jobs = _jobs([(100000, 400, 0.0), (80000, 20, 0.05)])
    budget = 100000 * 500 + 50000 * 500          # both do not fit at once
    srv = sv.Server(b, budget, 4, 10, clock=c, sleep=c.sleep, evict_after=0.02)
    rep = srv.run(jobs)
    long, short = jobs
    assert all(j.status == sv.DONE for j in jobs), [j.error for j in jobs]
    assert rep.evictions == 1 and long.evictions == 1 and short.evictions == 0
    assert long.result[0] == 400 and long.result[1]            # all steps, after a resume
    assert long.resume_step % 2 == 0 and 0 < long.resume_step < 400
    assert short.finished_at < long.finished_at                 # the waiter ran first
    assert rep.peak_bytes <= budget
    assert b.live == 0


def test_no_eviction_without_the_policy_or_when_it_fits():
    c = Clock()
    b = ResumableBackend(c, rate=1e7)
    jobs = _jobs([(100000, 200, 0.0), (80000, 20, 0.05)])
    rep = sv.Server(b, 100000 * 500 + 50000 * 500, 4, 10, clock=c, sleep=c.sleep).run(jobs)
    assert rep.evictions == 0 and jobs[1].admitted_at >= jobs[0].finished_at
    c2 = Clock()
    b2 = ResumableBackend(c2, rate=1e7)
    jobs = _jobs([(100000, 200, 0.0), (80000, 20, 0.05)])
    rep = sv.Server(b2, 10**9, 4, 10, clock=c2, sleep=c2.sleep, evict_after=0.0).run(jobs)
    assert rep.evictions == 0                                   # it fits: nothing to evict


def test_a_victim_is_evicted_at_most_max_evictions_times():
    c = Clock()
    b = ResumableBackend(c, rate=1e7)
    # three large requests, room for one at a time: evictions bounded
    jobs = _jobs([(100000, 300, 0.0), (100000, 300, 0.01), (100000, 300, 0.02)])
    rep = sv.Server(b, 100000 * 500, 4, 10, clock=c, sleep=c.sleep, evict_after=0.005,
                    max_evictions=1).run(jobs)
    assert all(j.status == sv.DONE for j in jobs)
    assert all(j.evictions <= 1 for j in jobs)
    assert all(j.result[0] == 300 for j in jobs)
    assert rep.peak_bytes <= 100000 * 500
