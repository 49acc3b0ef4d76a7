"""GPU: checkpoint and resume.  A run's state (positions, velocities) read
back at a detection boundary, the handle destroyed, a new handle given that
state and the step counter (dcm_set_step) continues exactly where the
uninterrupted run goes: bit for bit without Verlet lists (the resumed run
re-detects the interface at the same positions and recomputes the same
forces), and within the force tolerance with lists (the resume rebuilds
them, so their order, and the FP32 summation order of the list force,
differ).  The serving scheduler uses this to evict a running request under
HBM-budget pressure and to re-admit it later."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dcm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import dcm as d

    return d


def _run(dcm, s, prec, steps, skin, x=None, v=None, step0=0):
    with dcm.System(s.box, len(s.x), precision=prec, skin=skin) as sy:
        sy.set_state(s.x if x is None else x, s.v if v is None else v)
        if step0:
            sy.set_step(step0)
        sy.step(steps)
        sy.sync()
        return sy.get_state(), sy.energy_virial()


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_without_lists_is_bit_identical(dcm, prec):
    s = slabgen.make_slab(9001, seed=71)
    (xa, va, fa), ea = _run(dcm, s, prec, 12, 0.0)
    (x6, v6, _), _ = _run(dcm, s, prec, 6, 0.0)          # checkpoint at step 6 (detects)
    (xb, vb, fb), eb = _run(dcm, s, prec, 6, 0.0, x6, v6, step0=6)
    assert np.array_equal(xa, xb)
    assert np.array_equal(va, vb)
    assert np.array_equal(fa, fb)
    assert ea[0] == eb[0] and ea[1] == eb[1]


def test_resume_with_lists_within_tolerance(dcm, orc):
    s = slabgen.make_slab(9001, seed=72)
    (xa, va, fa), _ = _run(dcm, s, 1, 12, 0.5)
    (x6, v6, _), _ = _run(dcm, s, 1, 6, 0.5)
    (xb, vb, fb), _ = _run(dcm, s, 1, 6, 0.5, x6, v6, step0=6)
    L = np.asarray(s.box)
    dx = xa - xb
    dx -= np.round(dx / L) * L
    assert np.abs(dx).max() < 1e-9
    assert np.abs(va - vb).max() < 1e-6
    # both are within the force bar of the definition at their own positions
    for x, f in ((xa, fa), (xb, fb)):
        with dcm.System(s.box, len(s.x), precision=1, skin=0.5) as sy:
            sy.set_state(x, va)
            sy.compute_forces()
            _, rc, _ = sy.cutoffs()
            nc, _, _ = sy.cells()
        ref = orc.forces(x, rc, s.box, nc)
        err = np.linalg.norm(f - ref.f, axis=1)
        assert np.all(err <= 1e-6 + 1e-5 * np.linalg.norm(ref.f, axis=1))


def test_serving_eviction_resumes_bit_identical(dcm):
    # a budget that holds one of the two requests: the long one is evicted
    # for the short one and resumed from its checkpoint; its result equals
    # the same request run alone, bit for bit (no Verlet lists)
    from paper_1502_03234_gb300 import serving as sv

    slabs = [slabgen.make_slab(16000, seed=81, min_edge=17.0),
             slabgen.make_slab(9001, seed=82, min_edge=17.0)]

    def jobs():
        return [sv.Job(rid=0, n=16000, nsteps=120, box=slabs[0].box, x=slabs[0].x, v=slabs[0].v,
                       arrival=0.0),
                sv.Job(rid=1, n=9001, nsteps=20, box=slabs[1].box, x=slabs[1].x, v=slabs[1].v,
                       arrival=0.0)]

    backend = sv.DcmBackend(precision=dcm.DCM_MIXED, skin=0.0)
    js = jobs()
    budget = max(backend.estimate(j) for j in js) + 1
    rep = sv.Server(backend, budget, max_slots=2, chunk_steps=10, evict_after=0.0).run(
        js, realtime=False)
    assert all(j.status == sv.DONE for j in js), [j.error for j in js]
    assert rep.evictions >= 1 and js[0].evictions == 1
    alone = jobs()[:1]
    sv.Server(backend, budget, max_slots=1, chunk_steps=10).run(alone, realtime=False)
    for a, b in zip(alone[0].result, js[0].result):
        assert np.array_equal(a, b)
