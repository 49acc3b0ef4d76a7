"""GPU: dcm_update_state, the state of a running system replaced from the
host (a host-side thermostat or constraint, or the host's own copy handed
back each step).  The step counter, the cutoffs of the last detection and the
Verlet lists stay; the forces are recomputed from the new positions; the
lists are rebuilt only when the reuse test finds a particle moved beyond its
skin share.  The forces after an update are those of the definition (the
oracle) at the new positions with the handle's cutoffs."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen

pytestmark = pytest.mark.gpu

LISTS = dict(skin=0.6, skin_time=0.04, skin_floor=0.05)
REL, ABS = 1e-5, 1e-6


@pytest.fixture(scope="module")
def dcm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import dcm as d

    return d


def _check(orc, sy, box):
    x, _, f = sy.get_state()
    _, rc, _ = sy.cutoffs()
    npair = sy.pair_counts()
    nc, _, _ = sy.cells()
    ref = orc.forces(x, rc, box, nc)
    assert np.array_equal(npair, ref.npair)
    err = np.linalg.norm(f - ref.f, axis=1)
    bar = ABS + REL * np.linalg.norm(ref.f, axis=1)
    assert np.all(err <= bar), (err.max(), np.max(err / bar))


@pytest.mark.parametrize("prec", [0, 1])
def test_handing_back_the_running_state_keeps_lists_and_trajectory(dcm, prec):
    s = slabgen.make_slab(9001, seed=81)
    with dcm.System(s.box, len(s.x), precision=prec, **LISTS) as a, \
            dcm.System(s.box, len(s.x), precision=prec, **LISTS) as b:
        for sy in (a, b):
            sy.set_state(s.x, s.v)
            sy.step(5)                       # (an odd step: the next one detects)
        x, v, _ = a.get_state()
        builds = a.stats().list_builds
        a.update_state(x, v)
        a.compute_forces()
        a.sync()
        assert a.stats().list_builds == builds           # nothing moved: lists kept
        for _ in range(7):
            x, v, _ = a.get_state()
            a.update_state(x, v)
            a.step(1)
        b.step(7)
        a.sync()
        b.sync()
        xa, va, _ = a.get_state()
        xb, vb, _ = b.get_state()
        # the same trajectory (forces recomputed by the list force where the
        # uninterrupted run had them from the same kernel or the rebuild walk:
        # FP32 partial sums may round differently)
        assert np.allclose(xa, xb, rtol=0, atol=1e-9)
        assert np.allclose(va, vb, rtol=0, atol=1e-7)
        assert a.stats().step == b.stats().step


@pytest.mark.parametrize("prec", [0, 1])
def test_forces_after_an_update_are_the_definition(dcm, orc, prec):
    s = slabgen.make_slab(9001, seed=82)
    rng = np.random.default_rng(3)
    with dcm.System(s.box, len(s.x), precision=prec, **LISTS) as sy:
        sy.set_state(s.x, s.v)
        sy.step(4)
        x, v, _ = sy.get_state()
        builds = sy.stats().list_builds
        # a small move (well inside the skin shares): the lists stay
        xs = x + rng.uniform(-0.01, 0.01, x.shape)
        sy.update_state(xs, v)
        sy.compute_forces()
        sy.sync()
        assert sy.stats().list_builds == builds
        _check(orc, sy, s.box)
        # a large one for a few particles: the reuse test rebuilds
        xl = xs.copy()
        xl[rng.choice(len(x), 20, replace=False)] += 0.9
        sy.update_state(xl, v)
        sy.compute_forces()
        sy.sync()
        assert sy.stats().list_builds == builds + 1
        _check(orc, sy, s.box)
        sy.step(3)
        sy.sync()
        _check(orc, sy, s.box)


def test_update_before_any_force_is_a_set_state(dcm, orc):
    s = slabgen.make_slab(4001, seed=83)
    with dcm.System(s.box, len(s.x), precision=1, **LISTS) as sy:
        sy.set_step(7)
        sy.update_state(s.x, s.v)
        assert sy.stats().step == 7
        sy.compute_forces()
        sy.sync()
        _check(orc, sy, s.box)


def test_update_state_rejects_ensembles(dcm):
    mem = [slabgen.make_slab(n, seed=sd) for n, sd in [(3001, 84), (4001, 85)]]
    params = [dcm.default_params(precision=dcm.DCM_MIXED) for _ in mem]
    with dcm.Ensemble([m.box for m in mem], [len(m.x) for m in mem], params) as ens:
        for k, m in enumerate(mem):
            ens.set_system_state(k, m.x, m.v)
        with pytest.raises(dcm.DcmError) as e:
            ens.update_state(np.concatenate([m.x for m in mem]))
        assert e.value.code == dcm.DCM_ERR_ARG
