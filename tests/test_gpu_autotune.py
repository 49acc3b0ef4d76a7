"""GPU: the autotuner of the force kernels' launch shape (the analogue of the
thesis's schedule(dynamic,20) tuning, Section 5.1).  tune_live picks the list
lanes of the mixed-precision Verlet-list force on a live system and on a live
ensemble, and the lanes per cutoff class of the FP64 lanes walk; a tuned
handle's forces and interacting pairs must still be exactly those of the
definition (the oracle), and tuned_system reuses its cache."""
import os

import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen

pytestmark = pytest.mark.gpu

FP64_REL, FP64_ABS = 1e-5, 1e-6
LISTS = dict(skin=0.6, skin_time=0.04, skin_floor=0.05)


@pytest.fixture(scope="module")
def dcm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import dcm as d

    return d


def _check_against_oracle(orc, x, f, rc, npair, box, nc):
    ref = orc.forces(x, rc, box, nc)
    assert np.array_equal(npair, ref.npair)
    err = np.linalg.norm(f - ref.f, axis=1)
    bar = FP64_ABS + FP64_REL * np.linalg.norm(ref.f, axis=1)
    assert np.all(err <= bar), (err.max(), np.max(err / bar))


def test_tune_live_list_lanes_single_system(dcm, orc):
    from paper_1502_03234_gb300 import autotune

    s = slabgen.make_slab(16000, seed=61)
    log = []
    with dcm.System(s.box, len(s.x), precision=dcm.DCM_MIXED, **LISTS) as sy:
        sy.set_state(s.x, s.v)
        sy.step(4)
        best = autotune.tune_live(sy, reps=3, log=log.append)
        assert best["list_lanes"] in autotune.LIST_LANES
        # every uniform shape was timed, then the per-class descent
        assert len(log) >= len(autotune.LIST_LANES) + 1
        assert dcm.dcm_get_tuning(sy.h).list_lanes == best["list_lanes"]
        cls = best.get("list_lanes_class")
        got = list(dcm.dcm_get_tuning(sy.h).list_lanes_class)
        assert got[:4] == (list(cls)[:4] if cls else [0, 0, 0, 0])
        assert best["force_ms"] > 0
        sy.step(3)
        sy.sync()
        x, _, f = sy.get_state()
        _, rc, _ = sy.cutoffs()
        npair = sy.pair_counts()
        nc, _, _ = sy.cells()
    _check_against_oracle(orc, x, f, rc, npair, s.box, nc)


def test_tune_live_ensemble(dcm, orc):
    from paper_1502_03234_gb300 import autotune

    spec = [(5001, 0.65, 11), (12000, 0.8, 12), (9001, 0.7, 13), (3333, 0.85, 14)]
    mem = [slabgen.make_slab(n, t, seed=sd) for n, t, sd in spec]
    params = [dcm.default_params(precision=dcm.DCM_MIXED, **LISTS) for _ in mem]
    with dcm.Ensemble([m.box for m in mem], [len(m.x) for m in mem], params) as ens:
        for k, m in enumerate(mem):
            ens.set_system_state(k, m.x, m.v)
        ens.step(4)
        best = autotune.tune_live(ens, reps=3)
        assert best["list_lanes"] in autotune.LIST_LANES
        ens.step(3)
        ens.sync()
        npair_all = ens.pair_counts()
        _, rc_all, _ = ens.cutoffs()
        for k, m in enumerate(mem):
            x, _, f = ens.get_system_state(k)
            first, count = ens.ranges[k]
            # (the oracle's link cells only enumerate the pairs: any grid
            # whose cells hold the stencil gives the same pair set)
            nc = tuple(int(q) for q in np.floor(np.asarray(m.box) / 1.5))
            _check_against_oracle(orc, x, f, rc_all[first:first + count],
                                  npair_all[first:first + count], m.box, nc)


def test_tune_live_fp64_lanes(dcm, orc):
    from paper_1502_03234_gb300 import autotune

    s = slabgen.make_slab(9001, seed=62)
    with dcm.System(s.box, len(s.x), precision=dcm.DCM_FP64) as sy:
        sy.set_state(s.x, s.v)
        sy.step(2)
        best = autotune.tune_live(sy, reps=2)
        assert best["walk"] == dcm.DCM_WALK_LANES
        t = dcm.dcm_get_tuning(sy.h)
        assert list(t.lanes)[:4] == list(best["lanes"])[:4] or len(best["lanes"]) < 4
        sy.step(2)
        sy.sync()
        x, _, f = sy.get_state()
        _, rc, _ = sy.cutoffs()
        npair = sy.pair_counts()
        nc, _, _ = sy.cells()
    _check_against_oracle(orc, x, f, rc, npair, s.box, nc)


def test_tuned_system_caches_the_choice(dcm, orc, tmp_path):
    from paper_1502_03234_gb300 import autotune

    s = slabgen.make_slab(9001, seed=63)
    p = dcm.default_params(precision=dcm.DCM_MIXED, **LISTS)
    cache = os.path.join(tmp_path, "tune.json")
    calls = []
    sy, t = autotune.tuned_system(s.box, s.x, s.v, p, cache_path=cache, log=calls.append)
    sy.close()
    assert calls and os.path.exists(cache)               # tuned and stored
    key = autotune.key(len(s.x), p.rc_min, p.rc_max, p.precision, p.skin)
    assert key in autotune.load_cache(cache)
    again = []
    sy, t2 = autotune.tuned_system(s.box, s.x, s.v, p, cache_path=cache, log=again.append)
    assert not again                                     # from the cache, no timing
    assert (t2.cell_min, t2.list_lanes) == (t.cell_min, t.list_lanes)
    with sy:
        assert dcm.dcm_get_tuning(sy.h).list_lanes == t.list_lanes
        sy.step(3)
        sy.sync()
        x, _, f = sy.get_state()
        _, rc, _ = sy.cutoffs()
        npair = sy.pair_counts()
        nc, _, _ = sy.cells()
    _check_against_oracle(orc, x, f, rc, npair, s.box, nc)


@pytest.mark.parametrize("lanes", [[4, 8, 16, 32], [32, 16, 8, 4], [4, 4, 4, 4]])
def test_per_class_list_lanes_match_oracle(dcm, orc, lanes):
    # the class-ordered list force with lanes per cutoff class: the same pair
    # set and forces within the bar, whatever lanes each class gets
    s = slabgen.make_slab(12000, seed=64)
    with dcm.System(s.box, len(s.x), precision=dcm.DCM_MIXED, **LISTS) as sy:
        sy.set_state(s.x, s.v)
        sy.step(2)
        sy.set_tuning([1], 128, dcm.DCM_WALK_WARP, 8, lanes)
        assert list(dcm.dcm_get_tuning(sy.h).list_lanes_class)[:4] == lanes
        sy.step(5)
        sy.sync()
        assert sy.stats().list_builds >= 1
        x, _, f = sy.get_state()
        _, rc, _ = sy.cutoffs()
        npair = sy.pair_counts()
        nc, _, _ = sy.cells()
    _check_against_oracle(orc, x, f, rc, npair, s.box, nc)


def test_per_class_list_lanes_rejected_where_they_do_not_apply(dcm):
    s = slabgen.make_slab(4001, seed=65)
    with dcm.System(s.box, len(s.x), precision=dcm.DCM_FP64) as sy:
        with pytest.raises(dcm.DcmError) as e:
            sy.set_tuning([16], 128, dcm.DCM_WALK_LANES, 8, [4, 8, 16, 32])
        assert e.value.code == dcm.DCM_ERR_ARG
    with dcm.System(s.box, len(s.x), precision=dcm.DCM_MIXED, **LISTS) as sy:
        with pytest.raises(dcm.DcmError) as e:
            sy.set_tuning([1], 128, dcm.DCM_WALK_WARP, 8, [4, 8, 12, 32])
        assert e.value.code == dcm.DCM_ERR_ARG
