"""GPU: the batched ensemble (many systems in one handle, one set of kernels
and one persistent force launch per step).  Every member must match the
oracle and be identical to the same system run alone."""
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


def _members():
    # uneven sizes, temperatures and one member with r_c,max = 7
    spec = [(5001, 0.65, 6.0, 11), (16000, 0.8, 6.0, 12), (9001, 0.7, 7.0, 13), (3333, 0.85, 6.0, 14)]
    out = []
    for n, t, rcmax, seed in spec:
        out.append((slabgen.make_slab(n, t, seed=seed), rcmax))
    return out


def _minimg(d, box):
    L = np.asarray(box)
    return d - np.round(d / L) * L


@pytest.mark.parametrize("prec", [0, 1])
def test_ensemble_members_equal_single_runs(dcm, prec):
    mem = _members()
    params = [dcm.default_params(precision=prec, rc_max=rcmax) for _, rcmax in mem]
    boxes = [s.box for s, _ in mem]
    ns = [len(s.x) for s, _ in mem]
    with dcm.Ensemble(boxes, ns, params) as ens:
        for k, (s, _) in enumerate(mem):
            ens.set_system_state(k, s.x, s.v)
        ens.step(12)
        ens.sync()
        got = [ens.get_system_state(k) for k in range(len(mem))]
        tun = dcm.dcm_get_tuning(ens.h)
        lanes, block, walk = list(tun.lanes), tun.block, tun.walk
        e_mix = [ens.system_energy(k) for k in range(len(mem))]
    for k, (s, rcmax) in enumerate(mem):
        with dcm.System(s.box, len(s.x), dcm.default_params(precision=prec, rc_max=rcmax)) as one:
            one.set_tuning(lanes, block, walk)
            one.set_state(s.x, s.v)
            one.step(12)
            one.sync()
            x, v, f = one.get_state()
            e_one = one.energy_virial()
        # same arithmetic in the same order: identical, not just close
        assert np.array_equal(got[k][0], x), k
        assert np.array_equal(got[k][1], v), k
        assert np.array_equal(got[k][2], f), k
        assert e_mix[k][0] == e_one[0] and e_mix[k][1] == e_one[1]


@pytest.mark.parametrize("prec,skin", [(0, 0.0), (1, 0.5)])
def test_ensemble_members_match_oracle(dcm, orc, prec, skin):
    # with Verlet lists (skin 0.5, the benchmark setting) the ensemble shares
    # one rebuild decision, so a member's lists are rebuilt on a schedule set
    # by all members: still the same pairs, checked against the oracle
    mem = _members()
    params = [dcm.default_params(precision=prec, rc_max=rcmax, skin=skin) for _, rcmax in mem]
    with dcm.Ensemble([s.box for s, _ in mem], [len(s.x) for s, _ in mem], params) as ens:
        for k, (s, _) in enumerate(mem):
            ens.set_system_state(k, s.x, s.v)
        ens.step(10)
        ens.sync()
        got = [ens.get_system_state(k)[0] for k in range(len(mem))]
    for k, (s, rcmax) in enumerate(mem):
        p = orc.RunParams(det=orc.DetectParams(rc_min=3.0, rc_max=rcmax, voxel=1.0), dt=0.005,
                          detect_every=2, cell_min=1.5)
        xr, *_ = orc.run(s.x, s.v, s.box, p, 10)
        assert np.abs(_minimg(got[k] - xr, s.box)).max() < 1e-4, k


def test_ensemble_rejects_mixed_precision_members(dcm):
    s = slabgen.make_slab(3333, seed=3)
    p = [dcm.default_params(precision=0), dcm.default_params(precision=1)]
    with pytest.raises(dcm.DcmError):
        dcm.Ensemble([s.box, s.box], [3333, 3333], p)
