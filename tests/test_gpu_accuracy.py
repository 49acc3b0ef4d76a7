"""The linear cutoff function (Section 3.1, Fig. 12) on the GPU against the
oracle, and the force-accuracy measure of Section 6.1.1 (Eq. 20) computed
from GPU forces against the same measure from oracle forces, with the trends
of Fig. 34 (a larger r_c,max and the exponential function give smaller
errors).  The reference is a static r_c = 12 sigma (the thesis uses Ewald
sums, which are not part of this path)."""
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


def _minimg(d, box):
    L = np.asarray(box)
    return d - np.round(d / L) * L


def eq20(f, ref):
    d = np.linalg.norm(f - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    return np.sqrt(np.mean((d / r) ** 2)), np.sqrt((d * d).sum() / (r * r).sum())


@pytest.mark.parametrize("rc", [(3.0, 6.0), (4.5, 9.0)])
def test_linear_cutoff_detection_parity(dcm, orc, rc):
    s = slabgen.make_slab(16000 if rc[1] < 7 else 30000, seed=61)
    with dcm.System(s.box, len(s.x), rc_min=rc[0], rc_max=rc[1],
                    cutoff_fn=dcm.DCM_CUTOFF_LINEAR) as sy:
        sy.set_state(s.x, s.v)
        sy.detect_interface()
        d, rcv, cls = sy.cutoffs()
        x, _, _ = sy.get_state()
    det = orc.detect(x, s.box, orc.DetectParams(rc_min=rc[0], rc_max=rc[1], cutoff_fn=1))
    np.testing.assert_allclose(d, det.d, atol=1e-12, rtol=0)
    np.testing.assert_allclose(rcv, det.rc, rtol=1e-13, atol=0)
    assert np.array_equal(cls, det.cls)
    exp = orc.detect(x, s.box, orc.DetectParams(rc_min=rc[0], rc_max=rc[1]))
    assert np.all(rcv <= exp.rc + 1e-12) and np.any(rcv < exp.rc - 0.1)


@pytest.mark.parametrize("prec,skin", [(0, 0.0), (1, 0.5)])
def test_linear_cutoff_trajectory(dcm, orc, prec, skin):
    # 10 steps with detection every 2 (Verlet lists anticipate the cutoff with
    # the linear function): positions within 1e-4 of the oracle's
    s = slabgen.make_slab(16000, seed=62)
    with dcm.System(s.box, len(s.x), precision=prec, skin=skin,
                    cutoff_fn=dcm.DCM_CUTOFF_LINEAR) as sy:
        sy.set_state(s.x, s.v)
        sy.step(10)
        sy.sync()
        x, _, _ = sy.get_state()
    p = orc.RunParams(det=orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0, cutoff_fn=1),
                      dt=0.005, detect_every=2, cell_min=1.5)
    xr, *_ = orc.run(s.x, s.v, s.box, p, 10)
    assert np.abs(_minimg(x - xr, s.box)).max() < 1e-4


def test_force_error_against_large_static_cutoff(dcm, orc):
    # 20,000 atoms: L = 26.5 sigma holds the r_c = 12 reference (1-sigma link
    # cells keep the stencil inside the box)
    s = slabgen.make_slab(20000, seed=63)
    n = len(s.x)

    def gpu_forces(rc_min, rc_max, fn):
        with dcm.System(s.box, n, rc_min=rc_min, rc_max=rc_max, cutoff_fn=fn,
                        cell_min=1.0) as sy:
            sy.set_state(s.x, s.v)
            sy.detect_interface()
            sy.compute_forces()
            _, rc, _ = sy.cutoffs()
            x, _, f = sy.get_state()
            nc, _, _ = sy.cells()
        return x, rc, f, nc

    x, _, ref, nc = gpu_forces(12.0, 12.0, 0)
    ref_o = orc.forces(x, 12.0, s.box, nc).f
    np.testing.assert_allclose(ref, ref_o, rtol=1e-5, atol=1e-6)
    errs = {}
    for fn in (0, 1):
        for rc_max in (5.0, 6.0, 7.0):
            x, rc, f, nc = gpu_forces(3.0, rc_max, fn)
            fo = orc.forces(x, rc, s.box, nc).f
            e_gpu = eq20(f, ref)
            e_orc = eq20(fo, ref_o)
            np.testing.assert_allclose(e_gpu, e_orc, rtol=1e-4)
            errs[fn, rc_max] = e_gpu[1]
    # Fig. 34: the error falls as r_c,max grows, and the exponential
    # function (larger cutoffs everywhere) beats the linear one
    for fn in (0, 1):
        assert errs[fn, 5.0] > errs[fn, 6.0] > errs[fn, 7.0]
    for rc_max in (5.0, 6.0, 7.0):
        assert errs[0, rc_max] < errs[1, rc_max]
