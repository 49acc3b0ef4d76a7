"""GPU parity of the Mumford-Shah segmentation (Eq. 13, fixed densities): the
CUDA primal-dual iteration through the C ABI against the oracle's, bit for
bit on the labels and on the relaxed field u (both run the same FP64
operations in the same order), on random images and on a noisy slab."""
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


@pytest.mark.parametrize("nu", [0.0, 0.05, 0.3])
def test_segmentation_bit_exact(dcm, orc, nu):
    s = slabgen.make_slab(6000, seed=71)
    with dcm.System(s.box, len(s.x)) as sy:
        dims = sy.grid()[0]
        rng = np.random.default_rng(int(100 * nu))
        rho = rng.random(int(np.prod(dims))) * 1.2
        lab, u = sy.ms_segment(rho, 0.8, 0.1, nu, 150)
    ref, uref = orc.ms_segment(dims, rho, 0.8, 0.1, nu, 150)
    assert np.array_equal(lab, ref)
    assert np.array_equal(u, uref)


def test_noisy_slab_planes(dcm, orc):
    s = slabgen.make_slab(6000, seed=72)
    with dcm.System(s.box, len(s.x)) as sy:
        dims = sy.grid()[0]
        nx, ny, nz = dims
        z = np.repeat(np.arange(nz), nx * ny)
        clean = np.where((z >= nz // 3) & (z < 2 * nz // 3), 0, 1).astype(np.uint8)
        rng = np.random.default_rng(5)
        rho = np.where(clean == 0, 0.8, 0.05) + rng.uniform(-0.5, 0.5, clean.size)
        lab, u = sy.ms_segment(rho, 0.8, 0.05, 0.2, 1500)
    ref, uref = orc.ms_segment(dims, rho, 0.8, 0.05, 0.2, 1500)
    assert np.array_equal(lab, ref) and np.array_equal(u, uref)
    assert np.array_equal(lab, clean)


def test_argument_errors(dcm):
    s = slabgen.make_slab(4000, seed=73)
    with dcm.System(s.box, len(s.x)) as sy:
        nv = int(np.prod(sy.grid()[0]))
        with pytest.raises(dcm.DcmError) as e:
            sy.ms_segment(np.zeros(nv), 0.8, 0.1, -1.0, 10)
        assert e.value.code == dcm.DCM_ERR_ARG
        with pytest.raises(ValueError):
            sy.ms_segment(np.zeros(nv - 1), 0.8, 0.1, 0.1, 10)


# ---- Eq. 13 as the detection's segmentation step (DCM_SEG_MUMFORD_SHAH) --------
MS = dict(segmentation=1, ms_nu=0.005, ms_iters=50, ms_outer=4)


def _detect_both(dcm, orc, x, box, rc=(3.0, 6.0), ms=MS, **kw):
    with dcm.System(box, len(x), rc_min=rc[0], rc_max=rc[1], **ms, **kw) as sy:
        sy.set_state(x, None)
        sy.detect_interface()
        dims, B, Bs, S, D = sy.grid()
        d, rcv, cls = sy.cutoffs()
        xg, _, _ = sy.get_state()
    det = orc.detect(xg, box, orc.DetectParams(rc_min=rc[0], rc_max=rc[1], voxel=1.0,
                                               segmentation=1, ms_nu=ms["ms_nu"],
                                               ms_iters=ms["ms_iters"], ms_outer=ms["ms_outer"]))
    return (dims, B, Bs, S, D, d, rcv, cls), det


@pytest.mark.parametrize("rounds", [4, 1], ids=["alternating", "default-one-round"])
@pytest.mark.parametrize("n,seed,amp", [(16000, 91, 0.0), (262144, 92, 0.0), (65536, 93, 1.0)])
def test_detection_with_eq13_bit_exact(dcm, orc, n, seed, amp, rounds):
    s = slabgen.make_slab(n, seed=seed, capillary_amp=amp)
    ms = dict(MS, ms_outer=rounds)
    (dims, B, Bs, S, D, d, rcv, cls), det = _detect_both(dcm, orc, s.x, s.box, ms=ms)
    assert dims == det.dims
    assert np.array_equal(B, det.B) and np.array_equal(Bs, det.Bs)
    assert np.array_equal(S, det.S)                   # Eq. 13 labels, bit-exact
    np.testing.assert_allclose(D, det.D, atol=1e-12, rtol=0)
    np.testing.assert_allclose(d, det.d, atol=1e-12, rtol=0)
    np.testing.assert_allclose(rcv, det.rc, rtol=1e-13, atol=0)
    assert np.array_equal(cls, det.cls)
    # and it is not the K-means labelling
    km = orc.detect(s.x, s.box, orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0))
    print(f"N={n}: Eq. 13 changed {int((det.S != km.S).sum())} voxels against K-means")


def test_detection_with_eq13_in_an_ensemble(dcm, orc):
    mem = [slabgen.make_slab(9001, seed=94), slabgen.make_slab(16000, 0.8, seed=95)]
    params = [dcm.default_params(**MS) for _ in mem]
    with dcm.Ensemble([m.box for m in mem], [len(m.x) for m in mem], params) as ens:
        for k, m in enumerate(mem):
            ens.set_system_state(k, m.x, m.v)
        ens.detect_interface()
        _, rc_all, cls_all = ens.cutoffs()
        got = [ens.get_system_state(k)[0] for k in range(len(mem))]
        for k, m in enumerate(mem):
            first, count = ens.ranges[k]
            det = orc.detect(got[k], m.box, orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0,
                                                             segmentation=1))
            np.testing.assert_allclose(rc_all[first:first + count], det.rc, rtol=1e-13, atol=0)
            assert np.array_equal(cls_all[first:first + count], det.cls)


def test_steps_with_eq13_match_the_oracle(dcm, orc):
    s = slabgen.make_slab(16000, seed=96)
    with dcm.System(s.box, len(s.x), precision=dcm.DCM_MIXED, skin=0.5, **MS) as sy:
        sy.set_state(s.x, s.v)
        sy.step(10)
        sy.sync()
        x, _, _ = sy.get_state()
        st = sy.stats()
    assert st.kernels_detect > st.kernels_plain          # the segmentation is in the graph
    p = orc.RunParams(det=orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0, segmentation=1),
                      dt=0.005, detect_every=2, cell_min=1.5)
    xr, *_ = orc.run(s.x, s.v, s.box, p, 10)
    L = np.asarray(s.box)
    dx = x - xr
    dx -= np.round(dx / L) * L
    assert np.abs(dx).max() < 1e-4
