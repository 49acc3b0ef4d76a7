"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.  Bars: integer results bit-exact (cells, voxel counts,
smoothed values, labels, classes, interacting-pair counts); forces per particle
within 1e-6 + 1e-5 |F| in both precision modes (FP64, and MIXED: FP32 pairs
beyond 1.5 sigma, double-float close pairs, exact FP64 sums); positions within
1e-4 after 10 steps."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen

pytestmark = pytest.mark.gpu

FP64_REL, FP64_ABS = 1e-5, 1e-6


def _force_bar(f, ref_f, label=""):
    """the per-particle force bar |F - F_ref| <= 1e-6 + 1e-5 |F_ref|; prints
    the error distribution (max, p99, largest fraction of the bar)"""
    err = np.linalg.norm(f - ref_f, axis=1)
    fmag = np.linalg.norm(ref_f, axis=1)
    bar = FP64_ABS + FP64_REL * fmag
    print(f"{label} force error: max {err.max():.3e}, p99 {np.percentile(err, 99):.3e}, "
          f"max err/bar {np.max(err / bar):.3f}")
    assert np.all(err <= bar), (err.max(), np.max(err / bar))
    return err


@pytest.fixture(scope="module")
def dcm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import dcm as d

    return d


def _minimg(d, box):
    L = np.asarray(box)
    return d - np.round(d / L) * L


@pytest.mark.parametrize("n,seed", [(16000, 1), (5001, 2)])
def test_cells_bit_exact(dcm, orc, n, seed):
    s = slabgen.make_slab(n, seed=seed)
    with dcm.System(s.box, n) as sy:
        sy.set_state(s.x, s.v)
        sy.compute_forces()
        nc, start, sid = sy.cells()
        x, _, _ = sy.get_state()
    _, start_ref, sid_ref = orc.cell_list(x, s.box, nc)
    assert np.array_equal(start, start_ref)
    assert np.array_equal(sid, sid_ref)


@pytest.mark.parametrize("n,seed,rc", [(16000, 3, (3.0, 6.0)), (9001, 4, (3.0, 7.0))])
def test_detection_parity(dcm, orc, n, seed, rc):
    s = slabgen.make_slab(n, seed=seed)
    with dcm.System(s.box, n, rc_min=rc[0], rc_max=rc[1]) as sy:
        sy.set_state(s.x, s.v)
        sy.detect_interface()
        dims, B, Bs, S, D = sy.grid()
        d, rcv, cls = sy.cutoffs()
        x, _, _ = sy.get_state()
        st = sy.stats()
    det = orc.detect(x, s.box, orc.DetectParams(rc_min=rc[0], rc_max=rc[1], voxel=1.0))
    assert dims == det.dims
    assert np.array_equal(B, det.B)                   # Eq. 9, bit-exact
    assert np.array_equal(Bs, det.Bs)                 # exact integers
    assert np.array_equal(S, det.S)                   # labels bit-exact
    np.testing.assert_allclose(D, det.D, atol=1e-12, rtol=0)
    np.testing.assert_allclose(d, det.d, atol=1e-12, rtol=0)
    np.testing.assert_allclose(rcv, det.rc, rtol=1e-13, atol=0)
    assert np.array_equal(cls, det.cls)               # classes bit-exact
    assert st.cfsm_iters > 0 and st.kmeans_iters > 0


def _force_check(dcm, orc, s, prec, rc_pair=(3.0, 6.0), **kw):
    n = len(s.x)
    with dcm.System(s.box, n, precision=prec, rc_min=rc_pair[0], rc_max=rc_pair[1], **kw) as sy:
        sy.set_state(s.x, s.v)
        sy.detect_interface()
        sy.compute_forces()
        _, rc, _ = sy.cutoffs()
        x, _, f = sy.get_state()
        np_gpu = sy.pair_counts()
        nc, _, _ = sy.cells()
        pe, ke, w = sy.energy_virial()
        sy.sync()
    ref = orc.forces(x, rc, s.box, nc)
    assert np.array_equal(np_gpu, ref.npair)          # same interacting pairs
    err = np.linalg.norm(f - ref.f, axis=1)
    fmag = np.linalg.norm(ref.f, axis=1)
    return err, fmag, ref, (pe, ke, w), x, rc


@pytest.mark.parametrize("n,seed", [(16000, 5), (3333, 6)])
def test_forces_fp64(dcm, orc, n, seed):
    s = slabgen.make_slab(n, seed=seed)
    err, fmag, ref, (pe, ke, w), x, rc = _force_check(dcm, orc, s, dcm.DCM_FP64)
    assert np.all(err <= FP64_ABS + FP64_REL * fmag), err.max()
    assert pe == pytest.approx(ref.pe.sum(), rel=1e-10)
    np.testing.assert_allclose(w, ref.vir, rtol=1e-9, atol=1e-8)


@pytest.mark.parametrize("n,seed,rc_pair,cell", [(16000, 7, (3.0, 6.0), None),
                                                 (3333, 8, (3.0, 6.0), None),
                                                 (6000, 11, (3.0, 7.0), 1.0)])
def test_forces_mixed(dcm, orc, n, seed, rc_pair, cell):
    # the last case: 1-sigma cells and r_c,max = 7 give up to 225 stencil rows,
    # more than one row table of the warp walk, and wrapped rows in a small box
    s = slabgen.make_slab(n, seed=seed)
    kw = {} if cell is None else {"cell_min": cell}
    err, fmag, ref, (pe, ke, w), x, rc = _force_check(dcm, orc, s, dcm.DCM_MIXED, rc_pair, **kw)
    bar = FP64_ABS + FP64_REL * fmag
    print(f"mixed force error: max {err.max():.3e}, p99 {np.percentile(err, 99):.3e}, "
          f"max err/bar {np.max(err / bar):.3f}")
    assert np.all(err <= bar), (err.max(), np.max(err / bar))
    assert pe == pytest.approx(ref.pe.sum(), rel=1e-5)
    np.testing.assert_allclose(w, ref.vir, rtol=1e-4, atol=1e-2)


def test_forces_mixed_after_dynamics(dcm, orc):
    # a few hundred steps from the lattice start: close approaches down to
    # about 0.9 sigma, the regime the double-float close-pair path is for
    s = slabgen.make_slab(16000, seed=12)
    with dcm.System(s.box, len(s.x), precision=dcm.DCM_MIXED, skin=0.5) as sy:
        sy.set_state(s.x, s.v)
        sy.step(400)
        sy.sync()
        x, v, _ = sy.get_state()
    s.x, s.v = x, v
    err, fmag, ref, _, x, rc = _force_check(dcm, orc, s, dcm.DCM_MIXED)
    bar = FP64_ABS + FP64_REL * fmag
    print(f"mixed force error after 400 steps: max {err.max():.3e}, "
          f"p99 {np.percentile(err, 99):.3e}, max err/bar {np.max(err / bar):.3f}")
    assert np.all(err <= bar), (err.max(), np.max(err / bar))


def test_static_limit_newton3(dcm, orc):
    # r_c,min == r_c,max: DCM is the static cutoff; net force vanishes
    s = slabgen.make_slab(8000, seed=9)
    with dcm.System(s.box, len(s.x), rc_min=4.0, rc_max=4.0) as sy:
        sy.set_state(s.x, s.v)
        sy.compute_forces()
        x, _, f = sy.get_state()
        _, rc, _ = sy.cutoffs()
    assert np.all(rc == 4.0)
    fh, _ = orc.forces_static_half(x, 4.0, s.box)
    np.testing.assert_allclose(f, fh, rtol=1e-10, atol=1e-10)
    assert np.abs(f.sum(axis=0)).max() < 1e-9 * np.abs(f).sum()


@pytest.mark.parametrize("prec", [0, 1])
def test_ten_steps_positions(dcm, orc, prec):
    s = slabgen.make_slab(16000, seed=10)
    with dcm.System(s.box, len(s.x), precision=prec) as sy:
        sy.set_state(s.x, s.v)
        pe0, ke0, _ = sy.energy_virial()
        sy.step(10)
        sy.sync()
        x, v, f = sy.get_state()
        pe1, ke1, _ = sy.energy_virial()
    p = orc.RunParams(det=orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0), dt=0.005,
                      detect_every=2, cell_min=1.5)
    xr, vr, fr, rcr, ep, ek = orc.run(s.x, s.v, s.box, p, 10)
    dx = np.abs(_minimg(x - xr, s.box))
    assert dx.max() < 1e-4, dx.max()
    e0, e1 = pe0 + ke0, pe1 + ke1
    print(f"prec {prec}: |E(10)-E(0)|/|E(0)| = {abs(e1 - e0) / abs(e0):.3e} "
          f"(oracle {abs((ep[-1] + ek[-1]) - (ep[0] + ek[0])) / abs(ep[0] + ek[0]):.3e})")
    assert abs(e1 - e0) / abs(e0) < 1e-3


# ---- Verlet lists (skin > 0): the same pairs as the direct walk, always --------
WALKS = {"warp": 0, "lanes": 1}


@pytest.mark.parametrize("prec,skin,walk", [(0, 0.4, "lanes"), (1, 0.4, "warp"), (1, 0.25, "warp")])
def test_list_mode_forces(dcm, orc, prec, skin, walk):
    s = slabgen.make_slab(16000, seed=40)
    with dcm.System(s.box, len(s.x), precision=prec, skin=skin) as sy:
        sy.set_tuning([2, 1, 2, 2], 128, WALKS[walk])
        sy.set_state(s.x, s.v)
        sy.compute_forces()
        _, rc, _ = sy.cutoffs()
        x, _, f = sy.get_state()
        npair = sy.pair_counts()
        nc, _, _ = sy.cells()
        st = sy.stats()
    assert st.list_builds >= 1 and st.list_entries > 0
    ref = orc.forces(x, rc, s.box, nc)
    assert np.array_equal(npair, ref.npair)
    _force_bar(f, ref.f, f"prec {prec} lists")


# velocity-adaptive skin shares: (skin, skin_time, skin_floor)
ADAPTIVE = {"uniform": (0.3, 0.0, 0.0), "adaptive": (0.6, 0.04, 0.05)}


@pytest.mark.parametrize("prec,walk,skins", [(0, "lanes", "uniform"), (1, "warp", "uniform"),
                                             (1, "warp", "adaptive"), (0, "lanes", "adaptive")])
def test_list_mode_stays_complete_while_reused(dcm, orc, prec, walk, skins):
    # after many steps of list reuse and rebuilds the interacting pairs must
    # still be exactly those of the definition at the current positions
    s = slabgen.make_slab(9001, seed=41)
    skin, tau, floor = ADAPTIVE[skins]
    with dcm.System(s.box, len(s.x), precision=prec, skin=skin, skin_time=tau,
                    skin_floor=floor) as sy:
        sy.set_tuning([2, 1, 2, 2], 128, WALKS[walk])
        sy.set_state(s.x, s.v)
        sy.step(150)
        sy.sync()
        st = sy.stats()
        npair = sy.pair_counts()
        _, rc, _ = sy.cutoffs()
        x, _, f = sy.get_state()
        nc, _, _ = sy.cells()
    assert st.list_builds >= 3, st.list_builds          # rebuilt along the way
    assert st.list_builds < 150                          # and reused in between
    ref = orc.forces(x, rc, s.box, nc)
    assert np.array_equal(npair, ref.npair)
    _force_bar(f, ref.f, f"prec {prec} lists")


@pytest.mark.parametrize("lanes,skins", [(4, "uniform"), (8, "uniform"), (16, "uniform"),
                                         (32, "uniform"), (8, "adaptive")])
def test_list_force_kernel_on_a_reuse_step(dcm, orc, lanes, skins):
    # the forces of a step that reused its lists come from the list kernel
    # (4, 8, 16 or 32 lanes per particle): the same pairs as the definition at
    # the current positions
    s = slabgen.make_slab(12000, seed=44)
    skin, tau, floor = ADAPTIVE[skins]
    with dcm.System(s.box, len(s.x), precision=1, skin=skin + 0.1, skin_time=tau,
                    skin_floor=floor) as sy:
        sy.set_tuning([2, 1, 2, 2], 128, WALKS["warp"], lanes)
        sy.set_state(s.x, s.v)
        sy.step(3)
        for _ in range(30):
            b0 = sy.stats().list_builds
            sy.step(1)
            sy.sync()
            if sy.stats().list_builds == b0:
                break
        else:
            pytest.fail("no step reused its lists")
        npair = sy.pair_counts()
        _, rc, _ = sy.cutoffs()
        x, _, f = sy.get_state()
        nc, _, _ = sy.cells()
    ref = orc.forces(x, rc, s.box, nc)
    assert np.array_equal(npair, ref.npair)
    _force_bar(f, ref.f, "mixed lists")


def test_lanes_walk_is_the_fp64_walk(dcm):
    # DCM_MIXED always runs the warp kernels; asking it for the lanes walk
    # is refused, and the handle keeps working
    s = slabgen.make_slab(9001, seed=46)
    with dcm.System(s.box, len(s.x), precision=1, skin=0.6) as sy:
        with pytest.raises(dcm.DcmError):
            sy.set_tuning([2, 1, 2, 2], 128, WALKS["lanes"])
        sy.set_state(s.x, s.v)
        sy.step(2)
        sy.sync()


@pytest.mark.parametrize("first,then", [(8, 4), (4, 32)])
def test_list_lanes_switch_rebuilds_lists(dcm, orc, first, then):
    # a new launch shape between steps rebuilds the lists at the next step,
    # and the forces stay those of the definition
    s = slabgen.make_slab(9001, seed=46)
    with dcm.System(s.box, len(s.x), precision=1, skin=0.6, skin_time=0.04,
                    skin_floor=0.05) as sy:
        sy.set_tuning([2, 1, 2, 2], 128, WALKS["warp"], first)
        sy.set_state(s.x, s.v)
        sy.step(6)
        sy.sync()
        b0 = sy.stats().list_builds
        sy.set_tuning([2, 1, 2, 2], 128, WALKS["warp"], then)
        sy.step(1)
        sy.sync()
        assert sy.stats().list_builds == b0 + 1
        sy.step(2)
        sy.sync()
        npair = sy.pair_counts()
        _, rc, _ = sy.cutoffs()
        x, _, f = sy.get_state()
        nc, _, _ = sy.cells()
    ref = orc.forces(x, rc, s.box, nc)
    assert np.array_equal(npair, ref.npair)
    _force_bar(f, ref.f, "mixed lists")


def test_step_graph_branches_on_rebuild(dcm):
    # with the warp list kernels each captured step holds the rebuild-only
    # work in graph IF nodes: a step that reuses its lists launches fewer
    # kernels; without lists (or with the FP64 lanes kernels) there is no
    # branch
    s = slabgen.make_slab(9001, seed=43)
    counts = {}
    for prec, skin, flat in ((1, 0.3, 0), (0, 0.3, 0), (1, 0.0, 0), (1, 0.3, 1)):
        with dcm.System(s.box, len(s.x), precision=prec, skin=skin) as sy:
            sy.set_step_graph(dcm.DCM_GRAPH_FLAT if flat else dcm.DCM_GRAPH_BRANCHED)
            sy.set_state(s.x, s.v)
            sy.step(4)
            sy.sync()
            st = sy.stats()
            counts[prec, skin, flat] = (st.kernels_plain, st.kernels_plain_reuse,
                                        st.kernels_detect, st.kernels_detect_reuse)
    kp, kpr, kd, kdr = counts[1, 0.3, 0]
    assert 0 < kpr < kp and 0 < kdr < kd, counts
    assert kd - kdr == kp - kpr, counts          # the same rebuild-only work
    for key in ((0, 0.3, 0), (1, 0.0, 0), (1, 0.3, 1)):
        kp, kpr, kd, kdr = counts[key]
        assert kp == kpr > 0 and kd == kdr > kp, counts


def test_step_graph_shapes_agree(dcm):
    # the branched and the flat step graph run the same kernels on the same
    # data: bit-identical trajectories
    s = slabgen.make_slab(9001, seed=45)
    out = []
    for shape in (dcm.DCM_GRAPH_BRANCHED, dcm.DCM_GRAPH_FLAT):
        with dcm.System(s.box, len(s.x), precision=1, skin=0.3) as sy:
            sy.set_tuning([2, 1, 2, 2], 128, WALKS["warp"])
            sy.set_step_graph(shape)
            sy.set_state(s.x, s.v)
            sy.step(40)
            sy.sync()
            x, v, f = sy.get_state()
            out.append((x, v, f, sy.stats().list_builds))
    assert out[0][3] == out[1][3] >= 2
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)


def test_list_capacity_overflow_recovers(dcm, orc):
    # capacities far too small: every build overflows, the overflowing step
    # keeps its direct-walk forces, the density bound grows by 25 % per
    # build until the lists fit; forces stay exact throughout
    s = slabgen.make_slab(9001, seed=42)
    with dcm.System(s.box, len(s.x), precision=1, skin=0.3, list_density=0.05) as sy:
        sy.set_state(s.x, s.v)
        sy.step(40)
        sy.sync()
        st = sy.stats()
        npair = sy.pair_counts()
        _, rc, _ = sy.cutoffs()
        x, _, f = sy.get_state()
        nc, _, _ = sy.cells()
    assert st.list_builds >= 12, st.list_builds   # 0.05 * 1.25^k reaches ~0.8 after 13
    ref = orc.forces(x, rc, s.box, nc)
    assert np.array_equal(npair, ref.npair)
    _force_bar(f, ref.f, "mixed lists")


@pytest.mark.parametrize("prec", [0, 1])
def test_list_mode_ten_steps_match_oracle(dcm, orc, prec):
    s = slabgen.make_slab(16000, seed=10)
    with dcm.System(s.box, len(s.x), precision=prec, skin=0.4) as sy:
        sy.set_state(s.x, s.v)
        sy.step(10)
        sy.sync()
        x, _, _ = sy.get_state()
    p = orc.RunParams(det=orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0), dt=0.005,
                      detect_every=2, cell_min=1.5)
    xr, *_ = orc.run(s.x, s.v, s.box, p, 10)
    assert np.abs(_minimg(x - xr, s.box)).max() < 1e-4
