"""GPU parity of the small-component removal (Section 4.2, Fig. 20-21): the
CUDA union-find through the C ABI against the oracle's row-major labelling,
bit-exact on labels, on random grids (many components of every size, joined
across the periodic faces) and inside the detection, eager and in the
captured step graph, one system and an ensemble with per-system
thresholds."""
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


def planted_slab(n, seed, bubbles=6, r_bubble=2.2, r_drop=0.7, rigid=False):
    """A flat slab whose liquid has `bubbles` spherical holes; the particles
    taken out go to the vapor, so the segmentation has small vapor
    components in the liquid and small liquid components in the vapor.
    Packed (rigid False): each hole's particles in a droplet of radius
    r_drop -- overlapping particles, for detection only.  Rigid: the ball
    moved as it is to a place at least 0.9 sigma from every other particle,
    so the state can be stepped."""
    s = slabgen.make_slab(n, seed=seed)
    x = s.x.copy()
    L = np.asarray(s.box)
    rng = np.random.default_rng(seed)
    z_lo, z_hi = s.z_planes

    def dist2(p, q):
        d = p - q
        d -= np.round(d / L) * L
        return (d * d).sum(-1)

    for b in range(bubbles):
        c = np.array([rng.uniform(0, L[0]), rng.uniform(0, L[1]),
                      rng.uniform(z_lo + 4.0, z_hi - 4.0)])
        inside = np.nonzero(dist2(x, c) < r_bubble**2)[0]
        rest = np.setdiff1d(np.arange(len(x)), inside)
        for _ in range(1000):
            zc = rng.uniform(3.0, z_lo - 5.0) if b % 2 == 0 else rng.uniform(z_hi + 5.0, L[2] - 3.0)
            drop = np.array([rng.uniform(0, L[0]), rng.uniform(0, L[1]), zc])
            if rigid:
                moved = np.mod(x[inside] - c + drop, L)
                near = dist2(moved[:, None, :], x[rest][None, :, :]).min() if len(rest) else 9.0
                if near >= 0.81:
                    x[inside] = moved
                    break
            else:
                u = rng.normal(size=(inside.size, 3))
                u *= (r_drop * rng.random(inside.size) ** (1 / 3) / np.linalg.norm(u, axis=1))[:, None]
                x[inside] = np.mod(drop + u, L)
                break
        else:
            raise RuntimeError("no free place for a rigid ball")
    return s, x


def random_labels(dims, p, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(int(np.prod(dims))) >= p).astype(np.uint8)   # P(liquid) = p


@pytest.mark.parametrize("p", [0.2, 0.45, 0.55, 0.8])
@pytest.mark.parametrize("m", [1, 2, 5, 40])
def test_random_grids_match_oracle(dcm, orc, p, m):
    s = slabgen.make_slab(6000, seed=31)
    with dcm.System(s.box, len(s.x)) as sy:
        sy.set_state(s.x, s.v)
        sy.detect_interface()
        dims = sy.grid()[0]
        S = random_labels(dims, p, seed=int(100 * p) + m)
        out, fl = sy.remove_small_components(S, m)
        ref, fref = orc.remove_small_components(dims, S, m)
        assert np.array_equal(out, ref)
        assert fl == fref
        if m == 1:
            assert fl == 0
        # the handle's own labels are untouched
        assert np.array_equal(sy.grid()[3], orc.detect(sy.get_state()[0], s.box,
                                                        orc.DetectParams()).S)


def test_device_labels_and_order_case(dcm, orc):
    torch = pytest.importorskip("torch")
    s = slabgen.make_slab(6000, seed=32)
    with dcm.System(s.box, len(s.x), min_component_voxels=3) as sy:
        sy.set_state(s.x, s.v)
        sy.detect_interface()
        dims = sy.grid()[0]
        nx, ny, nz = dims
        # a 3x3x3 liquid shell around a one-voxel vapor cavity in an all-vapor
        # grid: threshold 27 removes the shell first (liquid before vapor),
        # 26 keeps it and fills the cavity
        S = np.ones(nx * ny * nz, np.uint8)
        for z in range(3, 6):
            for y in range(3, 6):
                S[3 + nx * (y + ny * z): 6 + nx * (y + ny * z)] = 0
        S[4 + nx * (4 + ny * 4)] = 1
        for m, flips in ((27, 26), (26, 1)):
            t = torch.from_numpy(S.copy()).cuda()
            _, fl = sy.remove_small_components(t, m)
            ref, fref = orc.remove_small_components(dims, S, m)
            assert fl == fref == flips
            assert np.array_equal(t.cpu().numpy(), ref)
        # whole-grid phases: all liquid with a threshold above the grid size
        # turns vapor, then back (the vapor grid is one small component)
        for fill in (0, 1):
            A = np.full(nx * ny * nz, fill, np.uint8)
            out, fl = sy.remove_small_components(A, A.size + 1)
            ref, fref = orc.remove_small_components(dims, A, A.size + 1)
            assert np.array_equal(out, ref) and fl == fref


@pytest.mark.parametrize("m", [16, 40])
def test_detection_with_removal_matches_oracle(dcm, orc, m):
    # the droplets come out as liquid components of 14-18 voxels: 16 removes
    # some (a component of exactly 16 stays), 40 all of them
    s, x = planted_slab(16000, seed=33)
    with dcm.System(s.box, len(x), min_component_voxels=m) as sy:
        sy.set_state(x, s.v)
        sy.detect_interface()
        dims, B, Bs, S, D = sy.grid()
        d, rcv, cls = sy.cutoffs()
        xs, _, _ = sy.get_state()
        st = sy.stats()
    det = orc.detect(xs, s.box, orc.DetectParams(min_component_voxels=m))
    plain = orc.detect(xs, s.box, orc.DetectParams())
    assert np.array_equal(B, det.B) and np.array_equal(Bs, det.Bs)
    assert np.array_equal(S, det.S)                      # labels bit-exact
    np.testing.assert_allclose(D, det.D, atol=1e-12, rtol=0)
    np.testing.assert_allclose(d, det.d, atol=1e-12, rtol=0)
    np.testing.assert_allclose(rcv, det.rc, rtol=1e-13, atol=0)
    assert np.array_equal(cls, det.cls)
    changed = int((det.S != plain.S).sum())
    assert st.cc_flipped == changed > 0                   # the planted components were removed
    if m == 40:
        # no component below 40 voxels is left in either phase
        for phase in (0, 1):
            lab, nc = orc.label_components(dims, S, phase)
            assert np.bincount(lab[lab >= 0], minlength=nc).min() >= 40


def test_captured_step_graph_removes_components(dcm, orc):
    # detection inside dcm_step (captured graph, every 2nd step): the labels
    # after the step are those of the oracle's detection at the step's
    # positions, with the removal
    s, x = planted_slab(16000, seed=34, r_bubble=2.6, rigid=True)
    with dcm.System(s.box, len(x), min_component_voxels=40, precision=1, skin=0.5) as sy:
        sy.set_state(x, 0.0 * s.v)
        sy.step(2)
        dims, _, _, S, _ = sy.grid()
        xs, _, _ = sy.get_state()
        st = sy.stats()
    det = orc.detect(xs, s.box, orc.DetectParams(min_component_voxels=40))
    assert np.array_equal(S, det.S)
    assert st.cc_flipped == int((det.S != orc.detect(xs, s.box, orc.DetectParams()).S).sum())


def test_ensemble_thresholds_per_system(dcm, orc):
    mem = [planted_slab(9000, seed=35), planted_slab(12000, seed=36), planted_slab(7000, seed=37)]
    thr = [40, 0, 5]
    params = [dcm.default_params(min_component_voxels=m) for m in thr]
    with dcm.Ensemble([s.box for s, _ in mem], [len(x) for _, x in mem], params) as ens:
        for k, (s, x) in enumerate(mem):
            ens.set_system_state(k, x, s.v)
        ens.detect_interface()
        d, rcv, cls = ens.cutoffs()
        ranges = [dcm.dcm_system_range(ens.h, k) for k in range(len(mem))]
        states = [ens.get_system_state(k)[0] for k in range(len(mem))]
    for k, ((s, _), m) in enumerate(zip(mem, thr)):
        a, c = ranges[k]
        det = orc.detect(states[k], s.box, orc.DetectParams(min_component_voxels=m))
        np.testing.assert_allclose(d[a:a + c], det.d, atol=1e-12, rtol=0)
        np.testing.assert_allclose(rcv[a:a + c], det.rc, rtol=1e-13, atol=0)
        assert np.array_equal(cls[a:a + c], det.cls), k


def test_negative_threshold_is_rejected(dcm):
    s = slabgen.make_slab(4000, seed=38)
    with pytest.raises(dcm.DcmError) as e:
        dcm.System(s.box, len(s.x), min_component_voxels=-1)
    assert e.value.code == dcm.DCM_ERR_ARG
    with dcm.System(s.box, len(s.x)) as sy:
        nv = int(np.prod(sy.grid()[0]))
        with pytest.raises(dcm.DcmError) as e:
            sy.remove_small_components(np.zeros(nv, np.uint8), -2)
        assert e.value.code == dcm.DCM_ERR_ARG
        with pytest.raises(ValueError):          # a grid of the wrong size never reaches the library
            sy.remove_small_components(np.zeros(nv - 1, np.uint8), 5)
