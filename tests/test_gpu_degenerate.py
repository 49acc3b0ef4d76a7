"""GPU parity on the degenerate inputs of the method: a box with no
interface (all vapor: dilute gas; all liquid: a dense lattice filling the
box), the smallest box the default stencil allows, and an empty system.
Labels, classes and pair counts bit-exact, distances within 1e-12, forces
within the mixed-precision bound, against the FP64 oracle."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen

pytestmark = pytest.mark.gpu

FP64_REL, FP64_ABS = 1e-5, 1e-6


@pytest.fixture(scope="module")
def dcm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import dcm as d

    return d


def _fcc(cells, a, jitter, seed):
    rng = np.random.default_rng(seed)
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(np.arange(cells), np.arange(cells), np.arange(cells),
                             indexing="ij"), -1).reshape(-1, 1, 3)
    x = ((g + base[None]) * a).reshape(-1, 3)
    x += rng.uniform(-jitter, jitter, x.shape)
    box = (cells * a,) * 3
    return np.mod(x, box[0]), box


def _check(dcm, orc, x, v, box, prec, skin=0.0):
    n = len(x)
    with dcm.System(box, n, precision=prec, skin=skin) as sy:
        sy.set_state(x, v)
        sy.detect_interface()
        sy.compute_forces()
        xg, _, f = sy.get_state()
        dims, B, Bs, S, D = sy.grid()
        d, rc, cls = sy.cutoffs()
        npair = sy.pair_counts()
        nc, _, _ = sy.cells()
    det = orc.detect(xg, box, orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0))
    assert np.array_equal(B, det.B)
    assert np.array_equal(S, det.S)
    np.testing.assert_allclose(D, det.D, atol=1e-12, rtol=0)
    np.testing.assert_allclose(d, det.d, atol=1e-12, rtol=0)
    assert np.array_equal(cls, det.cls)
    ref = orc.forces(xg, rc, box, nc)
    assert np.array_equal(npair, ref.npair)
    err = np.linalg.norm(f - ref.f, axis=1)
    fmag = np.linalg.norm(ref.f, axis=1)
    assert np.all(err <= FP64_ABS + FP64_REL * fmag), (err.max(), prec)
    return S


@pytest.mark.parametrize("prec", [0, 1])
def test_all_vapor_box(dcm, orc, prec):
    box = (22.0, 22.0, 22.0)
    x, v = slabgen.make_gas(600, box, seed=51)
    _check(dcm, orc, x, v, box, prec)


@pytest.mark.parametrize("prec,skin", [(0, 0.0), (1, 0.0), (1, 0.5)])
def test_all_liquid_box(dcm, orc, prec, skin):
    x, box = _fcc(10, slabgen.fcc_edge(0.8), 0.05, seed=52)       # 4000 atoms, no vapor
    rng = np.random.default_rng(53)
    v = rng.normal(0.0, np.sqrt(0.7), x.shape)
    _check(dcm, orc, x, v, box, prec, skin)


@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
def test_lattice_refined_in_place(dcm, orc, lanes):
    # a nearly perfect lattice at rest under one cutoff (r_c,min = r_c,max:
    # the detection of a box without interface then changes nothing): every
    # net force is close to zero, so on a step that reuses its Verlet lists
    # nearly every particle falls under the refinement threshold and the list
    # kernel evaluates it again in place (each warp takes its groups'
    # particles one after another); the bar 1e-6 + 1e-5 |F| is then close to
    # its absolute floor for all of them
    x, box = _fcc(10, slabgen.fcc_edge(0.8), 1e-3, seed=61)        # 4000 atoms
    n = len(x)
    with dcm.System(box, n, precision=1, skin=0.5, rc_min=3.0, rc_max=3.0) as sy:
        sy.set_tuning([2, 1, 2, 2], 128, 0, lanes)
        sy.set_state(x, np.zeros_like(x))
        sy.step(2)
        for _ in range(20):
            b0 = sy.stats().list_builds
            sy.step(1)
            sy.sync()
            if sy.stats().list_builds == b0:
                break
        else:
            pytest.fail("no step reused its lists")
        refined = sy.stats().refined
        npair = sy.pair_counts()
        _, rc, _ = sy.cutoffs()
        xg, _, f = sy.get_state()
        nc, _, _ = sy.cells()
    ref = orc.forces(xg, rc, box, nc)
    fmag = np.linalg.norm(ref.f, axis=1)
    assert np.mean(fmag < 0.5) > 0.9                 # the lattice is nearly at rest
    assert refined >= int(np.sum(fmag < 0.45))       # all of those were refined
    assert np.array_equal(npair, ref.npair)
    err = np.linalg.norm(f - ref.f, axis=1)
    assert np.all(err <= FP64_ABS + FP64_REL * fmag), (err.max(), lanes)


@pytest.mark.parametrize("edge,skin", [(13.6, 0.0), (16.6, 0.5)])
def test_smallest_box_for_the_stencil(dcm, orc, edge, skin):
    # the cell stencil must not wrap onto itself: 2 s_max + 1 <= cells per
    # edge, with s_max the stencil of r_c,max (+ skin with Verlet lists):
    # 9 cells of 1.5 sigma for r_c,max = 6, 11 for 6.5
    s = slabgen.make_slab(2048, seed=54, min_edge=edge)
    _check(dcm, orc, s.x, s.v, s.box, 1, skin)


def test_empty_system_is_rejected(dcm):
    with pytest.raises(dcm.DcmError) as e:
        dcm.System((20.0, 20.0, 80.0), 0)
    assert e.value.code == dcm.DCM_ERR_ARG


def test_skin_share_parameters(dcm):
    # the adaptive-share parameters only matter with lists: accepted with
    # skin 0, rejected when the floor exceeds half the skin
    s = slabgen.make_slab(4000, seed=53)
    with dcm.System(s.box, len(s.x), precision=1, skin=0.0, skin_time=0.06, skin_floor=0.07):
        pass
    with pytest.raises(dcm.DcmError) as e:
        dcm.System(s.box, len(s.x), precision=1, skin=0.4, skin_time=0.06, skin_floor=0.3)
    assert e.value.code == dcm.DCM_ERR_ARG
    with pytest.raises(dcm.DcmError) as e:
        dcm.System(s.box, len(s.x), precision=1, skin=0.4, skin_time=-1.0)
    assert e.value.code == dcm.DCM_ERR_ARG



def test_list_storage_above_int32_offsets_is_rejected(dcm):
    # list offsets are int32: storage for n x min((4/3) pi (6 + 0.7)^3,
    # 4 pi (3 + 0.7)^3) = 637 n entries passes 2^31 at n = 3.38 M
    n = 3_400_000
    L = (n / 0.32 / 4.0) ** (1.0 / 3.0)          # slab-shaped box, mean density 0.32
    with pytest.raises(dcm.DcmError) as e:
        dcm.System((L, L, 4.0 * L), n, precision=1, skin=0.7)
    assert e.value.code == dcm.DCM_ERR_ARG
    assert "2^31" in str(e.value)
