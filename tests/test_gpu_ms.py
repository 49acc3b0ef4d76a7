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
