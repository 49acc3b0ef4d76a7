"""GPU failure detection without a GPU fault: every device-side check sets a
flag the host reads; bounded waits give up and report; the handle stays
usable afterwards."""
import ctypes as C

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


def test_non_finite_velocity_is_flagged(dcm):
    s = slabgen.make_slab(4000, seed=21)
    v = s.v.copy()
    v[17, 1] = np.nan
    with dcm.System(s.box, len(s.x)) as sy:
        sy.set_state(s.x, v)
        sy.step(2)
        with pytest.raises(dcm.DcmError) as e:
            sy.sync()
        assert e.value.code == dcm.DCM_ERR_DEVICE_CHECK
        # flag cleared on report; a clean state runs again
        sy.set_state(s.x, s.v)
        sy.step(2)
        sy.sync()


def test_cfsm_iteration_cap_reports_not_converged(dcm):
    s = slabgen.make_slab(8000, seed=22)
    with dcm.System(s.box, len(s.x), cfsm_iter_max=1) as sy:
        sy.set_state(s.x, s.v)
        sy.detect_interface()
        with pytest.raises(dcm.DcmError) as e:
            sy.sync()
        assert e.value.code == dcm.DCM_ERR_NOT_CONVERGED


def test_bounded_wait_gives_up_and_handle_survives(dcm):
    s = slabgen.make_slab(4000, seed=23)
    with dcm.System(s.box, len(s.x)) as sy:
        rc = dcm.lib().dcm_check_bounded_wait(sy.h)
        assert rc == dcm.DCM_ERR_DEVICE_CHECK
        assert b"flags 0x4" in dcm.lib().dcm_last_error()
        sy.set_state(s.x, s.v)
        sy.compute_forces()
        sy.sync()


def test_host_side_argument_errors(dcm):
    s = slabgen.make_slab(4000, seed=24)
    with pytest.raises(dcm.DcmError) as e:
        dcm.System((11.0, 11.0, 44.0), 1000)
    assert e.value.code == dcm.DCM_ERR_BOX_TOO_SMALL
    with dcm.System(s.box, len(s.x)) as sy:
        with pytest.raises(dcm.DcmError) as e:
            sy.step(1)
        assert e.value.code == dcm.DCM_ERR_STATE
        with pytest.raises(dcm.DcmError) as e:
            sy.set_cutoffs(np.full(len(s.x), 9.0))
        assert e.value.code == dcm.DCM_ERR_ARG
