"""GPU: the allocation-free link-cell sort (dcm_cell_sort_noalloc), for callers
that cannot allocate device memory when they need a cell list, returns the
same cell list as the handle-based path, on two calls in a row (the shared
scratch array keeps the previous call's contents, so the second call checks
that it starts clean)."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen

pytestmark = pytest.mark.gpu


def test_noalloc_cell_sort_matches_handle_path_on_two_calls():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import dcm

    xd = None
    for n, seed in [(16000, 31), (9001, 32)]:
        s = slabgen.make_slab(n, seed=seed)
        with dcm.System(s.box, n) as sy:
            sy.set_state(s.x, s.v)
            sy.compute_forces()
            nc, start_ref, sid_ref = sy.cells()
            x, _, _ = sy.get_state()          # positions wrapped into the box, AoS
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        ncell = int(np.prod(nc))
        cs = torch.full((ncell + 1,), -1, dtype=torch.int32, device="cuda")
        sid = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        dcm.dcm_cell_sort_noalloc(xd, n, s.box, nc, cs, sid)
        torch.cuda.synchronize()
        assert np.array_equal(cs.cpu().numpy(), start_ref)      # bit-exact
        assert np.array_equal(sid.cpu().numpy(), sid_ref)

    # sizes beyond the fixed scratch are rejected before any launch
    big = dcm.lib().dcm_cell_sort_noalloc
    with pytest.raises(dcm.DcmError) as e:
        dcm.dcm_cell_sort_noalloc(xd, (1 << 19) + 1, s.box, nc, cs, sid)
    assert e.value.code == dcm.DCM_ERR_ARG
    with pytest.raises(dcm.DcmError) as e:
        dcm.dcm_cell_sort_noalloc(xd, n, s.box, (1024, 1024, 2), cs, sid)
    assert e.value.code == dcm.DCM_ERR_ARG
    # cell counts whose product wraps a 64-bit integer to 0
    with pytest.raises(dcm.DcmError) as e:
        dcm.dcm_cell_sort_noalloc(xd, n, s.box, (1 << 21, 1 << 21, 1 << 22), cs, sid)
    assert e.value.code == dcm.DCM_ERR_ARG
    del big
