"""GPU: device memory from the caller's allocator.  A handle created after
use_torch_allocator() takes every buffer from PyTorch's caching allocator on
the handle's stream (the memory shows in torch.cuda.memory_allocated while the
handle lives and is handed back when it is destroyed), and its steps are
bit-identical to those of a handle on the library's own cudaMallocAsync pool."""
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


def _run(dcm, s, **kw):
    with dcm.System(s.box, len(s.x), **kw) as sy:
        sy.set_state(s.x, s.v)
        sy.step(6)
        sy.sync()
        x, v, f = sy.get_state()
        nbytes = dcm.dcm_device_bytes(sy.h)
    return x, v, f, nbytes


@pytest.mark.parametrize("kw", [dict(precision=0), dict(precision=1, skin=0.6, skin_time=0.04,
                                                           skin_floor=0.05, segmentation=1)])
def test_torch_allocator_single_system(dcm, kw):
    import torch

    s = slabgen.make_slab(9001, seed=71)
    ref = _run(dcm, s, **kw)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    dcm.use_torch_allocator()
    try:
        with dcm.System(s.box, len(s.x), **kw) as sy:
            held = torch.cuda.memory_allocated() - base
            assert held >= dcm.dcm_device_bytes(sy.h) > 0   # every buffer from torch
            sy.set_state(s.x, s.v)
            sy.step(6)
            sy.sync()
            got = sy.get_state()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base       # all handed back
    finally:
        dcm.use_default_allocator()
    for a, b in zip(ref[:3], got):
        assert np.array_equal(a, b)


def test_torch_allocator_ensemble(dcm):
    import torch

    mem = [slabgen.make_slab(n, seed=sd) for n, sd in [(4001, 72), (6000, 73)]]
    params = [dcm.default_params(precision=dcm.DCM_MIXED) for _ in mem]
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    dcm.use_torch_allocator()
    try:
        with dcm.Ensemble([m.box for m in mem], [len(m.x) for m in mem], params) as ens:
            assert torch.cuda.memory_allocated() - base >= dcm.dcm_device_bytes(ens.h)
            for k, m in enumerate(mem):
                ens.set_system_state(k, m.x, m.v)
            ens.step(4)
            ens.sync()
            got = [ens.get_system_state(k) for k in range(len(mem))]
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        dcm.use_default_allocator()
    with dcm.Ensemble([m.box for m in mem], [len(m.x) for m in mem], params) as ens:
        for k, m in enumerate(mem):
            ens.set_system_state(k, m.x, m.v)
        ens.step(4)
        ens.sync()
        for k in range(len(mem)):
            for a, b in zip(ens.get_system_state(k), got[k]):
                assert np.array_equal(a, b)


def test_allocator_out_of_memory_releases_everything(dcm):
    # a caller's allocator that runs dry part way through dcm_create: the
    # call fails with DCM_ERR_OOM and hands back every buffer it got
    import ctypes as C

    import torch

    s = slabgen.make_slab(4001, seed=74)
    alloc_t = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    release_t = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
    calls = {"n": 0, "live": 0}

    def _alloc(nbytes, stream, ctx):
        calls["n"] += 1
        if calls["n"] > 7:
            return None
        calls["live"] += 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

    def _release(ptr, stream, ctx):
        calls["live"] -= 1
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, fr = alloc_t(_alloc), release_t(_release)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    dcm.dcm_set_allocator(fa, fr)
    try:
        with pytest.raises(dcm.DcmError) as e:
            dcm.System(s.box, len(s.x), precision=dcm.DCM_MIXED)
        assert e.value.code == dcm.DCM_ERR_OOM
    finally:
        dcm.use_default_allocator()
    torch.cuda.synchronize()
    assert calls["n"] == 8 and calls["live"] == 0
    assert torch.cuda.memory_allocated() == base
