"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/*.h declares (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(dcm_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libdcm():
    from paper_1502_03234_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libdcm):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(libdcm, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_1502_03234_gb300 import dcm

    assert _declared() <= set(dcm.EXPORTS) | {n for n in dir(dcm) if n.startswith("dcm_")}


def test_defaults_and_argument_errors_without_gpu(libdcm):
    # pure host paths: defaults, version, argument validation
    from paper_1502_03234_gb300 import dcm

    p = dcm.default_params()
    assert p.rc_min == 3.0 and p.rc_max == 6.0 and p.alpha == -0.5
    assert p.detect_every == 2 and p.smooth_order == 8 and p.dt == 0.005
    assert dcm.lib().dcm_version() == 1
    # invalid alpha is rejected before any device work
    bad = dcm.default_params(alpha=0.5)
    assert dcm.dcm_estimate_bytes((30.0, 30.0, 120.0), 1000, bad) == -1
    # a box narrower than 2 r_c,max is rejected
    assert dcm.dcm_estimate_bytes((11.0, 11.0, 40.0), 1000, dcm.default_params()) == -1
    est = dcm.dcm_estimate_bytes((61.56, 61.56, 246.2), 262144, dcm.default_params())
    assert 50e6 < est < 1e9


def test_component_and_cutoff_parameters_without_gpu(libdcm):
    # Section 4.2 and Fig. 12 parameters: validated and accounted for on the host
    from paper_1502_03234_gb300 import dcm

    box = (61.56, 61.56, 246.2)
    p = dcm.default_params()
    assert p.min_component_voxels == 0 and p.cutoff_fn == dcm.DCM_CUTOFF_EXP
    base = dcm.dcm_estimate_bytes(box, 262144, p)
    # the removal's buffers: parent and count per phase and a tile-local size
    # (5 int32 per voxel) on the 61 x 61 x 246 voxel grid
    cc = dcm.dcm_estimate_bytes(box, 262144, dcm.default_params(min_component_voxels=5))
    assert cc - base == 20 * 61 * 61 * 246
    lin = dcm.dcm_estimate_bytes(box, 262144, dcm.default_params(cutoff_fn=dcm.DCM_CUTOFF_LINEAR))
    assert lin == base
    assert dcm.dcm_estimate_bytes(box, 262144, dcm.default_params(min_component_voxels=-1)) == -1
    assert dcm.dcm_estimate_bytes(box, 262144, dcm.default_params(cutoff_fn=2)) == -1
    assert "cutoff_fn" in dcm.lib().dcm_last_error().decode()


def test_noalloc_sort_rejects_wrapping_cell_counts_without_gpu(libdcm):
    # three int32 cell counts whose product wraps int64 (2^21 * 2^21 * 2^22 =
    # 2^64 -> 0) or exceeds the fixed scratch are refused before any device
    # call: nothing is launched, the status is DCM_ERR_ARG
    from paper_1502_03234_gb300 import dcm

    f = dcm.lib().dcm_cell_sort_noalloc
    x = (ctypes.c_double * 3)()
    out = (ctypes.c_int32 * 4)()
    box = dcm.dcm_box(30.0, 30.0, 120.0)
    for nc in ((1 << 21, 1 << 21, 1 << 22), (1 << 20, 1 << 20, 1 << 23), (1 << 21, 1, 1),
               (1024, 1024, 2), (0x7fffffff, 0x7fffffff, 0x7fffffff)):
        ncv = (ctypes.c_int32 * 3)(*nc)
        rc = f(ctypes.cast(x, ctypes.c_void_p), 1, ctypes.byref(box), ncv,
               ctypes.cast(out, ctypes.c_void_p), ctypes.cast(out, ctypes.c_void_p), None)
        assert rc == dcm.DCM_ERR_ARG, nc
        assert "DCM_NOALLOC_MAX_CELLS" in dcm.lib().dcm_last_error().decode()


def test_noalloc_sort_binding_checks_buffers_without_gpu():
    # the binding refuses buffers of the wrong place, type, layout or length
    # (the library sees only pointers)
    torch = pytest.importorskip("torch")
    from paper_1502_03234_gb300 import dcm

    n, nc = 100, (4, 4, 16)
    box = (6.0, 6.0, 24.0)
    x = torch.zeros((n, 3), dtype=torch.float64)
    cs = torch.zeros(257, dtype=torch.int32)
    sid = torch.zeros(n, dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA"):
        dcm.dcm_cell_sort_noalloc(x, n, box, nc, cs, sid)
    with pytest.raises(ValueError, match="positive"):
        dcm.dcm_cell_sort_noalloc(x, n, box, (4, 0, 16), cs, sid)

    class FakeCuda:
        # stands in for a CUDA tensor's metadata; never reaches the library
        def __init__(self, dtype, numel, contiguous=True):
            self.is_cuda, self.dtype, self._n, self._c = True, dtype, numel, contiguous

        def numel(self):
            return self._n

        def is_contiguous(self):
            return self._c

    good = (FakeCuda(torch.float64, 3 * n), FakeCuda(torch.int32, 257), FakeCuda(torch.int32, n))
    bad_cases = [
        ((FakeCuda(torch.float32, 3 * n),) + good[1:], "float64"),
        ((FakeCuda(torch.float64, 3 * n - 1),) + good[1:], "at least"),
        ((good[0], FakeCuda(torch.int32, 256), good[2]), "at least"),
        ((good[0], FakeCuda(torch.int64, 257), good[2]), "int32"),
        ((good[0], good[1], FakeCuda(torch.int32, n - 1)), "at least"),
        ((good[0], good[1], FakeCuda(torch.int32, n, contiguous=False)), "contiguous"),
    ]
    for (xb, cb, sb), msg in bad_cases:
        with pytest.raises(ValueError, match=msg):
            dcm.dcm_cell_sort_noalloc(xb, n, box, nc, cb, sb)


def test_build_reuses_a_library_only_for_the_same_sources_and_machine(monkeypatch):
    # the rebuild check hashes the sources, flags, compiler and machine: an
    # unchanged tree keeps its library, another machine (an x86 build carried
    # to an Arm host) does not
    import platform

    from paper_1502_03234_gb300 import build

    nvcc = build._nvcc()
    a = build._fingerprint(nvcc)
    assert a == build._fingerprint(nvcc)
    monkeypatch.setattr(platform, "machine", lambda: "some-other-cpu")
    assert build._fingerprint(nvcc) != a
    import oracle

    monkeypatch.undo()
    o = oracle._fingerprint()
    monkeypatch.setattr(platform, "machine", lambda: "some-other-cpu")
    assert oracle._fingerprint() != o


def test_allocator_takes_both_functions_or_neither_without_gpu(libdcm):
    # the caller's device allocator: both callbacks or none (none = the
    # library's cudaMallocAsync / cudaFreeAsync on the handle's stream);
    # installing and removing one makes no device call
    from paper_1502_03234_gb300 import dcm

    alloc_t = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    release_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    a = alloc_t(lambda n, s, c: None)
    r = release_t(lambda p, s, c: None)
    with pytest.raises(dcm.DcmError) as e:
        dcm.dcm_set_allocator(a, None)
    assert e.value.code == dcm.DCM_ERR_ARG
    with pytest.raises(dcm.DcmError) as e:
        dcm.dcm_set_allocator(None, r)
    assert e.value.code == dcm.DCM_ERR_ARG
    dcm.dcm_set_allocator(a, r)
    dcm.use_default_allocator()
    assert dcm._ALLOCATOR is None
