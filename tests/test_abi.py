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
