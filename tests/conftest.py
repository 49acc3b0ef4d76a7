"""Shared test configuration.

Markers: ``gpu`` -- needs a CUDA device and the built ``libdcm.so``; the CPU
suite runs with ``-m "not gpu"``.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (CUDA) device and libdcm.so")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    oracle.set_threads(min(8, os.cpu_count() or 1))
    return oracle
