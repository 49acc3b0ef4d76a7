"""GB300-native hot path of the dynamic cutoff method (DCM) for Lennard-Jones
liquid/vapor slabs (Springer, arxiv 1502.03234).

The compute path is ``libdcm.so`` (hand-written CUDA for sm_103a behind a C
ABI, ``include/dcm.h``); ``paper_1502_03234_gb300.dcm`` is its ctypes binding.
Importing the package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["dcm", "slabgen"]
