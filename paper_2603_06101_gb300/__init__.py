"""GB300-native SBCI: the FCI sigma build and the SBCI1 solver as CUDA for sm_103a.

The compute path lives in ``libsbci.so`` (C ABI in ``include/sbci.h``); the
Python module ``paper_2603_06101_gb300.sbci`` is a ctypes binding with the same
entry-point names.  ``inputs`` holds the seeded synthetic workloads.
"""
__all__ = ["inputs", "sbci", "build"]
