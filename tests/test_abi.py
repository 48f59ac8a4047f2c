"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sbci_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2603_06101_gb300 import build, sbci

    if not os.path.exists(sbci.LIB_PATH):
        build.build()
    return sbci.LIB_PATH


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 13
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib_path):
    from paper_2603_06101_gb300 import sbci

    assert set(sbci.EXPORTS) <= _declared()


def test_host_only_calls_without_gpu(lib_path):
    """Entry points that need no device work behave on a CPU-only host."""
    from paper_2603_06101_gb300 import sbci

    lib = sbci.load()
    p = sbci.params()
    assert p.eps0 == 1e-10 and p.r0 == 1e-5 and p.max_cycle == 20
    assert lib.sbci_params_init(None) == sbci.SBCI_ERR_INVALID
    assert b"NULL" in lib.sbci_last_error()
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert lib.sbci_init_integrals(ctypes.byref(h), 17, 1, 1, None, None, 0.0, None) == sbci.SBCI_ERR_INVALID
    import numpy as np

    h1 = np.zeros((2, 2))
    eri = np.zeros((2, 2, 2, 2))
    h1[0, 0] = float("nan")
    st = lib.sbci_init_integrals(ctypes.byref(h), 2, 1, 1, h1.ctypes.data_as(ctypes.c_void_p),
                                 eri.ctypes.data_as(ctypes.c_void_p), 0.0, None)
    assert st == sbci.SBCI_ERR_NUMERIC
    h1[0, 0] = 0.0
    h1[0, 1] = 1.0  # not symmetric
    st = lib.sbci_init_integrals(ctypes.byref(h), 2, 1, 1, h1.ctypes.data_as(ctypes.c_void_p),
                                 eri.ctypes.data_as(ctypes.c_void_p), 0.0, None)
    assert st == sbci.SBCI_ERR_INVALID
