"""The library's host-side builders (csrc/strings.cpp), compiled by g++ through
tests/strings_host_shim.cpp, against the oracle and textbook results:

* occupation strings and single-excitation tables bit-exact against the
  oracle's operator-by-operator construction (strings in increasing bitmask
  order, entries (k, l, J, sign) packed as J | pair(k, l) << 20 | sign << 31);
* the cyclic Jacobi eigen-solver used by the initial guess, Davidson-Liu and
  SBCI2 subspace problems against LAPACK (numpy): eigenvalues within
  1e-13 max|lambda| (Jacobi is accurate to rounding in every eigenvalue),
  V orthonormal and A V = V Lambda to 1e-12 max|A|, including repeated
  eigenvalues and already diagonal input.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import strings as st

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers are missing")
    out = str(tmp_path_factory.mktemp("strings") / "libstrhost.so")
    csrc = os.path.join(ROOT, "paper_2603_06101_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I" + inc, "-I" + csrc,
                    os.path.join(ROOT, "tests", "strings_host_shim.cpp"), os.path.join(csrc, "strings.cpp"),
                    "-o", out], check=True)
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    L.host_string_sizes.argtypes = [ctypes.c_int, ctypes.c_int, P]
    L.host_build_strings.argtypes = [ctypes.c_int, ctypes.c_int, P, P]
    L.host_jacobi_eigh.argtypes = [ctypes.c_int, P, P, P]
    return L


def tables(lib, n, m):
    sz = np.zeros(2, dtype=np.int32)
    lib.host_string_sizes(n, m, sz.ctypes.data)
    masks = np.zeros(sz[0], dtype=np.uint32)
    links = np.zeros(int(sz[0]) * int(sz[1]), dtype=np.uint32)
    lib.host_build_strings(n, m, masks.ctypes.data, links.ctypes.data)
    return masks, links.reshape(int(sz[0]), int(sz[1]))


@pytest.mark.parametrize("n,m", [(1, 1), (5, 0), (5, 5), (6, 3), (7, 2), (8, 5), (10, 5), (12, 6), (13, 4),
                                 (14, 7)])
def test_tables_bit_exact(lib, n, m):
    masks, links = tables(lib, n, m)
    assert np.array_equal(masks.astype(np.int64), st.enumerate_strings(n, m).astype(np.int64))
    ref = st.excitation_list(n, m)
    assert links.shape == ref.shape[:2]
    J = (links & 0xFFFFF).astype(np.int64)
    pair = ((links >> 20) & 0x7FF).astype(np.int64)
    neg = (links >> 31).astype(np.int64)
    want_pair = np.array([[st.pair_index(int(k), int(l)) for k, l, _, _ in row] for row in ref],
                         dtype=np.int64).reshape(pair.shape)
    assert np.array_equal(J, ref[..., 2])
    assert np.array_equal(pair, want_pair)
    assert np.array_equal(neg, (ref[..., 3] < 0).astype(np.int64))


def eigh(lib, A):
    n = A.shape[0]
    A = np.ascontiguousarray(A, dtype=np.float64)
    w = np.zeros(n)
    V = np.zeros((n, n))
    lib.host_jacobi_eigh(n, A.ctypes.data, w.ctypes.data, V.ctypes.data)
    return w, V


def _check(lib, A):
    w, V = eigh(lib, A)
    ref = np.linalg.eigvalsh(A)
    scale = max(np.abs(ref).max(), 1e-300)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(w - ref).max() <= 1e-13 * scale * max(1, A.shape[0] / 8)
    assert np.abs(V.T @ V - np.eye(A.shape[0])).max() <= 1e-13 * max(1, A.shape[0] / 8)
    assert np.abs(A @ V - V * w).max() <= 1e-12 * max(np.abs(A).max(), 1e-300)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 24, 64])
def test_jacobi_random_symmetric(lib, n):
    rng = np.random.default_rng(100 + n)
    B = rng.standard_normal((n, n))
    _check(lib, (B + B.T) / 2)


def test_jacobi_special_spectra(lib):
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    _check(lib, Q @ np.diag([1.0, 1.0, 2.0, 2.0, 2.0, -3.0]) @ Q.T)  # repeated eigenvalues
    _check(lib, np.diag([3.0, -1.0, 2.0, 0.0]))  # diagonal: no rotation, sorted
    w, V = eigh(lib, np.zeros((3, 3)))
    assert np.array_equal(w, np.zeros(3)) and np.array_equal(V, np.eye(3))
    # a Gram matrix of nearly dependent vectors (the canonical-orthogonalisation case)
    X = rng.standard_normal((40, 5))
    X[:, 4] = X[:, 3] + 1e-7 * rng.standard_normal(40)
    _check(lib, X.T @ X)
