"""The library's host-side builders (csrc/strings.cpp), compiled by g++ through
tests/strings_host_shim.cpp, against the oracle and textbook results:

* occupation strings and single-excitation tables bit-exact against the
  oracle's operator-by-operator construction (strings in increasing bitmask
  order, entries (k, l, J, sign) packed as J | pair(k, l) << 20 | sign << 31);
* the cyclic Jacobi eigen-solver used by the initial guess, Davidson-Liu and
  SBCI2 subspace problems against LAPACK (numpy): eigenvalues within
  1e-13 max|lambda| (Jacobi is accurate to rounding in every eigenvalue),
  V orthonormal and A V = V Lambda to 1e-12 max|A|, including repeated
  eigenvalues and already diagonal input;
* the density-fitted factor W = F M F^T of the packed operator (reading L1):
  rank naux + 2 on density-fitted integrals and on stretched chains whose
  distant pair densities vanish, F M F^T equal to W (the operator as the
  context builds it, written out here from its definition) within 1e-12 of
  max|W|, the full form kept for full-rank integrals (H12 at 1.2 A) and for
  a pair matrix that is not positive semi-definite.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import strings as st
from paper_2603_06101_gb300 import inputs

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
    L.host_df_factor.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, P, P, ctypes.c_longlong]
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


def _packed_operator(I):
    """Pair matrix V = (ij|kl), kappa_ij = h_ij - 1/2 sum_m (im|mj), delta and
    W = 1/2 V + (kappa delta^T + delta kappa^T) / (2N) over packed pairs i >= j."""
    n = I.h1.shape[0]
    eri = I.eri.reshape(n, n, n, n)
    pairs = [(i, j) for i in range(n) for j in range(i + 1)]
    V = np.array([[eri[i, j, k, l] for (k, l) in pairs] for (i, j) in pairs])
    kmat = I.h1 - 0.5 * np.einsum("immj->ij", eri)
    kap = np.array([kmat[i, j] for (i, j) in pairs])
    dl = np.array([1.0 if i == j else 0.0 for (i, j) in pairs])
    N = I.nalpha + I.nbeta
    return V, kap, dl, N, 0.5 * V + (np.outer(kap, dl) + np.outer(dl, kap)) / (2 * N)


def df_factor(lib, V, kap, dl, N):
    npair = V.shape[0]
    V = np.ascontiguousarray(V, dtype=np.float64)
    kap = np.ascontiguousarray(kap, dtype=np.float64)
    dl = np.ascontiguousarray(dl, dtype=np.float64)
    cap = npair * (npair + 2)
    Ut = np.zeros(cap)
    UL = np.zeros(cap)
    rr = lib.host_df_factor(npair, V.ctypes.data, kap.ctypes.data, dl.ctypes.data, int(N), Ut.ctypes.data,
                            UL.ctypes.data, cap)
    if rr == 0:
        return 0, None, None
    return rr, Ut[:rr * npair].reshape(rr, npair), UL[:rr * npair].reshape(npair, rr)


@pytest.mark.parametrize("make,rank", [(lambda: inputs.random_df(14, 7, 3, 2), 42 + 2),
                                       (lambda: inputs.random_df(14, 3, 7, 7, naux=20), 20 + 2),
                                       (lambda: inputs.h_chain(12, 2.959854009887736), None)])
def test_df_factor_reproduces_the_operator(lib, make, rank):
    I = make()
    V, kap, dl, N, W = _packed_operator(I)
    rr, Ut, UL = df_factor(lib, V, kap, dl, N)
    assert rr > 0 and 2 * rr < 0.9 * V.shape[0]
    if rank is not None:
        assert rr == rank
    assert np.abs(UL @ Ut - W).max() <= 1e-12 * np.abs(W).max()
    # Ut rows: the Cholesky vectors, then kappa and delta
    assert np.array_equal(Ut[-2], kap) and np.array_equal(Ut[-1], dl)


def test_df_factor_keeps_the_full_form(lib):
    # full-rank integrals: the factorisation stops once 2 (r + 2) reaches 0.9 npair
    V, kap, dl, N, _ = _packed_operator(inputs.h_chain(12, 1.2))
    assert df_factor(lib, V, kap, dl, N)[0] == 0
    # a pair matrix with a negative direction: the remainder check rejects it
    I = inputs.random_df(12, 5, 3, 3, naux=6)
    V, kap, dl, N, _ = _packed_operator(I)
    u = np.random.default_rng(1).standard_normal(V.shape[0])
    Vbad = V - 0.5 * np.abs(V).max() * np.outer(u, u) / (u @ u)
    assert np.linalg.eigvalsh(Vbad).min() < 0
    assert df_factor(lib, Vbad, kap, dl, N)[0] == 0
    # all-zero integrals: nothing to factor
    assert df_factor(lib, np.zeros_like(V), kap, dl, N)[0] == 0
