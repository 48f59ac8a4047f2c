"""The SBCI2 pair controller (csrc/pair_ctl.h), compiled for the host by g++
(tests/pair_host_shim.cpp), against the oracle's pair step (oracle/sbci2.py)
and an independent generalized eigen-solver.

* Coefficients: for a random basis (x^a, x^b, y^a, y^b, z^a, z^b) and a
  random symmetric H, the controller's Ritz values are the two lowest
  eigenvalues of (B^T H B, B^T B) (scipy), and k V', A, C and B agree with the
  oracle's canonical orthogonalisation + eigh + pair_coefficients (k V' is the
  update x_{t+1} = k [B] V' and does not depend on the sign the eigen-solver
  gives an eigenvector); on both paths (Eq. S93; Eqs. S112-S121); with a
  repeated basis vector (the canonical orthogonalisation drops a direction;
  the coefficients are then not unique, the Ritz values are) and with an
  overlap of rank 1 (undefined, both sides).
* Decisions (Section S2.5, Eq. S127, Q7, Q8) on constructed scalars:
  convergence, each restart cause in its order of precedence, the rescaling
  factors 1/|x| and k/|x|, the cap.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import sbci2 as osb2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PH_RUN, PH_CONVERGED, PH_CAP = 0, 1, 2


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
    out = str(tmp_path_factory.mktemp("pair") / "libpairhost.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I" + inc,
                    "-I" + os.path.join(ROOT, "paper_2603_06101_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "pair_host_shim.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    L.host_pair_coef.argtypes = [P, P, ctypes.c_int, P]
    L.host_pair_coef.restype = ctypes.c_int
    L.host_pair_decide.argtypes = [P, P, P, P, P]
    return L


def _coef(lib, S, T, first):
    out = np.zeros(27)
    S = np.ascontiguousarray(S, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    ok = lib.host_pair_coef(S.ctypes.data, T.ctypes.data, int(first), out.ctypes.data)
    return ok, out


def _system(seed, n=40, dup=False):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    H = 0.5 * (A + A.T) + np.diag(np.arange(n, dtype=float))
    B = rng.standard_normal((n, 6))
    B[:, 2:4] *= 0.3  # y and z smaller than x, as in a step
    B[:, 4:6] *= 0.1
    if dup:
        B[:, 5] = B[:, 0]  # z^b = x^a: overlap of rank 5 (3 on the first path)
    return B, H


def _oracle_step(S, T, first):
    ix = [0, 1, 4, 5] if first else list(range(6))
    Ss, Ts = S[np.ix_(ix, ix)], T[np.ix_(ix, ix)]
    P = osb2.canonical_orthogonalisation(Ss)
    if P.shape[1] < 2:
        return None
    Hh = P.T @ (0.5 * (Ts + Ts.T)) @ P
    w, V = np.linalg.eigh(0.5 * (Hh + Hh.T))
    Vp = P @ V
    coef = osb2.pair_coefficients(Vp, first)
    if coef is None:
        return None
    A, Bc, C, k0, k1 = coef
    return w[:2], Vp[:, :2], A, Bc, C, np.array([k0, k1]), ix


@pytest.mark.parametrize("seed,first,dup", [(1, True, False), (2, False, False), (3, False, False),
                                             (4, True, True), (5, False, True)])
def test_pair_coefficients_against_oracle(lib, seed, first, dup):
    from scipy.linalg import eigh as geigh

    Bm, H = _system(seed, dup=dup)
    S, T = Bm.T @ Bm, Bm.T @ (H @ Bm)
    ok, out = _coef(lib, S, T, first)
    ref = _oracle_step(S, T, first)
    assert bool(ok) == (ref is not None)
    if ref is None:
        return
    w, Vp, A, Bc, C, k, ix = ref
    nb = int(out[26])
    assert nb == len(ix)
    scale = np.abs(w).max()
    assert np.abs(out[0:2] - w).max() < 1e-10 * scale
    if dup:  # the coefficients of a repeated vector are not unique: Ritz values only
        return
    gw = geigh(0.5 * (T + T.T)[np.ix_(ix, ix)], S[np.ix_(ix, ix)], eigvals_only=True)  # an independent solver
    assert np.abs(out[0:2] - gw[:2]).max() < 1e-9 * scale
    kv = out[2:4][None, :] * out[14:26].reshape(6, 2)[:nb]
    assert np.abs(kv - k[None, :] * Vp).max() < 1e-9 * np.abs(k[None, :] * Vp).max()
    assert np.abs(out[4] - A[0, 1]) < 1e-8 * max(1.0, abs(A[0, 1]))
    assert np.abs(out[5] - A[1, 0]) < 1e-8 * max(1.0, abs(A[1, 0]))
    assert np.abs(out[6:10] - Bc.ravel()).max() < 1e-8 * max(1.0, np.abs(Bc).max())
    assert np.abs(out[10:14] - C.ravel()).max() < 1e-8 * max(1.0, np.abs(C).max())


def test_rank_one_overlap_is_undefined(lib):
    rng = np.random.default_rng(7)
    v = 0.01 * rng.standard_normal(30)  # (overlap entries ~1e-3: rounding noise far below the 1e-14 cut)
    Bm = np.column_stack([v] * 6)
    H = np.diag(np.arange(30.0))
    S, T = Bm.T @ Bm, Bm.T @ (H @ Bm)
    for first in (True, False):
        ok, _ = _coef(lib, S, T, first)
        assert ok == 0 and _oracle_step(S, T, first) is None


PAR = np.array([1e-10, 1e-5, 1e-2, 1e-7, 0.1, 1.2, 1.0])


def _decide(lib, st, norms, t=3, sigma=40, max_sigma=1000, max_cycle2=10, first=0):
    ip = np.array([max_sigma, max_cycle2, t, sigma, first], dtype=np.int32)
    out = np.zeros(13)
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in (PAR, st, norms)]
    lib.host_pair_decide(args[0].ctypes.data, ip.ctypes.data, args[1].ctypes.data, args[2].ctypes.data,
                         out.ctypes.data)
    return out


def test_pair_decisions(lib):
    E0, E1 = -5.0, -4.0
    # converged: dE < eps0 and |z'| < r0 (Eq. S127)
    o = _decide(lib, [E0, E1, E0 - 1e-11, E1, 1.0, 1.0, 0.5, 0.5], [1e-12, 1e-8, 1.0, 1.0])
    assert o[0] == PH_CONVERGED and o[1] == 1
    # not converged, no cause: a plain step (t + 1, first = 0, energies taken)
    o = _decide(lib, [E0, E1, E0 - 1e-3, E1 - 1e-3, 1.0, 1.05, 0.5, 0.5], [1e-4, 1e-4, 1.0, 1.1])
    assert o[0] == PH_RUN and o[1] == 0 and o[2] == 0 and o[4] == 4 and o[3] == 0
    assert o[11] == E0 - 1e-3 and o[12] == E1 - 1e-3
    # cause a (|B_00| or |B_11| < b_th while dE < eps1) before cause b
    o = _decide(lib, [E0, E1, E0 - 1e-8, E1, 0.05, 1.0, 0.5, 1e-3], [1e-4, 1e-4, 4.0, 1.0])
    assert o[1] == 2 and o[2] == 1 and o[3] == 1 and o[4] == 0
    assert np.allclose(o[5:11], [0.5, 1.0, 0.5, 1.0, 0.05 / 2.0, 1.0])
    # cause b (min |k| < x_th1 or max |k| > x_th2)
    o = _decide(lib, [E0, E1, E0 - 1e-3, E1, 1.5, 1.0, 0.5, 0.5], [1e-4, 1e-4, 1.0, 1.0])
    assert o[1] == 3
    # cause c (|z'| > r1 after the first step of a cycle), not at t = 0
    o = _decide(lib, [E0, E1, E0 - 1e-3, E1, 1.0, 1.0, 0.5, 0.5], [4.0, 1e-4, 1.0, 1.0])
    assert o[1] == 4
    o = _decide(lib, [E0, E1, E0 - 1e-3, E1, 1.0, 1.0, 0.5, 0.5], [4.0, 1e-4, 1.0, 1.0], t=0)
    assert o[1] == 0
    # max_cycle2
    o = _decide(lib, [E0, E1, E0 - 1e-3, E1, 1.0, 1.0, 0.5, 0.5], [1e-4, 1e-4, 1.0, 1.0], t=9)
    assert o[1] == 5
    # the cap (Q8) after the step's rescaling
    o = _decide(lib, [E0, E1, E0 - 1e-3, E1, 1.0, 1.0, 0.5, 0.5], [1e-4, 1e-4, 1.0, 1.0], t=9, sigma=1000)
    assert o[0] == PH_CAP and o[2] == 1
