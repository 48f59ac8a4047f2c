"""The device controller's decision logic (csrc/ctl.h), compiled for the host
by g++ (tests/ctl_host_shim.cpp), against the oracle SBCI1.

* Subspace solves: every first-step (Eqs. S10-S24) and later-step (Eqs.
  S33-S55) problem of oracle runs, given as the 13 dot products the GPU
  reduces, must give the oracle's E_{t+1}, |k|, b, c and its second Ritz pair
  (S1.4).  The controller solves in FP32 Jacobi + one FP64 Rayleigh-quotient
  step for the lowest pair and keeps the second pair in FP32; tolerances:
  E_{t+1} 1e-12 relative to max|V|; |k| and the update x_{t+1} = x + b y_{t+1}
  1e-9 relative (the eigenvector of a 2x2/3x3 problem moves by eps |V| / gap);
  y_{t+1} = y - c z 1e-8 relative: c is a ratio of two eigenvector
  combinations whose denominator cancels when |c| is large (3e-9 seen at
  |c| = 2064), vectors compared in the metric of the step's overlap matrix;
  E2 1e-5 relative to max|V| and the second Ritz vector 1e-6 |V| / gap
  (FP32, gap = E2 - E_{t+1}; at least 1e-5).
* End-of-step decisions: the oracle's dE, |z'|, b, k and t give the same
  convergence (Eq. S61) and restart causes (Eqs. S62a-c, max_cycle).
* Mixed-precision stages: the switch at the end of the low-precision stage,
  the re-sync windows and the FP64 fallback of the refinement stage, and the
  caps, on synthetic states.
* Degenerate steps on constructed dot products: Gram-Schmidt breakdowns of y
  and z (reading R7) and undefined later-step coefficients (reading R15).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import sbci as osb
from oracle import sigma as sg
from oracle import slater_condon as sc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H_RUN, H_CONVERGED, H_SWITCH, H_CAP = 0, 1, 2, 3
FP64, TF32X3 = 0, 1
EVENT = {"": 0, "converged": 1, "restart:a": 2, "restart:b": 3, "restart:c": 4, "restart:max": 5, "undef": 8}


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def ctl(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers are missing")
    out = str(tmp_path_factory.mktemp("ctl") / "libctlhost.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I" + inc,
                    "-I" + os.path.join(ROOT, "paper_2603_06101_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "ctl_host_shim.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    lib.host_ctl_solve.argtypes = [D, ctypes.c_int, ctypes.c_double, ctypes.c_double, D]
    lib.host_ctl_solve.restype = ctypes.c_int
    lib.host_ctl_check.argtypes = [D, I, D, I]
    lib.host_ctl_check.restype = ctypes.c_int
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def solve(lib, dots, first, sx, gs_tol=1e-14):
    out = np.zeros(12)
    d = np.ascontiguousarray(dots, dtype=np.float64)
    halt = lib.host_ctl_solve(_dptr(d), int(first), float(sx), float(gs_tol), _dptr(out))
    return halt, out


def check(lib, *, E_prev, E_new, b=1.0, c=0.0, k=1.0, dz=1e-3, t=1, alpha=0, stage=1, prec=FP64,
          user_prec=FP64, n_sigma=10, n_stage1=0, n_sync=0, max_sigma=1000, refine_max_sigma=300,
          p=osb.SBCIParams(), mixed_eps=1e-8, mixed_r=1e-4, nxy=0.0):
    pr = np.array([p.eps0, p.r0, p.b_th, p.eps1, p.x_th1, p.x_th2, p.r1, mixed_eps, mixed_r, p.gs_tol,
                   E_prev, E_new, b, c, k], dtype=np.float64)
    ip = np.array([p.max_cycle, max_sigma, refine_max_sigma, user_prec, prec, stage, alpha, t, n_sigma,
                   n_stage1, n_sync], dtype=np.int32)
    dots = np.array([1.0, nxy, 1.0, dz * dz], dtype=np.float64)
    out = np.zeros(7, dtype=np.int32)
    halt = lib.host_ctl_check(_dptr(pr), _iptr(ip), _dptr(dots), _iptr(out))
    return halt, out


class Recording(osb.SBCI1):
    """The oracle SBCI1, recording each subspace problem as the 13 dots the
    device reduces (slot order S_NXX .. S_HZZ) with the oracle's answer."""

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.calls = []

    def _first_step(self, x, X, z, Z):
        out = super()._first_step(x, X, z, Z)
        d = [x @ x, 0.0, 0.0, x @ X, 0.0, 0.0, 0.0, x @ z, 0.0, z @ z, x @ Z, 0.0, z @ Z]
        self.calls.append(("first", np.array(d), out))
        return out

    def _later_step(self, x, X, y, Y, z, Z):
        out = super()._later_step(x, X, y, Y, z, Z)
        d = [x @ x, x @ y, y @ y, x @ X, x @ Y, y @ Y, 0.0, x @ z, y @ z, z @ z, x @ Z, y @ Z, z @ Z]
        self.calls.append(("later", np.array(d), out))
        return out


def _overlap(d):
    Nxx, Nxy, Nyy, Nxz, Nyz, Nzz = d[0], d[1], d[2], d[7], d[8], d[9]
    return np.array([[Nxx, Nxy, Nxz], [Nxy, Nyy, Nyz], [Nxz, Nyz, Nzz]])


def _nerr(a, b, N):
    """|a - b| / |b| for coefficient vectors in the basis (x, y, z), N its overlap."""
    den = np.sqrt(max(b @ N @ b, 0.0))
    return np.sqrt(max((a - b) @ N @ (a - b), 0.0)) / den if den > 0 else float(np.abs(a - b).max())


def _vmax(d, first):
    """max |V| of the subspace problem, the scale of E and E2."""
    return max(abs(d[3]), abs(d[5]), abs(d[12]) / max(d[9], 1e-300)) if not first else \
        max(abs(d[3]) / d[0], abs(d[12]) / max(d[9], 1e-300))


def _runs():
    runs = []
    for n, R, k in ((6, 1.0, 4), (6, 2.4, 2), (8, 1.3, 2)):
        I = inputs.h_chain(n, R)
        m = n // 2
        sig = sg.StringSigma(I.h1, I.eri, m, m)
        Dg = sc.diagonal_by_occupation(I.h1, I.eri, m, m)
        run = Recording(sig.apply, Dg, (sig.Na, sig.Nb))
        res = run.solve(k)
        assert all(r.converged for r in res)
        runs.append(((n, R), run))
    return runs


@pytest.fixture(scope="module")
def runs():
    return _runs()


def test_subspace_solves_match_the_oracle(ctl, runs):
    ncmp = {"first": 0, "later": 0, "c0": 0}
    for key, run in runs:
        calls = run.calls
        i = 0
        while i < len(calls):
            kind, d, (E, b, c, k, sec) = calls[i]
            first = kind == "first"
            sx = 1.0 / np.sqrt(d[0])
            halt, o = solve(ctl, d, first, sx)
            assert halt == H_RUN
            if not first and not np.all(np.isfinite([E, b, c, k])):
                # reading R15: the device takes the first-step path at once
                assert o[11] == 8
                i += 1
                kind, d, (E, b, c, k, sec) = calls[i]
                assert kind == "first"
                first = True
            else:
                assert o[11] == 0
            scale = _vmax(d, first)
            Nm = _overlap(d)
            assert abs(o[0] - E) <= 1e-12 * scale, (key, i)
            # the update in the basis (x, y, z): x_{t+1} = x + b y_{t+1} and
            # y_{t+1} = y - c z (first step: x_0 = sx x, b = 1, y = 0)
            if first:
                ad, ao = np.array([sx, 0.0, -o[2]]), np.array([sx, 0.0, -c])
                yd, yo = np.array([0.0, 0.0, -o[2]]), np.array([0.0, 0.0, -c])
            else:
                ad, ao = np.array([1.0, o[1], -o[1] * o[2]]), np.array([1.0, b, -b * c])
                yd, yo = np.array([0.0, 1.0, -o[2]]), np.array([0.0, 1.0, -c])
            assert o[1] == 1.0 if first else True
            assert _nerr(ad, ao, Nm) <= 1e-9, (key, i)
            assert _nerr(yd, yo, Nm) <= 1e-8, (key, i, o[2], c)
            # k carries the sign of the Ritz vector, which each eigen-solver
            # picks freely (z' and the next z flip with it; b and c are ratios)
            assert abs(abs(o[3]) - abs(k)) <= 1e-9 * abs(k), (key, i)
            assert abs(o[4] - sec[3]) <= 1e-5 * scale
            # second Ritz vector in the pre-update basis (x, y, z)
            if first:
                cv = np.array([o[5] * sx, 0.0, o[7]])
            else:
                cx = o[5]
                cy = o[6] + cx * o[1]
                cv = np.array([cx, cy, o[7] - cy * o[2]])
            ov = np.array(sec[:3])
            # FP32: the vector moves by ~2^-24 |V| / gap (gap to the lowest value)
            tol2 = max(1e-5, 1e-6 * scale / max(abs(sec[3] - E), 1e-300))
            assert min(_nerr(cv, s * ov, Nm) for s in (1.0, -1.0)) <= tol2, (key, i)
            ncmp["first" if first else "later"] += 1
            if not first and c == 0.0:
                ncmp["c0"] += 1
            i += 1
    assert ncmp["first"] > 20 and ncmp["later"] > 100


def test_step_decisions_match_the_oracle_trace(ctl, runs):
    p = osb.SBCIParams()
    n = 0
    for key, run in runs:
        E_prev = None
        for rec in run.trace:
            if rec.t == 0 and E_prev is None:
                E_prev = rec.energy + rec.dE  # a state's first record: E_t from |E_{t+1} - E_t|
            if rec.event == "undef":
                E_prev = rec.energy
                continue  # (the pending record's event 8 is set by the subspace solve)
            # E_t reproduced exactly: dE = |E_{t+1} - E_t| as the oracle recorded it
            E_t = rec.energy + rec.dE if abs(rec.energy + rec.dE - E_prev) < abs(rec.energy - rec.dE - E_prev) \
                else rec.energy - rec.dE
            halt, out = check(ctl, E_prev=E_t, E_new=rec.energy, b=rec.b, c=rec.c, k=rec.k, dz=rec.dz,
                              t=rec.t, alpha=rec.state, p=p)
            want = EVENT[rec.event]
            assert out[0] == want, (key, rec)
            if want == 1:
                assert halt == H_CONVERGED
                E_prev = None
            else:
                assert halt == H_RUN
                assert out[1] == (0 if want else rec.t + 1)
                E_prev = rec.energy
            n += 1
    assert n > 100


def test_low_precision_stage_switch_and_refinement_windows(ctl):
    base = dict(E_prev=-3.0, E_new=-3.0 - 1e-6, dz=1e-3, t=5, k=1.0, b=0.5)
    # stage 0 in low precision: switch (event 6) once dE < mixed_eps and |z'| < mixed_r
    halt, out = check(ctl, **{**base, "E_new": -3.0 - 1e-9, "dz": 5e-5}, stage=0, prec=TF32X3,
                      user_prec=TF32X3)
    assert halt == H_SWITCH and out[0] == 6
    halt, out = check(ctl, **base, stage=0, prec=TF32X3, user_prec=TF32X3, n_sync=40)
    assert halt == H_RUN and out[0] == 0  # no windows in stage 0
    # refinement stage: X made exact after max_cycle steps, FP64 after two windows
    halt, _ = check(ctl, **base, prec=TF32X3, user_prec=TF32X3, n_stage1=19, n_sync=19)
    assert halt == H_RUN
    halt, out = check(ctl, **base, prec=TF32X3, user_prec=TF32X3, n_stage1=20, n_sync=20)
    assert halt == H_SWITCH and out[0] == 0
    halt, _ = check(ctl, **base, prec=TF32X3, user_prec=TF32X3, n_stage1=40, n_sync=20)
    assert halt == H_CAP
    halt, _ = check(ctl, **base, prec=TF32X3, user_prec=TF32X3, n_stage1=30, n_sync=10,
                    refine_max_sigma=30)
    assert halt == H_CAP  # the refinement budget
    # after the FP64 fallback (prec FP64) and in FP64 solves: no windows
    for up in (TF32X3, FP64):
        halt, _ = check(ctl, **base, prec=FP64, user_prec=up, n_stage1=60, n_sync=60)
        assert halt == H_RUN
    # Eq. S61 comes first
    halt, out = check(ctl, E_prev=-3.0, E_new=-3.0 - 1e-11, dz=1e-6, t=5, prec=TF32X3,
                      user_prec=TF32X3, n_stage1=40, n_sync=20)
    assert halt == H_CONVERGED and out[0] == 1
    # a restart in the same step is still recorded and applied
    halt, out = check(ctl, **{**base, "k": 0.05}, prec=TF32X3, user_prec=TF32X3, n_stage1=20, n_sync=20)
    assert halt == H_SWITCH and out[0] == 3 and out[1] == 0 and out[2] == 1
    # the per-state cap
    halt, _ = check(ctl, **base, n_sigma=1000)
    assert halt == H_CAP


def test_restart_causes_in_order(ctl):
    p = osb.SBCIParams()
    # S62a only for excited states, with |b| < b_th and dE < eps1
    args = dict(E_prev=-2.0, E_new=-2.0 - 1e-8, b=1e-3, k=1.0, dz=1e-3, t=3)
    assert check(ctl, **args, alpha=1)[1][0] == 2
    assert check(ctl, **args, alpha=0)[1][0] == 0
    # S62b: |k| outside [x_th1, x_th2]
    assert check(ctl, **{**args, "k": 0.09})[1][0] == 3
    assert check(ctl, **{**args, "k": 1.21})[1][0] == 3
    assert check(ctl, **{**args, "k": -1.0})[1][0] == 0
    # S62c: |z'| > r1 for t > 0 only
    assert check(ctl, **{**args, "dz": 1.5})[1][0] == 4
    assert check(ctl, **{**args, "dz": 1.5, "t": 0})[1][0] == 0
    # max_cycle
    assert check(ctl, **{**args, "t": p.max_cycle - 1})[1][0] == 5
    assert check(ctl, **{**args, "t": p.max_cycle - 2})[1][0] == 0
    # S62a before S62b
    assert check(ctl, **{**args, "k": 0.05}, alpha=2)[1][0] == 2


def test_undefined_later_step_takes_the_first_step_path(ctl):
    """Reading R15: x, y, z orthonormal with x decoupled (H_xy = H_xz = 0) and
    the lowest Ritz vector inside span{y, z}: its x-component is exactly 0, so
    k, b and c of Eqs. S53-S55 are undefined.  The step is taken on the
    first-step path from x (y dropped): the 2x2 problem in (x, z) has its
    lowest vector along x (E = H_xx, k = 1, c = 0) and the record's event is 8."""
    Hxx, Hyy, Hyz, Hzz = -1.8, -2.0, 0.5, -1.5
    #        NXX  NXY  NYY  HXX  HXY  HYY  ZPZP NXZ  NYZ  NZZ  HXZ  HYZ  HZZ
    dots = [1.0, 0.0, 1.0, Hxx, 0.0, Hyy, 0.0, 0.0, 0.0, 1.0, 0.0, Hyz, Hzz]
    assert np.linalg.eigvalsh([[Hyy, Hyz], [Hyz, Hzz]])[0] < Hxx
    halt, o = solve(ctl, dots, first=0, sx=1.0)
    assert halt == H_RUN and o[11] == 8
    assert o[0] == Hxx and o[1] == 1.0 and o[2] == 0.0 and abs(o[3]) == 1.0
    assert o[9] == 0.0  # y dropped
    # the same problem posed as a first step gives the same parameters
    halt1, o1 = solve(ctl, dots, first=1, sx=1.0)
    assert halt1 == H_RUN and o1[11] == 0 and np.array_equal(o1[:4], o[:4])


def test_gram_schmidt_breakdowns(ctl):
    """Reading R7.  (1) After a step, y inside span{x} (N_xy^2 = N_xx N_yy):
    the next step takes the first-step path (t = 0, first = 1) without a
    restart record.  (2) A later step whose z lies in span{x, y}: c = 0 and
    the 2x2 problem in (x, y).  (3) A first step whose z lies in span{x}: no
    move (E = H_xx, c = 0, k = 1)."""
    halt, out = check(ctl, E_prev=-2.0, E_new=-2.0 - 1e-6, dz=1e-3, t=4, nxy=1.0)
    assert halt == H_RUN and out[0] == 0 and out[1] == 0 and out[2] == 1
    halt, out = check(ctl, E_prev=-2.0, E_new=-2.0 - 1e-6, dz=1e-3, t=4, nxy=0.5)
    assert halt == H_RUN and out[1] == 5 and out[2] == 0
    Hxx, Hxy, Hyy = -1.0, 0.3, -0.5
    #        NXX  NXY  NYY  HXX  HXY  HYY  ZPZP NXZ  NYZ  NZZ  HXZ  HYZ  HZZ
    dots = [1.0, 0.0, 1.0, Hxx, Hxy, Hyy, 0.0, 1.0, 0.0, 1.0, Hxx, Hxy, Hxx]  # z = x
    halt, o = solve(ctl, dots, first=0, sx=1.0)
    w, U = np.linalg.eigh([[Hxx, Hxy], [Hxy, Hyy]])
    assert halt == H_RUN and o[2] == 0.0 and abs(o[0] - w[0]) < 1e-14
    assert abs(o[1] - U[1, 0] / U[0, 0]) < 1e-12  # b: y coefficient over x coefficient
    assert abs(abs(o[3]) - 1.0 / abs(U[0, 0])) < 1e-12
    dots = [4.0, 0.0, 0.0, 4.0 * Hxx, 0.0, 0.0, 0.0, 2.0, 0.0, 1.0, 2.0 * Hxx, 0.0, Hxx]  # |x| = 2, z = x/2
    halt, o = solve(ctl, dots, first=1, sx=0.5)
    assert halt == H_RUN and o[0] == Hxx and o[2] == 0.0 and o[3] == 1.0
