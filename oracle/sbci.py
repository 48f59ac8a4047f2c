"""SBCI1 as the paper states it (oracle; test infrastructure only).

Follows Algorithm 1 (SBCI1 for state alpha) with Sections S1.1-S1.5:

* initial trial vectors from the lowest diagonal elements (S1.1, Eqs. S1-S3),
  or a given vector (then X_0 = H x_0 and E_0 its Rayleigh quotient, Eq. 2);
* excited-state start from the second eigenvector of V at the converging step
  (S1.4), orthogonalised against the stored states (Eqs. S4-S7);
* preconditioned, projected residual z (Eq. S8 / Eq. S31) with
  M^-1 = (D - E^0 I)^-1 (Eqs. 6-7);
* one H-product per step, Z = H z (Eq. S9 / Eq. S32);
* closed-form Gram-Schmidt, subspace matrix and parameters: first step
  (Eqs. S10-S24), later steps (Eqs. S33-S55);
* the momentum/position and H-image recurrences (Eqs. S25-S28, S56-S59);
* residual z' (Eq. S29 / Eq. S60) and convergence (Eq. S30 / Eq. S61);
* norm-triggered restart (Eqs. S62a-c and max_cycle).

Readings where the paper is silent or ambiguous, each with the reason it is
taken:

R1  z' = (X - E x)/k (Eqs. S29/S60); |z'| is then the residual norm of the
    unit vector x/|x| because |k| = |x| (Eq. S62b).
R2  The preconditioner denominator d = D_I - E^0 is replaced by
    sign(d) * guard when |d| < guard (guard = 1e-8; d = 0 -> +guard).
R3  E^0 is the current Rayleigh quotient E_t for state 0 and E_c^0 for
    excited states.
R4  A restart keeps x/|x| and X/|x|, sets y = Y = 0 and t = 0, and takes the
    first-step (2x2) path with z'_0 = X_0 - E_0 x_0; no extra H-product.
R5  max_cycle: a restart is triggered when t + 1 reaches max_cycle.
R6  A cap of ``max_sigma`` H-products per state ends the state unconverged.
R7  Gram-Schmidt breakdown: if a squared GS norm falls below gs_tol times the
    squared norm of the vector being orthogonalised, the direction is dropped
    (y dropped: first-step path; z dropped: c = 0 and the 2x2 problem in x, y).
R8  Initial determinants: the n_init lowest diagonal elements ordered by
    (D_I, flat index I), n_init = max(n_states, 2) unless given.
R9  X_0 of an excited state uses H x_c = E_c x_c (Eq. S5), no extra H-product.
R10 sector = 1 keeps c = c^T (Ia <-> Ib swap, n_alpha = n_beta): initial
    vectors and every z are symmetrised, z <- (z + z^T)/2.
R11 start_noise = eta > 0 adds eta * r_alpha / |r_alpha| to the (unit) start
    vector of every state, r_alpha a seeded SplitMix64 vector (``splitmix_vector``),
    with X += eta * H r_alpha / |r_alpha| and E_0 = the Rayleigh quotient, before
    the projection of Eqs. S4-S7.  An SBCI1 search keeps the spatial symmetry
    of its start vector; the small full-symmetry component lets it reach the
    lowest state of the orthogonal complement in symmetric molecules.  The
    default eta = 0 is the paper's choice (S1.1 / S1.4 starts as stated).
R15 If a later step's coefficients are undefined (a zero denominator in
    Eqs. S53-S55: the lowest Ritz vector of span{x, y, z} gives no finite k,
    b or c), that step is taken on the first-step path (Eqs. S10-S24) from
    x/|x| with y dropped, as a restart just before it would (trace event
    "undef").
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class SBCIParams:
    eps0: float = 1e-10  # S30/S61, no frozen core
    r0: float = 1e-5
    b_th: float = 1e-2  # S62a
    eps1: float = 1e-7
    x_th1: float = 0.1  # S62b
    x_th2: float = 1.2
    r1: float = 1.0  # S62c
    max_cycle: int = 20  # S1.5
    max_sigma: int = 1000  # R6, per state
    guard: float = 1e-8  # R2
    gs_tol: float = 1e-14  # S1.1 and R7
    sector: int = 0  # R10
    n_init: int | None = None  # R8
    start_noise: float = 0.0  # R11
    noise_seed: int = 0


@dataclass
class StepRecord:
    state: int
    t: int
    energy: float
    b: float
    c: float
    k: float
    dE: float
    dz: float
    event: str  # "", "converged", "restart:a", "restart:b", "restart:c", "restart:max"
    # right-hand side of Eq. S136 for this step's update, (2/c_{t-1}) Delta T
    # (Eqs. S134-S136 with the indices shifted to the update of step t, which
    # takes y_t to y_{t+1}): (b_{t-1}/c_{t-1}) (y_{t+1}^T M y_{t+1} - y_t^T M y_t),
    # M = D - E_{t+1}; NaN on first steps and where c_{t-1} = 0
    s136: float = float("nan")


@dataclass
class StateResult:
    energy: float
    vector: np.ndarray
    converged: bool
    n_sigma: int
    n_step: int
    restarts: dict = field(default_factory=dict)


_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix_vector(seed: int, alpha: int, n: int) -> np.ndarray:
    """Counter-based pseudo-random vector in [-1, 1): the SplitMix64 output
    function (Steele, Lea & Flood 2014; Vigna's splitmix64) applied to
    seed + GOLDEN * (alpha * 2^40 + I + 1) for I = 0..n-1, top 53 bits -> [0, 1)."""
    idx = (np.arange(n, dtype=np.uint64) + np.uint64(1)) + np.uint64((alpha << 40) & _M64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + idx * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def _guarded(d: np.ndarray, guard: float) -> np.ndarray:
    return np.where(np.abs(d) < guard, np.where(d < 0.0, -guard, guard), d)


def _sym(v: np.ndarray, shape) -> np.ndarray:
    m = v.reshape(shape)
    return (0.5 * (m + m.T)).reshape(-1)


def restart_cause(p, alpha, b, k, dE, dz, t):
    """Restart test of Section S1.5 after a step that did not converge, in the
    order the paper lists it: Eq. S62a (alpha > 0, |b| < b_th and the energy
    change below eps1), Eq. S62b (|k| = |x_{t+1}| outside [x_th1, x_th2]),
    Eq. S62c (|z'| > r1 on a later step, t > 0), then the max_cycle period
    (reading R5: t + 1 reaches max_cycle).  Returns "a", "b", "c", "max" or ""."""
    if alpha > 0 and abs(b) < p.b_th and dE < p.eps1:
        return "a"
    if abs(k) < p.x_th1 or abs(k) > p.x_th2:
        return "b"
    if dz > p.r1 and t > 0:
        return "c"
    if t + 1 >= p.max_cycle:
        return "max"
    return ""


class SBCI1:
    """SBCI1 driver over a sigma callable ``apply(v) -> H v`` (no e_core)."""

    def __init__(self, apply, diag: np.ndarray, shape, params: SBCIParams | None = None):
        self.apply = apply
        self.diag = np.asarray(diag, dtype=np.float64).reshape(-1)
        self.shape = tuple(shape)  # (Na, Nb)
        self.p = params or SBCIParams()
        self.trace: list[StepRecord] = []
        self.n_sigma = 0

    # -- helpers --------------------------------------------------------------
    def H(self, v):
        self.n_sigma += 1
        return np.asarray(self.apply(v.reshape(self.shape)), dtype=np.float64).reshape(-1)

    def _project(self, v, xc):
        """(1 - sum_i x_c^i x_c^iT) v (Eq. S8 / S31)."""
        for u in xc:
            v = v - u * (u @ v)
        return v

    # -- S1.1 -----------------------------------------------------------------
    def initial_guess(self, nstates: int):
        """Eqs. S1-S3: lowest-diagonal determinants, GS, subspace eigh."""
        n_init = self.p.n_init or max(nstates, 2)
        N = self.diag.size
        order = np.lexsort((np.arange(N), self.diag))  # (D_I, I) ascending
        basis = []
        for I in order[:n_init]:
            e = np.zeros(N)
            e[I] = 1.0
            if self.p.sector:
                e = _sym(e, self.shape)
            for u in basis:
                e = e - u * (u @ e)
            nrm = np.linalg.norm(e)
            if nrm < self.p.gs_tol:
                continue
            basis.append(e / nrm)
        Xm = [self.H(u) for u in basis]
        A = np.array([[u @ Xv for Xv in Xm] for u in basis])
        w, U = np.linalg.eigh(0.5 * (A + A.T))
        self.init_space = (basis, U, w)
        x0 = sum(U[i, 0] * basis[i] for i in range(len(basis)))
        X0 = sum(U[i, 0] * Xm[i] for i in range(len(basis)))
        return x0, X0, float(w[0])

    # -- one state (Algorithm 1) ----------------------------------------------
    def solve_state(self, alpha: int, x0, X0, E0, xc, Ec):
        p = self.p
        sigma0 = self.n_sigma
        # Algorithm 1 start: project out the stored states, Eqs. S4-S7
        ov = [u @ x0 for u in xc]
        x0p = x0 - sum((o * u for o, u in zip(ov, xc)), np.zeros_like(x0))
        X0p = X0 - sum((e * o * u for e, o, u in zip(Ec, ov, xc)), np.zeros_like(X0))
        nrm = np.linalg.norm(x0p)
        x, X = x0p / nrm, X0p / nrm
        E = E0
        y = np.zeros_like(x)
        Y = np.zeros_like(x)
        zp = X - E * x  # residual (H - E_0) x_0 of Algorithm 1, |x| = 1
        t = 0
        nstep = 0
        restarts = {"a": 0, "b": 0, "c": 0, "max": 0}
        second = None
        bc_prev = None  # (b, c) of the previous step, for the Eq. S136 diagnostic
        while True:
            if self.n_sigma - sigma0 >= p.max_sigma:
                return StateResult(E, x / np.linalg.norm(x), False, self.n_sigma - sigma0,
                                   nstep, restarts), second
            E_pre = E if alpha == 0 else Ec[0]  # R3
            w = zp / _guarded(self.diag - E_pre, p.guard)  # Eq. S31
            if p.sector:
                w = _sym(w, self.shape)
            z = self._project(w, xc)
            Z = self.H(z)  # Eq. S32
            if t > 0:
                Nxx, Nxy, Nyy = x @ x, x @ y, y @ y
                if Nyy - Nxy * Nxy / Nxx < p.gs_tol * Nyy:  # R7: y inside span{x}
                    nx = np.sqrt(Nxx)
                    x, X = x / nx, X / nx
                    y = np.zeros_like(x)
                    Y = np.zeros_like(x)
                    t = 0
            undefined = False
            if t > 0:
                E_new, b, c, k, sec = self._later_step(x, X, y, Y, z, Z)
                if not np.all(np.isfinite([E_new, b, c, k])):
                    # R15: a zero denominator in S53-S55 leaves the later step
                    # undefined; this step is taken on the first-step path
                    # from x/|x| with y dropped, as after a restart
                    nx = np.sqrt(x @ x)
                    x, X = x / nx, X / nx
                    y = np.zeros_like(x)
                    Y = np.zeros_like(x)
                    t = 0
                    undefined = True
            if t == 0:
                E_new, b, c, k, sec = self._first_step(x, X, z, Z)
                y_new = -c * z  # S25
                Y_new = -c * Z  # S26
                x_new = x + y_new  # S27 (b_0 = 1)
                X_new = X + Y_new  # S28
            else:
                y_new = y - c * z  # S56
                Y_new = Y - c * Z  # S57
                x_new = x + b * y_new  # S58
                X_new = X + b * Y_new  # S59
            s136 = float("nan")
            if t > 0 and bc_prev is not None and bc_prev[1] != 0.0:
                # Section S4: the kinetic-energy change of the update with the
                # mass M = D - E_{t+1} (the preconditioner's matrix), scaled by 2/c
                M = self.diag - E_new
                s136 = (bc_prev[0] / bc_prev[1]) * (y_new @ (M * y_new) - y @ (M * y))
            bc_prev = (b, c)
            # second Ritz vector in terms of the pre-update vectors (S1.4)
            cx, cy, cz, E2 = sec
            second = (cx * x + cy * y + cz * z, cx * X + cy * Y + cz * Z, E2)
            zp_new = (X_new - E_new * x_new) / k  # S60 (R1)
            dE = abs(E_new - E)
            dz = float(np.linalg.norm(zp_new))
            nstep += 1
            x, X, y, Y, zp = x_new, X_new, y_new, Y_new, zp_new
            if dE < p.eps0 and dz < p.r0:  # S61
                self.trace.append(StepRecord(alpha, t, E_new, b, c, k, dE, dz, "converged", s136))
                return StateResult(E_new, x / np.linalg.norm(x), True, self.n_sigma - sigma0,
                                   nstep, restarts), second
            cause = restart_cause(p, alpha, b, k, dE, dz, t)
            self.trace.append(StepRecord(alpha, t, E_new, b, c, k, dE, dz,
                                         f"restart:{cause}" if cause else ("undef" if undefined else ""),
                                         s136))
            E = E_new
            if cause:  # restart of Algorithm 1 with R4
                restarts[cause] += 1
                nx = np.linalg.norm(x)
                x, X = x / nx, X / nx
                y = np.zeros_like(x)
                Y = np.zeros_like(x)
                zp = X - E * x
                t = 0
            else:
                t += 1

    def _first_step(self, x, X, z, Z):
        """Eqs. S10-S24 (x normalised, y = 0)."""
        p = self.p
        Nxz, Nzz = x @ z, z @ z
        Hxx, Hxz, Hzz = x @ X, x @ Z, z @ Z
        g = Nzz - Nxz * Nxz
        if g < p.gs_tol * Nzz or g <= 0.0:  # R7: z inside span{x}
            return Hxx, 0.0, 0.0, 1.0, (0.0, 0.0, 0.0, Hxx)
        Bz = 1.0 / np.sqrt(g)  # S12
        Bx = -Nxz * Bz  # S13
        V = np.array([[Hxx, Bx * Hxx + Bz * Hxz],
                      [Bx * Hxx + Bz * Hxz, Bx * Bx * Hxx + Bz * Bz * Hzz + 2 * Bx * Bz * Hxz]])
        lam, U = np.linalg.eigh(V)
        vx, vz = U[0, 0], U[1, 0]
        k = 1.0 / (vx + vz * Bx)  # S23
        c = -vz * Bz / (vx + vz * Bx)  # S24
        wx, wz = U[0, 1], U[1, 1]
        sec = (wx + wz * Bx, 0.0, wz * Bz, float(lam[1]))
        return float(lam[0]), 1.0, float(c), float(k), sec

    def _later_step(self, x, X, y, Y, z, Z):
        """Eqs. S33-S55."""
        p = self.p
        Nxx, Nxy, Nxz = x @ x, x @ y, x @ z
        Nyy, Nyz, Nzz = y @ y, y @ z, z @ z
        Hxx, Hxy, Hxz = x @ X, x @ Y, x @ Z
        Hyy, Hyz, Hzz = y @ Y, y @ Z, z @ Z
        Ax = 1.0 / np.sqrt(Nxx)  # S34
        gy = Nyy - Nxy * Nxy / Nxx
        By = 1.0 / np.sqrt(gy)  # S36
        Bx = -Nxy / Nxx * By  # S37
        P = Bx * Nxz + By * Nyz  # S42
        gz = Nzz - Nxz * Nxz / Nxx - P * P
        if gz < p.gs_tol * Nzz or gz <= 0.0:  # R7: z inside span{x, y}
            V = np.array([[Ax * Ax * Hxx, Ax * (Bx * Hxx + By * Hxy)],
                          [Ax * (Bx * Hxx + By * Hxy),
                           Bx * Bx * Hxx + By * By * Hyy + 2 * Bx * By * Hxy]])
            lam, U = np.linalg.eigh(V)
            vx, vy = U[0, 0], U[1, 0]
            k = 1.0 / (vx * Ax + vy * Bx)
            b = vy * By * k
            wx, wy = U[0, 1], U[1, 1]
            return float(lam[0]), float(b), 0.0, float(k), \
                (wx * Ax + wy * Bx, wy * By, 0.0, float(lam[1]))
        Cz = 1.0 / np.sqrt(gz)  # S39
        Cy = -P * By * Cz  # S40
        Cx = -(Nxz / Nxx + P * Bx) * Cz  # S41
        hx = Cx * Hxx + Cy * Hxy + Cz * Hxz  # x^T H zbar / 1
        hy = Cx * Hxy + Cy * Hyy + Cz * Hyz  # y^T H zbar
        V = np.empty((3, 3))
        V[0, 0] = Ax * Ax * Hxx  # S44a
        V[0, 1] = V[1, 0] = Ax * (Bx * Hxx + By * Hxy)  # S44b
        V[0, 2] = V[2, 0] = Ax * hx  # S44c
        V[1, 1] = Bx * Bx * Hxx + By * By * Hyy + 2 * Bx * By * Hxy  # S44d
        V[1, 2] = V[2, 1] = Bx * hx + By * hy  # S44e (ybar^T H zbar)
        V[2, 2] = (Cx * Cx * Hxx + Cy * Cy * Hyy + Cz * Cz * Hzz
                   + 2 * Cx * Cy * Hxy + 2 * Cx * Cz * Hxz + 2 * Cy * Cz * Hyz)  # S44f
        lam, U = np.linalg.eigh(V)
        vx, vy, vz = U[:, 0]
        den = vx * Ax + vy * Bx + vz * Cx
        k = 1.0 / den  # S53
        b = (vy * By + vz * Cy) / den  # S54
        c = -vz * Cz / (vy * By + vz * Cy)  # S55
        wx, wy, wz = U[:, 1]
        sec = (wx * Ax + wy * Bx + wz * Cx, wy * By + wz * Cy, wz * Cz, float(lam[1]))
        return float(lam[0]), float(b), float(c), float(k), sec

    def _mix_noise(self, x0, X0, alpha):
        """R11: x0 <- x0/|x0| + eta r/|r|, X0 likewise with H r, E0 = RQ."""
        r = splitmix_vector(self.p.noise_seed, alpha, x0.size)
        if self.p.sector:
            r = _sym(r, self.shape)
        nr = np.linalg.norm(r)
        R = self.H(r)
        nx = np.linalg.norm(x0)
        eta = self.p.start_noise
        x = x0 / nx + (eta / nr) * r
        X = X0 / nx + (eta / nr) * R
        return x, X, float(x @ X) / float(x @ x)

    # -- driver ---------------------------------------------------------------
    def solve(self, nstates: int, c0: np.ndarray | None = None):
        """States 0..nstates-1 in sequence (Fig. 1A)."""
        xc, Ec, results = [], [], []
        self.init_space = None
        if c0 is None:
            x0, X0, E0 = self.initial_guess(nstates)
        else:
            x0 = np.asarray(c0, dtype=np.float64).reshape(-1).copy()
            if self.p.sector:
                x0 = _sym(x0, self.shape)
            x0 /= np.linalg.norm(x0)
            X0 = self.H(x0)
            E0 = float(x0 @ X0)
        if self.p.start_noise > 0.0:
            x0, X0, E0 = self._mix_noise(x0, X0, 0)
        for alpha in range(nstates):
            res, second = self.solve_state(alpha, x0, X0, E0, xc, Ec)
            results.append(res)
            xc.append(res.vector)
            Ec.append(res.energy)
            if alpha + 1 < nstates:
                x0, X0, E0 = second  # S1.4
                if self.p.start_noise > 0.0:
                    x0, X0, E0 = self._mix_noise(x0, X0, alpha + 1)
        return results
