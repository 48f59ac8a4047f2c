"""SBCI2 as the paper states it (oracle; test infrastructure only).

Algorithm 2 with Sections S2.1-S2.5: states are found one by one from the
lowest upward while the pair (alpha, alpha+1) is updated together
(Fig. 1B); the highest state is found by SBCI1 (``oracle.sbci``).

* start vectors x_0^i = sum_j U_0[j, i] x_{-1}^j from the subspace of the
  lowest-diagonal determinants (Eqs. S74-S76);
* pair start: projection against the stored states with X by E_c x_c, and
  normalisation (Algorithm 2 line 1, Eqs. S77-S80);
* preconditioned, projected residuals z (Eqs. S81, S101) and two H-products
  Z = H z per step (Eqs. S82, S102);
* canonical orthogonalisation of {x^a, x^b, (y^a, y^b,) z^a, z^b}: overlap S,
  eigenvalues below 1e-14 dropped, P = U s^(-1/2) (Eqs. S83, S103); H in that
  basis (Eqs. S84, S104), its two lowest eigenvectors V' = P V (Eqs. S85-S87,
  S105-S107);
* first-step coefficients (Eq. S93) and later-step coefficients
  (Eqs. S112, S116, S117, S121); updates of y, Y, x, X (Eqs. S94-S97,
  S122-S125); residual z' and the convergence test on the lower state
  (Eqs. S98-S100, S126-S128);
* restarts S130a-c and max_cycle = 10 (Section S2.5).

Readings where the paper is silent or ambiguous, each with the reason it is
taken:

Q1  Start vectors: determinants by ascending (D_I, I), symmetrised when
    sector = 1 and Gram-Schmidt orthonormalised (dropped below gs_tol), until
    max(k, n_init or 2) vectors hold, so that every upper state has a start
    (S2.2 asks for n determinants; a swap pair gives one sector vector).
Q2  The upper start vector of a later pair (state alpha+1 from Eq. S75) is
    projected against the stored states and then against the new lower vector
    x_0^alpha, normalised, and its E_0 is its Rayleigh quotient x_0^T X_0 (the
    S75 eigenvalue belongs to the unprojected vector).
Q3  The preconditioner shift E^0 is the current E_t of state 0 while the
    ground pair runs and E_c^0 afterwards (SBCI1's R3), for both residuals.
Q4  The subspace matrix is (T + T^T)/2 with T = B^T [H B] from the carried
    H-images.
Q5  Canonical orthogonalisation drops overlap eigenvalues below 1e-14 in
    absolute value (as written; the vectors are not rescaled first).
Q6  If a step's coefficients are undefined (a zero or non-finite
    denominator in Eqs. S93, S116, S117 or a singular 2x2 matrix in Eq. S121),
    the step is taken on the first-step path from the same x and z with y
    dropped (SBCI1's R15).
Q7  A restart (Algorithm 2 lines 19-20, "go to 4") keeps x/|x| and X/|x|,
    E_0 = E_{t+1}, sets y = Y = 0 and t = 0, and takes the first-step path with
    z'_0 = X_0 - E_0 x_0; no extra H-product.  The last state starts from the
    normalised upper vector of the last pair, its E and X (SBCI1 then
    projects it, Eqs. S4-S7).
Q8  A cap of max_sigma H-products per lower state ends the pair with that
    state unconverged (stored as is).
Q9  x_{t+1} and X_{t+1} are evaluated as k_i v^i = k_i [basis] V'[:, i] and
    k_i [H-images] V'[:, i], the vectors Eqs. S124-S125 give in exact
    arithmetic (Eq. S110).  Written as x_t + B y_{t+1}, they cancel to |k| of
    their terms when |k| is small (k reaches 1e-12 on H6 when the pair's Ritz
    vectors swap order), and x and X then lose different digits.
Q10 That upper start vector gets X_0 = H x_0 by one H-product after its
    projections.  Eq. S78's shortcut H x_c = E_c x_c is exact only for exact
    eigenvectors; a fresh S75 vector has overlaps of order one with the stored
    states, so the shortcut carries their residuals (about r0) into X_0, and
    the pair's Ritz values then sit about 1e-7 hartree off on H6 (below the
    exact value).  The lower vector, orthogonal to the stored states up to
    rounding, keeps the shortcut.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .sbci import SBCI1, SBCIParams, StateResult, _guarded, _sym


@dataclass
class PairStep:
    state: int                 # alpha (lower state of the pair)
    t: int
    energies: tuple            # (E_{t+1}^alpha, E_{t+1}^{alpha+1})
    k: tuple                   # (k0, k1)
    dE: float
    dz: float
    first: bool                # first-step path (Eq. S93)
    rank: int                  # basis vectors kept by the canonical orthogonalisation
    event: str                 # "", "converged", "restart:a|b|c|max", "undef"


def canonical_orthogonalisation(S: np.ndarray, tol: float = 1e-14):
    """P = U s^(-1/2) over the overlap eigenvalues s >= tol (Eqs. S83, S103)."""
    s, U = np.linalg.eigh(0.5 * (S + S.T))
    keep = s >= tol
    return U[:, keep] / np.sqrt(s[keep])


def pair_coefficients(Vp: np.ndarray, first: bool):
    """A, B, C and k0, k1 from V' = P V (columns 0 and 1): Eq. S93 on the first
    step (basis x^a, x^b, z^a, z^b), Eqs. S112, S116, S117, S121 afterwards
    (basis x^a, x^b, y^a, y^b, z^a, z^b).  Returns None if undefined."""
    with np.errstate(divide="ignore", invalid="ignore"):
        if first:
            k0 = 1.0 / Vp[0, 0]
            k1 = 1.0 / Vp[1, 1]
            a_ab = Vp[1, 0] / Vp[0, 0]
            a_ba = Vp[0, 1] / Vp[1, 1]
            C = np.array([[-Vp[2, 0] / Vp[0, 0], -Vp[3, 0] / Vp[0, 0]],
                          [-Vp[2, 1] / Vp[1, 1], -Vp[3, 1] / Vp[1, 1]]])
            B = np.eye(2)
        else:
            a_ab = Vp[1, 0] / Vp[2, 0]
            a_ba = Vp[0, 1] / Vp[3, 1]
            k0 = 1.0 / (Vp[0, 0] - Vp[3, 0] * a_ba)
            k1 = 1.0 / (Vp[1, 1] - Vp[2, 1] * a_ab)
            B = np.array([[k0 * Vp[2, 0], k0 * Vp[3, 0]],
                          [k1 * Vp[2, 1], k1 * Vp[3, 1]]])
            M = np.array([[Vp[2, 0], Vp[3, 0]], [Vp[2, 1], Vp[3, 1]]])
            R = np.array([[Vp[4, 0], Vp[5, 0]], [Vp[4, 1], Vp[5, 1]]])
            det = M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]
            if not (np.isfinite(det) and det != 0.0):
                return None
            C = -np.array([[M[1, 1], -M[0, 1]], [-M[1, 0], M[0, 0]]]) @ R / det
    vals = np.concatenate([[k0, k1, a_ab, a_ba], B.ravel(), C.ravel()])
    if not np.all(np.isfinite(vals)):
        return None
    A = np.array([[0.0, a_ab], [a_ba, 0.0]])
    return A, B, C, k0, k1


class SBCI2:
    """SBCI2 driver over a sigma callable ``apply(v) -> H v`` (no e_core)."""

    def __init__(self, apply, diag, shape, params: SBCIParams | None = None, max_cycle2: int = 10,
                 step_hook=None):
        self.apply = apply
        self.diag = np.asarray(diag, dtype=np.float64).reshape(-1)
        self.shape = tuple(shape)
        self.p = params or SBCIParams()
        self.max_cycle2 = max_cycle2
        self.step_hook = step_hook  # called with a dict of the step's vectors and coefficients
        self.trace: list[PairStep] = []
        self.n_sigma = 0

    def H(self, v):
        self.n_sigma += 1
        return np.asarray(self.apply(v.reshape(self.shape)), dtype=np.float64).reshape(-1)

    def _project(self, v, xc):
        for u in xc:
            v = v - u * (u @ v)
        return v

    # -- Q1 / Eqs. S74-S76 ----------------------------------------------------
    def start_vectors(self, k: int):
        n_v = max(k, self.p.n_init or 2)
        N = self.diag.size
        order = np.lexsort((np.arange(N), self.diag))
        basis = []
        for I in order:
            if len(basis) >= n_v:
                break
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
        if len(basis) < k:
            raise ValueError("the space holds fewer than k start vectors")
        Xm = [self.H(u) for u in basis]
        A = np.array([[u @ Xv for Xv in Xm] for u in basis])
        w, U = np.linalg.eigh(0.5 * (A + A.T))
        xs = [sum(U[j, i] * basis[j] for j in range(len(basis))) for i in range(len(basis))]
        Xs = [sum(U[j, i] * Xm[j] for j in range(len(basis))) for i in range(len(basis))]
        return xs, Xs, w

    # -- one pair (Algorithm 2) -----------------------------------------------
    def solve_pair(self, alpha, xa, Xa, Ea, xb, Xb, Eb, xc, Ec):
        p = self.p
        sigma0 = self.n_sigma
        # line 1, Eqs. S77-S80: project against the stored states, normalise
        xs, Xs = [], []
        for x, X in ((xa, Xa), (xb, Xb)):
            ov = [u @ x for u in xc]
            x = x - sum((o * u for o, u in zip(ov, xc)), np.zeros_like(x))
            X = X - sum((e * o * u for e, o, u in zip(Ec, ov, xc)), np.zeros_like(X))
            n = np.linalg.norm(x)
            xs.append(x / n)
            Xs.append(X / n)
        x = xs
        X = Xs
        E = [Ea, Eb]
        y = [np.zeros_like(x[0]), np.zeros_like(x[0])]
        Y = [np.zeros_like(x[0]), np.zeros_like(x[0])]
        zp = [X[i] - E[i] * x[i] for i in range(2)]  # line 3
        first = True
        t = 0
        restarts = {"a": 0, "b": 0, "c": 0, "max": 0}
        nstep = 0
        while True:
            if self.n_sigma - sigma0 >= p.max_sigma:  # Q8
                n = np.linalg.norm(x[0])
                return (StateResult(E[0], x[0] / n, False, self.n_sigma - sigma0, nstep, restarts),
                        (x[1] / np.linalg.norm(x[1]), X[1] / np.linalg.norm(x[1]), E[1]))
            E_pre = E[0] if alpha == 0 else Ec[0]  # Q3
            z, Z = [], []
            for i in range(2):  # Eqs. S81 / S101, then S82 / S102
                zi = zp[i] / _guarded(self.diag - E_pre, p.guard)
                if p.sector:
                    zi = _sym(zi, self.shape)
                zi = self._project(zi, xc)
                z.append(zi)
            for i in range(2):
                Z.append(self.H(z[i]))
            step = None
            for path_first in ((True,) if first else (False, True)):
                if path_first:
                    Bv = [x[0], x[1], z[0], z[1]]
                    HB = [X[0], X[1], Z[0], Z[1]]
                else:
                    Bv = [x[0], x[1], y[0], y[1], z[0], z[1]]
                    HB = [X[0], X[1], Y[0], Y[1], Z[0], Z[1]]
                Bm = np.column_stack(Bv)
                S = Bm.T @ Bm
                T = Bm.T @ np.column_stack(HB)
                P = canonical_orthogonalisation(S)
                if P.shape[1] < 2:
                    continue
                Hh = P.T @ (0.5 * (T + T.T)) @ P
                w, V = np.linalg.eigh(0.5 * (Hh + Hh.T))
                Vp = P @ V
                coef = pair_coefficients(Vp, path_first)
                if coef is not None:
                    step = (path_first, coef, w, P.shape[1], Bv, HB, Vp)
                    break
            if step is None:
                raise RuntimeError("SBCI2: no defined step (subspace rank below 2)")
            path_first, (A, Bc, C, k0, k1), w, rank, Bv, HB, Vp = step
            k = (k0, k1)
            undef = path_first and not first
            if path_first:  # y dropped (first step, Q6)
                yo = [np.zeros_like(x[0]), np.zeros_like(x[0])]
                Yo = [np.zeros_like(x[0]), np.zeros_like(x[0])]
            else:
                yo, Yo = y, Y
            # Eqs. S72 / S94 / S122 and S123: y_{t+1} = y_t - C z_t + A x_t
            yn = [yo[i] - C[i, 0] * z[0] - C[i, 1] * z[1] + A[i, 1 - i] * x[1 - i] for i in range(2)]
            Yn = [Yo[i] - C[i, 0] * Z[0] - C[i, 1] * Z[1] + A[i, 1 - i] * X[1 - i] for i in range(2)]
            # Eqs. S73 / S96 / S124 and S125, x_{t+1} = x_t + B y_{t+1}, evaluated
            # as k_i v^i = k_i [B] V'[:, i] and its H-image (Eq. S110; Q9)
            xn = [k[i] * sum(Vp[j, i] * Bv[j] for j in range(len(Bv))) for i in range(2)]
            Xn = [k[i] * sum(Vp[j, i] * HB[j] for j in range(len(Bv))) for i in range(2)]
            En = [float(w[0]), float(w[1])]
            if self.step_hook is not None:
                self.step_hook(dict(basis=Bv, x_old=x, y_new=yn, B=Bc, A=A, C=C, k=k,
                                    x_new=xn, X_new=Xn, E_new=En, first=path_first))
            nstep += 1
            # Eqs. S98 / S126, S99 / S127
            zpn = [(Xn[i] - En[i] * xn[i]) / k[i] for i in range(2)]
            dE = abs(En[0] - E[0])
            dz = float(np.linalg.norm(zpn[0]))
            rec = PairStep(alpha, t, tuple(En), k, dE, dz, path_first, rank, "undef" if undef else "")
            self.trace.append(rec)
            if dE < p.eps0 and dz < p.r0:
                rec.event = "converged"
                na, nb = np.linalg.norm(xn[0]), np.linalg.norm(xn[1])
                return (StateResult(En[0], xn[0] / na, True, self.n_sigma - sigma0, nstep, restarts),
                        (xn[1] / nb, Xn[1] / nb, En[1]))
            # Section S2.5
            cause = None
            if (abs(Bc[0, 0]) < p.b_th or abs(Bc[1, 1]) < p.b_th) and dE < p.eps1:
                cause = "a"
            elif min(abs(k0), abs(k1)) < p.x_th1 or max(abs(k0), abs(k1)) > p.x_th2:
                cause = "b"
            elif dz > p.r1 and t > 0:
                cause = "c"
            elif t + 1 >= self.max_cycle2:
                cause = "max"
            if cause is not None:  # Q7
                restarts[cause] += 1
                rec.event = "restart:" + cause
                for i in range(2):
                    n = np.linalg.norm(xn[i])
                    xn[i] = xn[i] / n
                    Xn[i] = Xn[i] / n
                x, X = xn, Xn
                E = En
                y = [np.zeros_like(x[0]), np.zeros_like(x[0])]
                Y = [np.zeros_like(x[0]), np.zeros_like(x[0])]
                zp = [X[i] - E[i] * x[i] for i in range(2)]
                first = True
                t = 0
                continue
            x, X, y, Y = xn, Xn, yn, Yn
            E = En
            zp = zpn
            first = False
            t += 1

    def solve(self, nstates: int):
        """States 0..nstates-1 (Fig. 1B): pairs (alpha, alpha+1) for
        alpha = 0..nstates-2, then SBCI1 for the last state."""
        xs, Xs, w = self.start_vectors(nstates)
        xc, Ec, results = [], [], []
        if nstates == 1:
            one = SBCI1(self.apply, self.diag, self.shape, self.p)
            res, _ = one.solve_state(0, xs[0], Xs[0], float(w[0]), xc, Ec)
            self.n_sigma += one.n_sigma
            return [res]
        lower = (xs[0], Xs[0], float(w[0]))
        for alpha in range(nstates - 1):
            xa, Xa, Ea = lower
            if alpha == 0:
                xb, Xb, Eb = xs[1], Xs[1], float(w[1])
            else:  # Q2
                xb, Xb = xs[alpha + 1], Xs[alpha + 1]
                ov = [u @ xb for u in xc]
                xb = xb - sum((o * u for o, u in zip(ov, xc)), np.zeros_like(xb))
                Xb = Xb - sum((e * o * u for e, o, u in zip(Ec, ov, xc)), np.zeros_like(Xb))
                o = xa @ xb
                xb = xb - o * xa
                n = np.linalg.norm(xb)
                xb = xb / n
                Xb = self.H(xb)  # Q10
                Eb = float(xb @ Xb)
            res, lower = self.solve_pair(alpha, xa, Xa, Ea, xb, Xb, Eb, xc, Ec)
            results.append(res)
            xc.append(res.vector)
            Ec.append(res.energy)
        # the last state by SBCI1 from the pair's upper vector (Fig. 1B)
        one = SBCI1(self.apply, self.diag, self.shape, self.p)
        xl, Xl, El = lower
        res, _ = one.solve_state(nstates - 1, xl, Xl, El, xc, Ec)
        self.n_sigma += one.n_sigma
        results.append(res)
        return results
