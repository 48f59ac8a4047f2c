"""Block Davidson-Liu eigen-solver (oracle; test infrastructure only).

The paper measures SBCI against the Davidson method (Davidson 1975; Liu 1978)
as implemented in PySCF, with the diagonal preconditioner (D - E^0 I)^-1
(Introduction; Materials and Methods).  This module states that method
plainly, with every choice the paper leaves open fixed so that a second
implementation can follow the same schedule step by step:

D1  Start: determinants in ascending (D_I, I) order, each symmetrised
    (sector = 1: v <- (v + v^T)/2) and Gram-Schmidt orthonormalised against
    the ones before it (dropped if its norm falls below gs_tol), until the
    start holds n_v = max(k, n_init or 2) vectors.  Their H-images are the
    first H-products.
D2  Each iteration: T = V^T (H V), subspace matrix A = (T + T^T)/2, its
    eigenpairs by eigh; Ritz values theta_a (a < k, ascending), Ritz vectors
    x_a = V s_a, residuals r_a = (H V) s_a - theta_a x_a.
D3  State a has converged when |theta_a - theta_a(previous iteration)| < eps0
    and |r_a| < r0 (the thresholds of Eq. S61; the first iteration has no
    previous value).  All k converged: stop.
D4  Collapse: if m + (unconverged states) > max_space, V <- V S_k and
    H V <- (H V) S_k (the k Ritz vectors and their H-images; no H-product).
D5  Correction of each unconverged state a, in ascending a: t = r_a / d with
    d = D - theta_a guarded as in SBCI (|d| < guard -> sign(d) guard,
    d = 0 -> +guard); symmetrised when sector = 1; orthogonalised twice
    against the current V (classical Gram-Schmidt, t <- t - V (V^T t)); kept
    if |t|^2 >= gs_tol |t_0|^2 (t_0 = t before the projections), normalised,
    appended to V, and its H-image is one H-product.
D6  An iteration that adds no vector (every correction dropped, or the cap
    of max_sigma H-products in total reached) ends the solve: converged if
    every |r_a| < r0 (the next iteration would repeat the same theta), else
    unconverged.
D7  max_space defaults to max(12, 4k) vectors (12 is PySCF's default subspace
    size; the paper does not state the value it ran with).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class DavidsonResult:
    energies: np.ndarray        # Ritz values theta_a (electronic)
    vectors: np.ndarray         # [Ndet, k] Ritz vectors
    residuals: np.ndarray       # |r_a|
    converged: bool
    n_iter: int                 # iterations of D2 (subspace eigen-solves)
    n_sigma: int                # H-products, start included
    n_collapse: int
    trace: list = field(default_factory=list)  # per iteration: (m, theta[k], |r|[k])


def _guarded(d: np.ndarray, guard: float) -> np.ndarray:
    return np.where(np.abs(d) < guard, np.where(d < 0.0, -guard, guard), d)


def _sym(v: np.ndarray, shape) -> np.ndarray:
    m = v.reshape(shape)
    return (0.5 * (m + m.T)).reshape(-1)


def start_vectors(diag: np.ndarray, shape, k: int, n_init: int | None = None, sector: bool = False,
                  gs_tol: float = 1e-14) -> list:
    """D1: orthonormal start vectors from the lowest diagonal elements."""
    n_v = max(k, n_init or 2)
    N = diag.size
    order = np.lexsort((np.arange(N), diag))  # (D_I, I) ascending
    basis = []
    for I in order:
        if len(basis) >= n_v:
            break
        e = np.zeros(N)
        e[I] = 1.0
        if sector:
            e = _sym(e, shape)
        for u in basis:
            e = e - u * (u @ e)
        nrm = np.linalg.norm(e)
        if nrm < gs_tol:
            continue
        basis.append(e / nrm)
    if len(basis) < k:
        raise ValueError("the space holds fewer than k start vectors")
    return basis


def davidson_liu(apply, diag, shape, k: int, *, eps0: float = 1e-10, r0: float = 1e-5,
                 max_space: int | None = None, max_sigma: int = 1000, guard: float = 1e-8,
                 gs_tol: float = 1e-14, sector: bool = False, n_init: int | None = None) -> DavidsonResult:
    """Lowest k eigenpairs of H by D1-D6.  apply(v) returns H v for v of
    ``shape`` (electronic H); diag = D_I."""
    diag = np.asarray(diag, dtype=np.float64).reshape(-1)
    max_space = max_space or max(12, 4 * k)
    if max_space < 2 * k:
        raise ValueError("max_space must hold at least 2k vectors")

    def H(v):
        return np.asarray(apply(v.reshape(shape)), dtype=np.float64).reshape(-1)

    V = start_vectors(diag, shape, k, n_init, sector, gs_tol)
    AV = [H(v) for v in V]
    n_sigma = len(V)
    theta_prev = None
    trace = []
    n_collapse = 0
    it = 0
    while True:
        it += 1
        Vm = np.column_stack(V)
        AVm = np.column_stack(AV)
        T = Vm.T @ AVm
        w, S = np.linalg.eigh(0.5 * (T + T.T))
        theta, Sk = w[:k], S[:, :k]
        X = Vm @ Sk
        R = AVm @ Sk - X * theta
        rn = np.linalg.norm(R, axis=0)
        trace.append((len(V), theta.copy(), rn.copy()))
        de = np.full(k, np.inf) if theta_prev is None else np.abs(theta - theta_prev)
        conv = (de < eps0) & (rn < r0)
        if np.all(conv):
            return DavidsonResult(theta, X, rn, True, it, n_sigma, n_collapse, trace)
        theta_prev = theta.copy()
        unconv = [a for a in range(k) if not conv[a]]
        if len(V) + len(unconv) > max_space:  # D4
            V = [X[:, a].copy() for a in range(k)]
            AV = [AVm @ Sk[:, a] for a in range(k)]
            n_collapse += 1
        added = 0
        for a in unconv:  # D5
            if n_sigma >= max_sigma:
                break
            t = R[:, a] / _guarded(diag - theta[a], guard)
            if sector:
                t = _sym(t, shape)
            n0 = t @ t
            for _ in range(2):
                Vm = np.column_stack(V)
                t = t - Vm @ (Vm.T @ t)
            nt = t @ t
            if not (nt > 0.0 and nt >= gs_tol * n0):
                continue
            t = t / np.sqrt(nt)
            V.append(t)
            AV.append(H(t))
            n_sigma += 1
            added += 1
        if added == 0:  # D6
            return DavidsonResult(theta, X, rn, bool(np.all(rn < r0)), it, n_sigma, n_collapse, trace)
