"""Reference eigen-solvers (oracle; test infrastructure only).

* ``lowest_dense``: numpy.linalg.eigh of the dense Slater-Condon H.
* ``lowest_lanczos``: scipy.sparse.linalg.eigsh (implicitly restarted Lanczos)
  on the string-driven sigma.
* ``davidson``: a textbook block Davidson (Davidson 1975; Liu 1978) with the
  diagonal preconditioner (D - theta)^-1 -- the method the paper compares SBCI
  against (Introduction; Materials and Methods), written from its published
  definition.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def lowest_dense(H: np.ndarray, k: int):
    w, v = np.linalg.eigh(H)
    return w[:k], v[:, :k]


def lowest_lanczos(apply, ndet: int, k: int, tol: float = 1e-12, v0=None):
    op = spla.LinearOperator((ndet, ndet), matvec=lambda v: apply(v).reshape(-1),
                             dtype=np.float64)
    w, v = spla.eigsh(op, k=k, which="SA", tol=tol, v0=v0)
    order = np.argsort(w)
    return w[order], v[:, order]


def davidson(apply, diag: np.ndarray, k: int, tol: float = 1e-8, max_iter: int = 200,
             max_space: int | None = None, guard: float = 1e-8):
    """Lowest k eigenpairs.  Converged when every wanted residual norm < tol."""
    n = diag.size
    max_space = max_space or max(8 * k, 20)
    order = np.argsort(diag, kind="stable")
    V = np.zeros((n, 0))
    for i in order[:k]:
        e = np.zeros(n)
        e[i] = 1.0
        V = np.column_stack([V, e])
    AV = np.column_stack([apply(V[:, j]).reshape(-1) for j in range(V.shape[1])])
    for _ in range(max_iter):
        T = V.T @ AV
        theta, S = np.linalg.eigh(0.5 * (T + T.T))
        theta, S = theta[:k], S[:, :k]
        X = V @ S
        R = AV @ S - X * theta
        rn = np.linalg.norm(R, axis=0)
        if np.all(rn < tol):
            return theta, X
        if V.shape[1] + k > max_space:  # collapse onto the current Ritz vectors
            V, _ = np.linalg.qr(X)
            AV = np.column_stack([apply(V[:, j]).reshape(-1) for j in range(V.shape[1])])
        for j in range(k):
            if rn[j] < tol:
                continue
            d = diag - theta[j]
            d = np.where(np.abs(d) < guard, np.where(d < 0, -guard, guard), d)
            t = R[:, j] / d
            for _ in range(2):
                t -= V @ (V.T @ t)
            nt = np.linalg.norm(t)
            if nt < 1e-14:
                continue
            t /= nt
            V = np.column_stack([V, t])
            AV = np.column_stack([AV, apply(t).reshape(-1)])
    raise RuntimeError("Davidson did not converge")
