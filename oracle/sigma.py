"""String-driven sigma = H c (oracle; test infrastructure only).

The paper forms Z = H z once per step (Eq. S9, Eq. S32) and leaves the
product to PySCF.  This module writes it from the second-quantised spin-free
Hamiltonian in the spatial-orbital excitation operators
E_ij = E^alpha_ij + E^beta_ij:

    H = sum_ij h_ij E_ij + 1/2 sum_ijkl (ij|kl) (E_ij E_kl - delta_jk E_il)

so that, with D[k,l] = E_kl c and G[i,j] = sum_kl (ij|kl) D[k,l],

    sigma = sum_ij h_ij D[i,j] + 1/2 sum_ij E_ij G[i,j]
            - 1/2 sum_il (sum_j (ij|jl)) D[i,l]      (+ e_core c).

E_kl acts on the alpha string index of c (rows) and on the beta string index
(columns) through the string matrices M_kl[I, J] = <I|E_kl|J>, read off the
excitation lists of ``oracle.strings``: E^a_kl c = M^a_kl c and
E^b_kl c = c (M^b_kl)^T.  No packing of orbital pairs, no absorption of the
one-electron part and no fusion: each step is the definition above.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .strings import excitation_list


def excitation_matrices(norb: int, nelec: int):
    """M[k][l] = sparse <I|E_kl|J> over the strings of ``nelec`` electrons."""
    table = excitation_list(norb, nelec)
    nstr = table.shape[0]
    rows = {(k, l): ([], [], []) for k in range(norb) for l in range(norb)}
    for J in range(nstr):  # the list of J holds (k, l, I, s): E_kl |J> = s |I>
        for k, l, I, s in table[J]:
            r = rows[(int(k), int(l))]
            r[0].append(int(I))
            r[1].append(J)
            r[2].append(float(s))
    M = [[None] * norb for _ in range(norb)]
    for (k, l), (ii, jj, vv) in rows.items():
        M[k][l] = sp.csr_matrix((vv, (ii, jj)), shape=(nstr, nstr))
    return M


class StringSigma:
    """sigma = (H - e_core) c for one (h1, eri, nalpha, nbeta), FP64."""

    def __init__(self, h1, eri, nalpha: int, nbeta: int, block_rows: int = 256):
        self.h1 = np.asarray(h1, dtype=np.float64)
        self.eri = np.asarray(eri, dtype=np.float64)
        self.n = self.h1.shape[0]
        self.nalpha, self.nbeta = nalpha, nbeta
        self.Ma = excitation_matrices(self.n, nalpha)
        self.Mb = excitation_matrices(self.n, nbeta) if nbeta != nalpha else self.Ma
        self.Na = self.Ma[0][0].shape[0]
        self.Nb = self.Mb[0][0].shape[0]
        self.block_rows = block_rows
        # one-electron operator of the normal-ordering correction: sum_j (ij|jl)
        self.kcorr = np.einsum("ijjl->il", self.eri)

    @property
    def ndet(self) -> int:
        return self.Na * self.Nb

    def E(self, k: int, l: int, c: np.ndarray) -> np.ndarray:
        """(E^a_kl + E^b_kl) c for c of shape [Na, Nb]."""
        return self.Ma[k][l] @ c + (self.Mb[k][l] @ c.T).T

    def apply(self, c: np.ndarray) -> np.ndarray:
        n = self.n
        c = np.asarray(c, dtype=np.float64).reshape(self.Na, self.Nb)
        if self.Na * self.Nb * n * n <= 64_000_000:
            return self._apply_full(c)
        return self._apply_blocked(c)

    def _apply_full(self, c):
        n = self.n
        D = np.stack([self.E(k, l, c) for k in range(n) for l in range(n)])  # [n*n, Na, Nb]
        sigma = np.einsum("kl,klab->ab", self.h1, D.reshape(n, n, self.Na, self.Nb))
        sigma -= 0.5 * np.einsum("il,ilab->ab", self.kcorr, D.reshape(n, n, self.Na, self.Nb))
        G = (self.eri.reshape(n * n, n * n) @ D.reshape(n * n, -1)).reshape(n * n, self.Na, self.Nb)
        for i in range(n):
            for j in range(n):
                sigma += 0.5 * self.E(i, j, G[i * n + j])
        return sigma

    def _apply_blocked(self, c):
        """Same sums, with D and G formed for a block of alpha rows at a time.

        sigma is linear in D, so the alpha-excitation part of E_ij G is the sum
        over row blocks of M^a_ij[:, block] G[block]; the beta part stays in
        the block's rows.
        """
        n = self.n
        Na, Nb = self.Na, self.Nb
        sigma = np.zeros((Na, Nb))
        eri2 = self.eri.reshape(n * n, n * n)
        for a0 in range(0, Na, self.block_rows):
            a1 = min(Na, a0 + self.block_rows)
            rows = slice(a0, a1)
            D = np.empty((n * n, a1 - a0, Nb))
            for k in range(n):
                for l in range(n):
                    D[k * n + l] = (self.Ma[k][l][rows] @ c) + (self.Mb[k][l] @ c[rows].T).T
            sigma[rows] += np.einsum("kl,klab->ab", self.h1, D.reshape(n, n, a1 - a0, Nb))
            sigma[rows] -= 0.5 * np.einsum("il,ilab->ab", self.kcorr,
                                           D.reshape(n, n, a1 - a0, Nb))
            G = (eri2 @ D.reshape(n * n, -1)).reshape(n * n, a1 - a0, Nb)
            for i in range(n):
                for j in range(n):
                    Gij = G[i * n + j]
                    sigma += 0.5 * (self.Ma[i][j][:, rows] @ Gij)
                    sigma[rows] += 0.5 * (self.Mb[i][j] @ Gij.T).T
        return sigma
