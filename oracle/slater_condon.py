"""Determinant-pair matrix elements of H (oracle; test infrastructure only).

Independent of ``oracle.sigma``: this module never uses string excitation
lists.  A determinant is a bitmask over 2n spin orbitals, alpha orbital p at
bit p and beta orbital q at bit n+q, and it stands for the product of creators
in ascending spin-orbital order (all alpha creators left of all beta ones,
the determinant convention of ``oracle.strings``).

Spin-orbital integrals from the spatial ones:
  h_so[p, q] = h[p mod n, q mod n] if spin(p) == spin(q) else 0,
  <pq|rs>    = (pr|qs) if spin(p)==spin(r) and spin(q)==spin(s) else 0.

The Hamiltonian is H = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs <pq|rs> a+_p a+_q a_s a_r
(+ e_core, which these routines leave out).  The paper's H "represented in
terms of Slater determinants" (Results, SBCI1 algorithm) is this matrix.
"""
from __future__ import annotations

import numpy as np

from .strings import enumerate_strings


def _bits(mask: int, nbits: int) -> list[int]:
    return [p for p in range(nbits) if (mask >> p) & 1]


def _annihilate(mask: int, p: int):
    if not (mask >> p) & 1:
        return None
    sign = -1 if bin(mask & ((1 << p) - 1)).count("1") % 2 else 1
    return sign, mask & ~(1 << p)


def _create(mask: int, p: int):
    if (mask >> p) & 1:
        return None
    sign = -1 if bin(mask & ((1 << p) - 1)).count("1") % 2 else 1
    return sign, mask | (1 << p)


def apply_ops(mask: int, ops):
    """Apply a product of operators right-to-left.

    ``ops`` is a sequence of (kind, p), kind '+' (create) or '-' (annihilate),
    written left to right as in the operator product.  Returns (sign, mask) or
    None if the result vanishes.
    """
    sign = 1
    for kind, p in reversed(ops):
        r = _create(mask, p) if kind == "+" else _annihilate(mask, p)
        if r is None:
            return None
        s, mask = r
        sign *= s
    return sign, mask


class SpinOrbitalHamiltonian:
    """Spin-orbital view of (h1, eri) for 2n spin orbitals."""

    def __init__(self, h1: np.ndarray, eri: np.ndarray):
        self.n = h1.shape[0]
        self.h1 = np.asarray(h1, dtype=np.float64)
        self.eri = np.asarray(eri, dtype=np.float64)

    def spin(self, p: int) -> int:
        return p // self.n

    def h(self, p: int, q: int) -> float:
        if self.spin(p) != self.spin(q):
            return 0.0
        return float(self.h1[p % self.n, q % self.n])

    def g(self, p: int, q: int, r: int, s: int) -> float:
        """Physicists' <pq|rs> = (pr|qs) with spin selection."""
        if self.spin(p) != self.spin(r) or self.spin(q) != self.spin(s):
            return 0.0
        n = self.n
        return float(self.eri[p % n, r % n, q % n, s % n])


def determinants(norb: int, nalpha: int, nbeta: int) -> list[int]:
    """Spin-orbital masks in flat order Ia * Nb + Ib (the CI-vector order)."""
    sa = enumerate_strings(norb, nalpha)
    sb = enumerate_strings(norb, nbeta)
    return [int(a) | (int(b) << norb) for a in sa for b in sb]


def matrix_element(so: SpinOrbitalHamiltonian, bra: int, ket: int) -> float:
    """<bra|H|ket> by the Slater-Condon rules (no e_core)."""
    nb = 2 * so.n
    diff = bra ^ ket
    ndiff = bin(diff).count("1")
    if ndiff == 0:
        occ = _bits(ket, nb)
        e = sum(so.h(p, p) for p in occ)
        for p in occ:
            for q in occ:
                e += 0.5 * (so.g(p, q, p, q) - so.g(p, q, q, p))
        return e
    if ndiff == 2:
        p = _bits(ket & diff, nb)[0]  # in ket only
        r = _bits(bra & diff, nb)[0]  # in bra only
        res = apply_ops(ket, [("+", r), ("-", p)])
        sign = res[0]
        val = so.h(r, p)
        for q in _bits(ket, nb):
            val += so.g(r, q, p, q) - so.g(r, q, q, p)
        return sign * val
    if ndiff == 4:
        p, q = _bits(ket & diff, nb)
        r, s = _bits(bra & diff, nb)
        res = apply_ops(ket, [("+", r), ("+", s), ("-", q), ("-", p)])
        sign = res[0]
        return sign * (so.g(r, s, p, q) - so.g(r, s, q, p))
    return 0.0


def dense_hamiltonian(h1, eri, nalpha: int, nbeta: int) -> np.ndarray:
    """Dense H over all determinants (Slater-Condon), flat Ia*Nb+Ib order."""
    so = SpinOrbitalHamiltonian(h1, eri)
    dets = determinants(so.n, nalpha, nbeta)
    N = len(dets)
    H = np.zeros((N, N))
    for i in range(N):
        for j in range(i, N):
            if bin(dets[i] ^ dets[j]).count("1") <= 4:
                v = matrix_element(so, dets[i], dets[j])
                H[i, j] = v
                H[j, i] = v
    return H


def diagonal(h1, eri, nalpha: int, nbeta: int) -> np.ndarray:
    """D_I = H_II for every determinant (the preconditioner's D, Eq. 6-7)."""
    so = SpinOrbitalHamiltonian(h1, eri)
    return np.array([matrix_element(so, d, d) for d in determinants(so.n, nalpha, nbeta)])


def connected(so: SpinOrbitalHamiltonian, ket: int):
    """Every determinant within a double excitation of ``ket`` (including itself)."""
    nb = 2 * so.n
    occ = _bits(ket, nb)
    vir = [p for p in range(nb) if not (ket >> p) & 1]
    out = [ket]
    for p in occ:
        for r in vir:
            if so.spin(p) == so.spin(r):
                out.append(ket ^ (1 << p) ^ (1 << r))
    for i, p in enumerate(occ):
        for q in occ[i + 1:]:
            for j, r in enumerate(vir):
                for s in vir[j + 1:]:
                    if so.spin(p) + so.spin(q) == so.spin(r) + so.spin(s):
                        out.append(ket ^ (1 << p) ^ (1 << q) ^ (1 << r) ^ (1 << s))
    return out


def sampled_sigma_rows(h1, eri, nalpha: int, nbeta: int, c: np.ndarray, rows):
    """sigma_I = sum_J H_IJ c_J for the flat determinant indices ``rows``.

    Enumerates every J connected to I by at most a double excitation and uses
    the Slater-Condon element; independent of the string-driven sigma.
    """
    so = SpinOrbitalHamiltonian(h1, eri)
    n = so.n
    sa = enumerate_strings(n, nalpha)
    sb = enumerate_strings(n, nbeta)
    ra = {int(m): i for i, m in enumerate(sa)}
    rb = {int(m): i for i, m in enumerate(sb)}
    Nb = len(sb)
    cf = np.asarray(c).reshape(-1)
    out = np.zeros(len(rows))
    lowmask = (1 << n) - 1
    for t, I in enumerate(rows):
        ia, ib = divmod(int(I), Nb)
        bra = int(sa[ia]) | (int(sb[ib]) << n)
        acc = 0.0
        for ket in connected(so, bra):
            J = ra[ket & lowmask] * Nb + rb[ket >> n]
            acc += matrix_element(so, bra, ket) * cf[J]
        out[t] = acc
    return out


def brute_force_hamiltonian(h1, eri, nalpha: int, nbeta: int) -> np.ndarray:
    """Dense H by applying every term of the second-quantised H operator.

    O(Ndet * (2n)^4); meant for n <= 4 only, as the pin of the Slater-Condon
    rules above.
    """
    so = SpinOrbitalHamiltonian(h1, eri)
    nb = 2 * so.n
    dets = determinants(so.n, nalpha, nbeta)
    index = {d: i for i, d in enumerate(dets)}
    N = len(dets)
    H = np.zeros((N, N))
    for j, ket in enumerate(dets):
        for p in range(nb):
            for q in range(nb):
                v = so.h(p, q)
                if v == 0.0:
                    continue
                res = apply_ops(ket, [("+", p), ("-", q)])
                if res is not None:
                    H[index[res[1]], j] += v * res[0]
        for p in range(nb):
            for q in range(nb):
                for r in range(nb):
                    for s in range(nb):
                        v = so.g(p, q, r, s)
                        if v == 0.0:
                            continue
                        res = apply_ops(ket, [("+", p), ("+", q), ("-", s), ("-", r)])
                        if res is not None:
                            H[index[res[1]], j] += 0.5 * v * res[0]
    return H


def diagonal_by_occupation(h1, eri, nalpha: int, nbeta: int) -> np.ndarray:
    """The Slater-Condon diagonal summed per spin block, for large spaces.

    For occupations a (alpha) and b (beta) of determinant I:
      H_II = sum_{p in a} h_pp + sum_{p in b} h_pp
             + 1/2 sum_{p,q in a} [(pp|qq) - (pq|qp)] + 1/2 sum_{p,q in b} [(pp|qq) - (pq|qp)]
             + sum_{p in a, q in b} (pp|qq)
    which is the ndiff == 0 rule of ``matrix_element`` with the spin
    selection carried out.  Returns the flat [Na*Nb] vector.
    """
    n = h1.shape[0]
    sa = enumerate_strings(n, nalpha)
    sb = enumerate_strings(n, nbeta)
    occa = ((sa[:, None] >> np.arange(n)) & 1).astype(np.float64)
    occb = ((sb[:, None] >> np.arange(n)) & 1).astype(np.float64)
    J = np.einsum("ppqq->pq", eri)
    K = np.einsum("pqqp->pq", eri)
    hd = np.diag(h1)
    ea = occa @ hd + 0.5 * np.einsum("ip,pq,iq->i", occa, J - K, occa)
    eb = occb @ hd + 0.5 * np.einsum("ip,pq,iq->i", occb, J - K, occb)
    eab = occa @ J @ occb.T
    return (ea[:, None] + eb[None, :] + eab).reshape(-1)
