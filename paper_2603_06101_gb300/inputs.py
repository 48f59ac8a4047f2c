"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the SBCI method or of the sigma build: it
only produces the *problem data* that the method starts from (one- and
two-electron integrals, initial vectors, serving traces).  The paper takes
these from PySCF (Materials and Methods); here they are synthetic stand-ins
with the structure of the paper's workloads:

* hydrogen chains in the STO-3G minimal basis, Loewdin-orthonormalised
  (closed-form s-type Gaussian integrals, Boys F0);
* random density-fitted integrals (ij|kl) = sum_P B^P_ij B^P_kl, which are
  8-fold symmetric and positive semidefinite as a pair matrix;
* Gaussian random CI vectors;
* a Poisson serving trace over hydrogen chains.

Integral conventions: ``h1[i, j]`` is the core Hamiltonian, ``eri[i, j, k, l]``
is the chemists'-notation integral (ij|kl), real orbitals, ``e_core`` is the
nuclear repulsion (0 for the random model).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

#: CODATA 2018 Bohr radius in Angstrom.
BOHR_ANGSTROM = 0.529177210903

# STO-3G contraction of a Slater 1s function with exponent zeta = 1.24
# (Hehre, Stewart, Pople, J. Chem. Phys. 51, 2657 (1969)): Gaussian exponents
# already scaled by zeta^2, and contraction coefficients that multiply
# normalised primitives.
STO3G_H_EXPONENTS = (3.42525091, 0.62391373, 0.16885540)
STO3G_H_COEFFS = (0.15432897, 0.53532814, 0.44463454)


def boys_f0(t):
    """Boys function of order zero, F0(t) = 1/2 sqrt(pi/t) erf(sqrt(t)), F0(0)=1."""
    from scipy.special import erf

    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    big = t > 1e-12
    out[big] = 0.5 * np.sqrt(np.pi / t[big]) * erf(np.sqrt(t[big]))
    small = ~big
    out[small] = 1.0 - t[small] / 3.0  # leading terms of the series at t -> 0
    return out


def _prim_norm(a):
    return (2.0 * a / np.pi) ** 0.75


def sto3g_chain_ao_integrals(centres_bohr):
    """AO integrals for one STO-3G 1s function per hydrogen at ``centres_bohr``.

    Closed forms for s-type primitive Gaussians (Szabo & Ostlund, Appendix A):
    overlap, kinetic, nuclear attraction and electron repulsion, the last two
    through F0.  Returns (S, T, V, eri_ao, e_nuc), all float64.
    """
    R = np.asarray(centres_bohr, dtype=np.float64).reshape(-1, 3)
    nat = R.shape[0]
    a = np.array(STO3G_H_EXPONENTS)
    d = np.array(STO3G_H_COEFFS) * _prim_norm(a)
    # renormalise the contraction so that S_ii = 1 exactly
    ap = a[:, None] + a[None, :]
    d = d / np.sqrt((d[:, None] * d[None, :] * (np.pi / ap) ** 1.5).sum())
    npr = a.size
    # primitive index f = A*npr + p  (centre A, primitive p)
    ex = np.tile(a, nat)
    cf = np.tile(d, nat)
    cen = np.repeat(R, npr, axis=0)
    nf = ex.size
    g = ex[:, None] + ex[None, :]
    mu = ex[:, None] * ex[None, :] / g
    r2 = ((cen[:, None, :] - cen[None, :, :]) ** 2).sum(-1)
    kab = np.exp(-mu * r2)
    P = (ex[:, None, None] * cen[:, None, :] + ex[None, :, None] * cen[None, :, :]) / g[..., None]
    dd = cf[:, None] * cf[None, :]
    s_p = (np.pi / g) ** 1.5 * kab
    t_p = mu * (3.0 - 2.0 * mu * r2) * s_p
    v_p = np.zeros_like(s_p)
    for C in range(nat):
        rpc2 = ((P - R[C]) ** 2).sum(-1)
        v_p += -2.0 * np.pi / g * kab * boys_f0(g * rpc2)

    def contract2(x):
        return (dd * x).reshape(nat, npr, nat, npr).sum(axis=(1, 3))

    S, T, V = contract2(s_p), contract2(t_p), contract2(v_p)
    # electron repulsion over primitive pairs (f1,f2) x (f3,f4)
    gp = g.reshape(-1)
    Pp = P.reshape(-1, 3)
    kp = (kab * dd).reshape(-1)
    g1 = gp[:, None]
    g2 = gp[None, :]
    rpq2 = ((Pp[:, None, :] - Pp[None, :, :]) ** 2).sum(-1)
    val = 2.0 * np.pi ** 2.5 / (g1 * g2 * np.sqrt(g1 + g2)) * kp[:, None] * kp[None, :] \
        * boys_f0(g1 * g2 / (g1 + g2) * rpq2)
    eri = val.reshape(nat, npr, nat, npr, nat, npr, nat, npr).sum(axis=(1, 3, 5, 7))
    e_nuc = 0.0
    for A in range(nat):
        for B in range(A):
            e_nuc += 1.0 / float(np.sqrt(((R[A] - R[B]) ** 2).sum()))
    return S, T, V, eri, e_nuc


def lowdin_transform(S, hcore, eri_ao):
    """Transform AO integrals to the symmetric (Loewdin) orthonormal basis S^-1/2."""
    w, U = np.linalg.eigh(S)
    X = (U * (1.0 / np.sqrt(w))) @ U.T
    h = X.T @ hcore @ X
    eri = np.einsum("pi,qj,rk,sl,pqrs->ijkl", X, X, X, X, eri_ao, optimize=True)
    # restore the exact symmetries that rounding in the transform breaks
    h = 0.5 * (h + h.T)
    eri = 0.5 * (eri + eri.transpose(1, 0, 2, 3))
    eri = 0.5 * (eri + eri.transpose(0, 1, 3, 2))
    eri = 0.5 * (eri + eri.transpose(2, 3, 0, 1))
    return h, eri


@dataclass
class Integrals:
    """One- and two-electron integrals of an active space."""

    norb: int
    nalpha: int
    nbeta: int
    h1: np.ndarray  # [n, n]
    eri: np.ndarray  # [n, n, n, n], (ij|kl)
    e_core: float
    label: str = ""


def h_chain(natoms: int, spacing_angstrom: float, nalpha: int | None = None,
            nbeta: int | None = None) -> Integrals:
    """Linear H_n chain on the z axis, STO-3G, Loewdin basis, S_z = 0 by default."""
    R = spacing_angstrom / BOHR_ANGSTROM
    centres = np.zeros((natoms, 3))
    centres[:, 2] = np.arange(natoms) * R
    S, T, V, eri_ao, e_nuc = sto3g_chain_ao_integrals(centres)
    h, eri = lowdin_transform(S, T + V, eri_ao)
    na = natoms // 2 if nalpha is None else nalpha
    nb = natoms - na if nbeta is None else nbeta
    return Integrals(natoms, na, nb, np.ascontiguousarray(h), np.ascontiguousarray(eri),
                     float(e_nuc), f"H{natoms} R={spacing_angstrom:g}A")


def random_df(norb: int, seed: int, nalpha: int | None = None,
              nbeta: int | None = None, naux: int | None = None) -> Integrals:
    """Random density-fitted model Hamiltonian.

    Draw order from ``numpy.random.default_rng(seed)``:
    1. h diagonal, n values ~ N(-2, 0.5)  (second argument: standard deviation);
    2. h strict upper triangle, row-major, n(n-1)/2 values ~ N(0, 0.1), mirrored;
    3. B[P, i<=j] for P < naux (default 3n), upper triangle row-major,
       ~ N(0, 0.05), mirrored.
    (ij|kl) = sum_P B[P,i,j] B[P,k,l]; e_core = 0.
    """
    rng = np.random.default_rng(seed)
    n = norb
    naux = 3 * n if naux is None else naux
    h = np.zeros((n, n))
    h[np.diag_indices(n)] = rng.normal(-2.0, 0.5, size=n)
    iu = np.triu_indices(n, 1)
    off = rng.normal(0.0, 0.1, size=iu[0].size)
    h[iu] = off
    h[(iu[1], iu[0])] = off
    iu0 = np.triu_indices(n, 0)
    B = np.zeros((naux, n, n))
    vals = rng.normal(0.0, 0.05, size=(naux, iu0[0].size))
    B[:, iu0[0], iu0[1]] = vals
    B[:, iu0[1], iu0[0]] = vals
    eri = np.einsum("pij,pkl->ijkl", B, B, optimize=True)
    na = n // 2 if nalpha is None else nalpha
    nb = n - na if nbeta is None else nbeta
    return Integrals(n, na, nb, h, np.ascontiguousarray(eri), 0.0, f"randDF n={n} seed={seed}")


def random_vector(n_alpha_strings: int, n_beta_strings: int, seed: int,
                  normalise: bool = True) -> np.ndarray:
    """Gaussian CI vector c[Ia, Ib] ~ N(0,1) in flat row-major order."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((n_alpha_strings, n_beta_strings))
    if normalise:
        c /= np.linalg.norm(c)
    return c


def n_strings(norb: int, nelec: int) -> int:
    return math.comb(norb, nelec)


@dataclass
class Request:
    """One solve of the serving stream."""

    arrival_s: float
    natoms: int
    spacing_angstrom: float
    nstates: int


def serving_trace(n_requests: int = 256, seed: int = 4, rate_per_s: float = 100.0,
                  sizes=(6, 8, 10, 12), spacing=(0.7, 3.0), states=(1, 4)):
    """Poisson arrivals over hydrogen chains.

    Draw order from ``default_rng(seed)``: exponential inter-arrival gaps
    (mean 1/rate), chain size uniform over ``sizes``, spacing ~ U(spacing),
    number of states uniform over the inclusive range ``states``.
    ``rate_per_s = inf`` puts every arrival at t = 0 (saturation run).
    """
    rng = np.random.default_rng(seed)
    if math.isinf(rate_per_s):
        gaps = np.zeros(n_requests)
        rng.exponential(1.0, size=n_requests)  # keep later draws aligned
    else:
        gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    arr = np.cumsum(gaps) - gaps[0]
    nat = rng.choice(np.asarray(sizes), size=n_requests)
    sp = rng.uniform(spacing[0], spacing[1], size=n_requests)
    ns = rng.integers(states[0], states[1] + 1, size=n_requests)
    return [Request(float(arr[i]), int(nat[i]), float(sp[i]), int(ns[i]))
            for i in range(n_requests)]
