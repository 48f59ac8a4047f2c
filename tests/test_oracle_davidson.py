"""Pins for the oracle block Davidson-Liu solver (the method the paper compares
SBCI with): exact energies from dense and Lanczos eigen-solvers, the Ritz
property, the transpose-symmetric sector, the collapse path, and a space
smaller than the subspace limit."""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import davidson, eigen, spin
from oracle import slater_condon as sc
from oracle import sigma as sg


@pytest.fixture(scope="module")
def h6():
    I = inputs.h_chain(6, 1.0)
    sig = sg.StringSigma(I.h1, I.eri, 3, 3)
    H = sc.dense_hamiltonian(I.h1, I.eri, 3, 3)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 3, 3)
    return I, sig, H, D


def test_lowest_four_equal_dense_eigh(h6):
    I, sig, H, D = h6
    w = np.linalg.eigvalsh(H)
    res = davidson.davidson_liu(sig.apply, D, (20, 20), 4, eps0=1e-12, r0=1e-8, max_space=200)
    assert res.converged
    assert np.abs(res.energies - w[:4]).max() < 1e-11
    X = res.vectors
    assert np.abs(X.T @ X - np.eye(4)).max() < 1e-10
    # Ritz property on the dense matrix, independent of the string sigma
    for a in range(4):
        assert np.linalg.norm(H @ X[:, a] - res.energies[a] * X[:, a]) < 1e-8
    # without a collapse every subspace vector cost one H-product
    assert res.n_collapse == 0 and res.n_sigma == res.trace[-1][0]


def test_default_thresholds_reach_1e8(h6):
    """With the SBCI thresholds (eps0 = 1e-10, r0 = 1e-5) the energies are within
    |r|^2 / gap of the exact ones."""
    I, sig, H, D = h6
    w = np.linalg.eigvalsh(H)
    res = davidson.davidson_liu(sig.apply, D, (20, 20), 3)
    assert res.converged and np.all(res.residuals < 1e-5)
    assert np.abs(res.energies - w[:3]).max() < 1e-8


def test_sector_equals_symmetric_subspace_eigh(h6):
    """sector = 1: the lowest states among vectors with c = c^T, pinned by eigh of
    H restricted to an orthonormal basis of that subspace; <S^2> of every state
    is even (0, 2, 6, ...)."""
    I, sig, H, D = h6
    n = 20
    cols = []
    for a in range(n):
        for b in range(a, n):
            v = np.zeros((n, n))
            if a == b:
                v[a, a] = 1.0
            else:
                v[a, b] = v[b, a] = 1.0 / np.sqrt(2.0)
            cols.append(v.reshape(-1))
    B = np.column_stack(cols)
    ws = np.linalg.eigvalsh(B.T @ H @ B)
    res = davidson.davidson_liu(sig.apply, D, (n, n), 4, sector=True, eps0=1e-12, r0=1e-8)
    assert res.converged
    assert np.abs(res.energies - ws[:4]).max() < 1e-11
    for a in range(4):
        x = res.vectors[:, a].reshape(n, n)
        assert np.abs(x - x.T).max() < 1e-12
        s2 = spin.s_squared(x, 6, 3, 3)
        S = (-1.0 + np.sqrt(1.0 + 4.0 * s2)) / 2.0
        assert abs(S - round(S)) < 1e-6 and round(S) % 2 == 0


def test_collapse_path_same_energies(h6):
    I, sig, H, D = h6
    w = np.linalg.eigvalsh(H)
    res = davidson.davidson_liu(sig.apply, D, (20, 20), 3, max_space=6, eps0=1e-12, r0=1e-8)
    assert res.converged and res.n_collapse > 0
    assert np.abs(res.energies - w[:3]).max() < 1e-11
    assert max(m for m, _, _ in res.trace) <= 6


def test_whole_space_smaller_than_subspace():
    """H2 (4 determinants): the subspace reaches the whole space, every
    correction is then dropped, and the Ritz values are the exact eigenvalues."""
    I = inputs.h_chain(2, 0.74)
    sig = sg.StringSigma(I.h1, I.eri, 1, 1)
    H = sc.dense_hamiltonian(I.h1, I.eri, 1, 1)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 1, 1)
    res = davidson.davidson_liu(sig.apply, D, (2, 2), 2, max_space=8)
    assert res.converged
    assert np.abs(res.energies - np.linalg.eigvalsh(H)[:2]).max() < 1e-12
    assert res.n_sigma <= 4


def test_h8_against_lanczos():
    I = inputs.h_chain(8, 1.3)
    sig = sg.StringSigma(I.h1, I.eri, 4, 4)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 4, 4)
    wl, _ = eigen.lowest_lanczos(sig.apply, sig.ndet, 3)
    res = davidson.davidson_liu(sig.apply, D, (70, 70), 3, eps0=1e-12, r0=1e-8)
    assert res.converged
    assert np.abs(res.energies - wl).max() < 1e-10


def test_start_vectors_fill_k_in_sector():
    """D1 in the sector: swapped determinant pairs give one vector, so more
    determinants than k are read until k vectors exist."""
    D = np.array([0.0, 1.0, 1.0, 2.0])  # 2 x 2 space: (0,0), (0,1), (1,0), (1,1)
    V = davidson.start_vectors(D, (2, 2), 3, sector=True)
    assert len(V) == 3
    M = np.column_stack(V)
    assert np.abs(M.T @ M - np.eye(3)).max() < 1e-15
    assert np.allclose(V[1], [0.0, np.sqrt(0.5), np.sqrt(0.5), 0.0])
    with pytest.raises(ValueError):
        davidson.start_vectors(D, (2, 2), 4, sector=True)
