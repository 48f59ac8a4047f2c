"""Pins for the oracle Hamiltonian and sigma: brute force, Slater-Condon, S^2."""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import slater_condon as sc
from oracle import sigma as sg
from oracle import spin


def _systems_small():
    return [
        ("H2", inputs.h_chain(2, 0.74), 1, 1),
        ("H4", inputs.h_chain(4, 1.0), 2, 2),
        ("rand4_21", inputs.random_df(4, 7), 2, 1),
        ("rand4_13", inputs.random_df(4, 8), 1, 3),
    ]


@pytest.mark.parametrize("name,I,na,nb", _systems_small())
def test_slater_condon_equals_brute_force_operator(name, I, na, nb):
    Hb = sc.brute_force_hamiltonian(I.h1, I.eri, na, nb)
    Hs = sc.dense_hamiltonian(I.h1, I.eri, na, nb)
    assert np.abs(Hb - Hs).max() < 1e-12
    assert np.abs(Hs - Hs.T).max() == 0.0


@pytest.mark.parametrize("I,na,nb", [
    (inputs.h_chain(4, 1.0), 2, 2),
    (inputs.h_chain(6, 1.0), 3, 3),
    (inputs.random_df(5, 11), 3, 2),
    (inputs.random_df(6, 12), 2, 3),
])
def test_string_sigma_equals_dense(I, na, nb):
    H = sc.dense_hamiltonian(I.h1, I.eri, na, nb)
    sig = sg.StringSigma(I.h1, I.eri, na, nb)
    rng = np.random.default_rng(1)
    for _ in range(3):
        c = rng.standard_normal((sig.Na, sig.Nb))
        ref = H @ c.reshape(-1)
        out = sig.apply(c).reshape(-1)
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


def test_blocked_sigma_equals_full():
    I = inputs.random_df(7, 5)
    sig = sg.StringSigma(I.h1, I.eri, 4, 3, block_rows=7)
    c = inputs.random_vector(sig.Na, sig.Nb, 2)
    a = sig._apply_full(c)
    b = sig._apply_blocked(c)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_hermiticity_and_diagonal():
    I = inputs.h_chain(8, 1.3)
    sig = sg.StringSigma(I.h1, I.eri, 4, 4)
    u = inputs.random_vector(70, 70, 3)
    v = inputs.random_vector(70, 70, 4)
    a = u.reshape(-1) @ sig.apply(v).reshape(-1)
    b = sig.apply(u).reshape(-1) @ v.reshape(-1)
    assert abs(a - b) < 1e-12 * max(abs(a), 1.0)
    d1 = sc.diagonal_by_occupation(I.h1, I.eri, 4, 4)
    rows = list(range(0, 4900, 97))
    e = np.zeros(4900)
    for r in rows:
        e[:] = 0.0
        e[r] = 1.0
        assert abs(sig.apply(e.reshape(70, 70)).reshape(-1)[r] - d1[r]) < 1e-12
    I6 = inputs.random_df(6, 9)
    assert np.abs(sc.diagonal(I6.h1, I6.eri, 3, 2) - sc.diagonal_by_occupation(I6.h1, I6.eri, 3, 2)).max() < 1e-12


def test_sampled_rows_equal_string_sigma():
    I = inputs.random_df(8, 21)
    sig = sg.StringSigma(I.h1, I.eri, 4, 4)
    c = inputs.random_vector(70, 70, 5)
    full = sig.apply(c).reshape(-1)
    rows = np.random.default_rng(0).choice(4900, 40, replace=False)
    samp = sc.sampled_sigma_rows(I.h1, I.eri, 4, 4, c, rows)
    assert np.abs(samp - full[rows]).max() < 1e-12 * np.abs(full).max()


def test_s_squared_of_eigenvectors():
    I = inputs.h_chain(4, 1.5)
    H = sc.dense_hamiltonian(I.h1, I.eri, 2, 2)
    w, V = np.linalg.eigh(H)
    for j in range(V.shape[1]):
        s2 = spin.s_squared(V[:, j], 4, 2, 2)
        S = round((-1 + np.sqrt(1 + 4 * s2)) / 2 * 2) / 2
        # degenerate multiplets mix; only check when the level is isolated
        if (j == 0 or w[j] - w[j - 1] > 1e-8) and (j == len(w) - 1 or w[j + 1] - w[j] > 1e-8):
            assert abs(s2 - S * (S + 1)) < 1e-8
    # H2 triplet (Sz = 0 component) and singlet ground state
    I2 = inputs.h_chain(2, 0.74)
    H2 = sc.dense_hamiltonian(I2.h1, I2.eri, 1, 1)
    w2, V2 = np.linalg.eigh(H2)
    assert abs(spin.s_squared(V2[:, 0], 2, 1, 1)) < 1e-10
    s2s = sorted(spin.s_squared(V2[:, j], 2, 1, 1) for j in range(4))
    assert np.allclose(s2s, [0, 0, 0, 2], atol=1e-10)
    # a single high-spin determinant: Sz = 1 -> S^2 = 2
    e = np.zeros(6)
    e[0] = 1.0
    assert abs(spin.s_squared(e, 4, 3, 1) - 2.0) < 1e-12


def test_transpose_symmetric_sector_is_even_spin():
    """c = c^T vectors of the H4 ground/excited singlets: the eigenvectors that
    are transpose-symmetric have S^2 in {0, 6}, antisymmetric ones S^2 = 2."""
    I = inputs.h_chain(4, 1.2)
    H = sc.dense_hamiltonian(I.h1, I.eri, 2, 2)
    w, V = np.linalg.eigh(H)
    for j in range(V.shape[1]):
        isolated = (j == 0 or w[j] - w[j - 1] > 1e-8) and (j == len(w) - 1 or w[j + 1] - w[j] > 1e-8)
        if not isolated:
            continue
        m = V[:, j].reshape(6, 6)
        s2 = spin.s_squared(V[:, j], 4, 2, 2)
        if np.abs(m - m.T).max() < 1e-10:
            assert min(abs(s2), abs(s2 - 6)) < 1e-8
        elif np.abs(m + m.T).max() < 1e-10:
            assert abs(s2 - 2) < 1e-8


def test_planted_sign_error_is_caught():
    """A flipped sign in one excitation entry must break sigma == dense H."""
    I = inputs.h_chain(4, 1.0)
    H = sc.dense_hamiltonian(I.h1, I.eri, 2, 2)
    sig = sg.StringSigma(I.h1, I.eri, 2, 2)
    M = sig.Ma[1][0].tolil()
    r, c = M.nonzero()
    M[r[0], c[0]] = -M[r[0], c[0]]
    sig.Ma[1][0] = M.tocsr()
    v = inputs.random_vector(6, 6, 0)
    assert np.abs(sig.apply(v).reshape(-1) - H @ v.reshape(-1)).max() > 1e-6
