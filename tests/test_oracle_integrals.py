"""Pins for the synthetic integral inputs (textbook values, symmetry, invariance)."""
import json
import os

import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import slater_condon as sc
from oracle import sigma as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_h2_ao_integrals_match_szabo_ostlund():
    g = _load("h2_sto3g_szabo_ostlund.json")
    tol = g["tolerance"]
    S, T, V, eri, e_nuc = inputs.sto3g_chain_ao_integrals(np.array([[0, 0, 0], [0, 0, g["R_bohr"]]]))
    H = T + V
    assert abs(S[0, 0] - 1.0) < 1e-14
    assert abs(S[0, 1] - g["S12"]) < tol
    assert abs(T[0, 0] - g["T11"]) < tol
    assert abs(T[0, 1] - g["T12"]) < tol
    assert abs(V[0, 0] - g["V_total_11"]) < tol
    assert abs(V[0, 1] - g["V_total_12"]) < tol
    assert abs(H[0, 0] - g["Hcore11"]) < tol
    assert abs(H[0, 1] - g["Hcore12"]) < tol
    assert abs(eri[0, 0, 0, 0] - g["eri_1111"]) < tol
    assert abs(eri[0, 0, 1, 1] - g["eri_1122"]) < tol
    assert abs(eri[1, 0, 0, 0] - g["eri_2111"]) < tol
    assert abs(eri[1, 0, 1, 0] - g["eri_2121"]) < tol
    assert abs(e_nuc - g["E_nuc"]) < tol


def test_h_atom_energy():
    g = _load("h_atom_sto3g.json")
    S, T, V, eri, e_nuc = inputs.sto3g_chain_ao_integrals(np.zeros((1, 3)))
    assert abs(T[0, 0] + V[0, 0] - g["E_H_atom"]) < g["tolerance"]


def _h2_closed_form(S, Hc, eri_ao, e_nuc):
    """Minimal-basis H2 FCI in the sigma_g / sigma_u MOs: a 2x2 CI problem.

    psi_1 = (phi_1 + phi_2)/sqrt(2(1+S)), psi_2 = (phi_1 - phi_2)/sqrt(2(1-S));
    the CI matrix between |1a 1b> and |2a 2b> is
    [[2 h11 + J11, K12], [K12, 2 h22 + J22]] and its lowest root is
    (H11 + H22)/2 - sqrt(((H22 - H11)/2)^2 + K12^2).
    """
    s = S[0, 1]
    C = np.array([[1, 1], [1, -1]]) / np.sqrt(np.array([2 * (1 + s), 2 * (1 - s)]))
    h = C.T @ Hc @ C
    mo = np.einsum("pi,qj,rk,sl,pqrs->ijkl", C, C, C, C, eri_ao)
    H11 = 2 * h[0, 0] + mo[0, 0, 0, 0]
    H22 = 2 * h[1, 1] + mo[1, 1, 1, 1]
    K = mo[0, 1, 1, 0]
    e_hf = H11 + e_nuc
    e_fci = 0.5 * (H11 + H22) - np.sqrt(0.25 * (H22 - H11) ** 2 + K * K) + e_nuc
    return e_hf, e_fci


def test_h2_fci_closed_form_and_textbook():
    g = _load("h2_sto3g_szabo_ostlund.json")
    S, T, V, eri_ao, e_nuc = inputs.sto3g_chain_ao_integrals(np.array([[0, 0, 0], [0, 0, g["R_bohr"]]]))
    e_hf, e_fci = _h2_closed_form(S, T + V, eri_ao, e_nuc)
    assert abs(e_hf - g["E_HF_total"]) < g["tolerance"]
    assert abs(e_fci - g["E_FCI_total"]) < g["tolerance"]
    I = inputs.h_chain(2, g["R_bohr"] * inputs.BOHR_ANGSTROM)
    H = sc.dense_hamiltonian(I.h1, I.eri, 1, 1)
    assert abs(np.linalg.eigvalsh(H)[0] + I.e_core - e_fci) < 1e-12
    sig = sg.StringSigma(I.h1, I.eri, 1, 1)
    Hs = np.column_stack([sig.apply(e.reshape(2, 2)).reshape(-1) for e in np.eye(4)])
    assert abs(np.linalg.eigvalsh(Hs)[0] + I.e_core - e_fci) < 1e-12


@pytest.mark.parametrize("make", [lambda: inputs.h_chain(6, 1.0), lambda: inputs.random_df(6, 3)])
def test_eri_eightfold_symmetry(make):
    I = make()
    e = I.eri
    for perm in ["jikl", "ijlk", "jilk", "klij", "lkij", "klji", "lkji"]:
        assert np.abs(e - np.einsum("ijkl->" + perm, e)).max() < 1e-13
    assert np.abs(I.h1 - I.h1.T).max() == 0.0


def test_random_df_psd_and_seeded():
    I = inputs.random_df(8, 14)
    n = I.norb
    w = np.linalg.eigvalsh(I.eri.reshape(n * n, n * n))
    assert w.min() > -1e-12
    J = inputs.random_df(8, 14)
    assert np.array_equal(I.eri, J.eri) and np.array_equal(I.h1, J.h1)
    K = inputs.random_df(8, 15)
    assert not np.array_equal(I.h1, K.h1)
    d = np.diag(I.h1)
    assert abs(d.mean() + 2.0) < 1.0


def test_fci_energy_invariant_under_orbital_rotation():
    """FCI is exact within the orbital space: any orthogonal rotation of the
    orbitals leaves the spectrum unchanged (Loewdin vs canonical MOs)."""
    I = inputs.h_chain(4, 1.1)
    H = sc.dense_hamiltonian(I.h1, I.eri, 2, 2)
    _, C = np.linalg.eigh(I.h1)  # a canonical-like basis
    h2 = C.T @ I.h1 @ C
    e2 = np.einsum("pi,qj,rk,sl,pqrs->ijkl", C, C, C, C, I.eri)
    H2 = sc.dense_hamiltonian(h2, e2, 2, 2)
    assert np.abs(np.linalg.eigvalsh(H) - np.linalg.eigvalsh(H2)).max() < 1e-10
