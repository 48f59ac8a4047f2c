"""Pins for the oracle SBCI2 (Algorithm 2, Sections S2.1-S2.5): exact energies
in both sectors, the Ritz property of every step checked on the dense
Hamiltonian, the coefficient formulas checked against the update rule they
were solved from (Eq. S111), and the H-image drift."""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import sbci, sbci2
from oracle import slater_condon as sc
from oracle import sigma as sg


@pytest.fixture(scope="module")
def h6():
    I = inputs.h_chain(6, 1.0)
    sig = sg.StringSigma(I.h1, I.eri, 3, 3)
    H = sc.dense_hamiltonian(I.h1, I.eri, 3, 3)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 3, 3)
    return I, sig, H, D


def _sector_eigs(H, n):
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
    return np.linalg.eigvalsh(B.T @ H @ B)


class StepChecks:
    """Per-step checks on the dense H, independent of the string sigma."""

    def __init__(self, H):
        self.H = H
        self.n = 0
        self.worst = {"ritz": 0.0, "update": 0.0, "knorm": 0.0, "drift": 0.0, "energy": 0.0,
                      "ritz_all": 0.0, "exact_steps": 0}

    def __call__(self, d):
        H = self.H
        self.n += 1
        Bm = np.column_stack(d["basis"])
        # the span the step works in: overlap eigenvectors with eigenvalue >= 1e-14
        # (Eqs. S83, S103), orthonormalised; then the two lowest Ritz pairs of the
        # dense H in it
        sv, Us = np.linalg.eigh(Bm.T @ Bm)
        keep = sv >= 1e-14
        Q, _ = np.linalg.qr(Bm @ Us[:, keep])
        w, V = np.linalg.eigh(Q.T @ H @ Q)
        # strict checks on steps whose basis is well conditioned (the kept
        # overlap eigenvalues amplify rounding by s^-1/2, Q5) and whose carried
        # H-images are exact
        exact = sv[keep].min() >= 1e-8 and max(
            np.linalg.norm(d["X_new"][i] - H @ d["x_new"][i]) / np.linalg.norm(d["x_new"][i])
            for i in range(2)) < 1e-12
        self.worst["exact_steps"] += int(exact)
        R2 = Q @ V[:, :2]  # the two lowest Ritz vectors (orthonormal)
        for i in range(2):
            xu = d["x_new"][i] / np.linalg.norm(d["x_new"][i])
            # distance of x from the span of the two lowest Ritz vectors (the
            # pair is defined up to a rotation when their Ritz values coincide)
            off = np.linalg.norm(xu - R2 @ (R2.T @ xu))
            self.worst["ritz_all"] = max(self.worst["ritz_all"], off)
            if exact:
                self.worst["ritz"] = max(self.worst["ritz"], off)
                self.worst["energy"] = max(self.worst["energy"], abs(d["E_new"][i] - w[i]))
            x = d["x_new"][i]
            if exact:
                self.worst["knorm"] = max(self.worst["knorm"],
                                          abs(np.linalg.norm(x) - abs(d["k"][i])) / abs(d["k"][i]))
            X = d["X_new"][i]
            self.worst["drift"] = max(self.worst["drift"], np.linalg.norm(X - H @ x) / np.linalg.norm(x))
            # Eq. S111: x_t + B y_{t+1} = k v, with y_{t+1} = y_t - C z + A x_t
            lhs = d["x_old"][i] + d["B"][i, 0] * d["y_new"][0] + d["B"][i, 1] * d["y_new"][1]
            scale = (np.linalg.norm(d["x_old"][i]) + abs(d["B"][i, 0]) * np.linalg.norm(d["y_new"][0])
                     + abs(d["B"][i, 1]) * np.linalg.norm(d["y_new"][1]))
            self.worst["update"] = max(self.worst["update"], np.linalg.norm(lhs - x) / scale)


@pytest.mark.parametrize("sector", [0, 1])
def test_four_states_exact_and_every_step_pinned(h6, sector):
    I, sig, H, D = h6
    chk = StepChecks(H)
    run = sbci2.SBCI2(sig.apply, D, (20, 20), sbci.SBCIParams(sector=sector), step_hook=chk)
    res = run.solve(4)
    assert all(r.converged for r in res)
    E = np.sort([r.energy for r in res])
    w = np.linalg.eigvalsh(H)[:4] if sector == 0 else _sector_eigs(H, 20)[:4]
    assert np.abs(E - w).max() < 1e-8
    assert chk.n > 20
    # x_{t+1}^a, x_{t+1}^b lie in the span of the two lowest Ritz vectors of the
    # step's subspace (Eqs. S90, S110), E_{t+1} are its Ritz values and
    # |x_{t+1}| = |k|: checked on the dense H where the step's basis is well
    # conditioned (smallest kept overlap eigenvalue >= 1e-8), and loosely on
    # every step (the 1e-14 cut of Q5 keeps directions that amplify rounding)
    assert chk.worst["exact_steps"] > 20
    assert chk.worst["ritz"] < 1e-7 and chk.worst["energy"] < 1e-9 and chk.worst["knorm"] < 1e-9
    assert chk.worst["ritz_all"] < 1e-3
    # the coefficients solve the update rule (Eqs. S93, S112, S116, S117, S121)
    assert chk.worst["update"] < 1e-12
    # the carried H-images stay H x (Q9, Q10)
    assert chk.worst["drift"] < 1e-12
    X = np.column_stack([r.vector for r in res])
    assert np.abs(X.T @ X - np.eye(4)).max() < 1e-7


def test_pair_then_sbci1_counts(h6):
    """k = 2: one pair, then SBCI1 for the last state (Fig. 1B); k = 1: SBCI1 only."""
    I, sig, H, D = h6
    w = np.linalg.eigvalsh(H)
    run = sbci2.SBCI2(sig.apply, D, (20, 20))
    res = run.solve(2)
    assert abs(res[0].energy - w[0]) < 1e-8 and abs(res[1].energy - w[1]) < 1e-8
    assert {s.state for s in run.trace} == {0}
    run1 = sbci2.SBCI2(sig.apply, D, (20, 20))
    res1 = run1.solve(1)
    assert abs(res1[0].energy - w[0]) < 1e-8 and run1.trace == []


def test_first_step_coefficients_closed_form():
    """Eq. S93 on a hand-made V' (columns: lowest, second-lowest Ritz vector)."""
    Vp = np.array([[0.8, 0.1], [0.2, 0.9], [-0.3, 0.4], [0.5, -0.6]])
    A, B, C, k0, k1 = sbci2.pair_coefficients(Vp, True)
    assert np.allclose(B, np.eye(2))
    assert np.isclose(k0, 1 / 0.8) and np.isclose(k1, 1 / 0.9)
    assert np.isclose(A[0, 1], 0.2 / 0.8) and np.isclose(A[1, 0], 0.1 / 0.9)
    assert np.allclose(C, [[0.3 / 0.8, -0.5 / 0.8], [-0.4 / 0.9, 0.6 / 0.9]])


def test_later_step_coefficients_solve_eq_s111():
    """Eqs. S112, S116, S117, S121 on a random V': the rows of (I + B A, B, -B C)
    equal k_i V'[:, i] (the coefficient identity behind Eq. S111)."""
    rng = np.random.default_rng(7)
    Vp = rng.standard_normal((6, 2))
    A, B, C, k0, k1 = sbci2.pair_coefficients(Vp, False)
    k = np.array([k0, k1])
    lhs = np.hstack([np.eye(2) + B @ A, B, -B @ C])
    assert np.allclose(lhs, (Vp * k).T, rtol=1e-12, atol=1e-12)


def test_undefined_later_step_returns_none():
    Vp = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0], [0.0, 0.0], [0.3, 0.1], [0.2, 0.4]])
    assert sbci2.pair_coefficients(Vp, False) is None


def test_canonical_orthogonalisation_drops_dependent_direction():
    a = np.array([1.0, 0.0, 0.0])
    b = np.array([0.0, 1.0, 0.0])
    Bm = np.column_stack([a, b, a + b])
    P = sbci2.canonical_orthogonalisation(Bm.T @ Bm)
    assert P.shape == (3, 2)
    E = Bm @ P
    assert np.allclose(E.T @ E, np.eye(2))


def test_h8_three_states_against_lanczos():
    from oracle import eigen

    I = inputs.h_chain(8, 1.3)
    sig = sg.StringSigma(I.h1, I.eri, 4, 4)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 4, 4)
    wl, _ = eigen.lowest_lanczos(sig.apply, sig.ndet, 3)
    run = sbci2.SBCI2(sig.apply, D, (70, 70))
    res = run.solve(3)
    assert all(r.converged for r in res)
    assert np.abs(np.sort([r.energy for r in res]) - wl).max() < 1e-9
