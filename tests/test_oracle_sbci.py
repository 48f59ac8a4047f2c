"""Pins for the oracle eigen-solvers and SBCI1 (exact energies, Ritz property, invariants)."""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import eigen, sbci, spin
from oracle import slater_condon as sc
from oracle import sigma as sg


@pytest.fixture(scope="module")
def h6():
    I = inputs.h_chain(6, 1.0)
    sig = sg.StringSigma(I.h1, I.eri, 3, 3)
    H = sc.dense_hamiltonian(I.h1, I.eri, 3, 3)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 3, 3)
    return I, sig, H, D


def test_eigensolvers_agree(h6):
    I, sig, H, D = h6
    w, _ = eigen.lowest_dense(H, 4)
    wl, _ = eigen.lowest_lanczos(sig.apply, sig.ndet, 4)
    wd, _ = eigen.davidson(sig.apply, D, 4, tol=1e-9)
    assert np.abs(w - wl).max() < 1e-10
    assert np.abs(w - wd).max() < 1e-10


def test_sbci1_random_start_ground_state(h6):
    """The small-chain workload: random c (seed 0), zero momentum, one state."""
    I, sig, H, D = h6
    w = np.linalg.eigvalsh(H)
    run = sbci.SBCI1(sig.apply, D, (20, 20))
    res = run.solve(1, c0=inputs.random_vector(20, 20, 0))
    assert res[0].converged
    assert abs(res[0].energy - w[0]) < 1e-8
    v = res[0].vector
    assert np.linalg.norm(H @ v - res[0].energy * v) < 1e-4


def test_sbci1_four_states(h6):
    I, sig, H, D = h6
    w = np.linalg.eigvalsh(H)
    run = sbci.SBCI1(sig.apply, D, (20, 20))
    res = run.solve(4)
    E = np.array([r.energy for r in res])
    assert all(r.converged for r in res)
    assert np.abs(E - w[:4]).max() < 1e-8
    X = np.column_stack([r.vector for r in res])
    assert np.abs(X.T @ X - np.eye(4)).max() < 1e-8


def test_splitmix_vector_reference_values():
    """SplitMix64 output function against values computed by hand from its
    definition (bit operations on Python integers)."""
    def ref(seed, alpha, i):
        M = (1 << 64) - 1
        z = (seed + 0x9E3779B97F4A7C15 * ((alpha << 40) + i + 1)) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        return 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0
    v = sbci.splitmix_vector(12345, 2, 50)
    assert all(v[i] == ref(12345, 2, i) for i in range(50))
    assert abs(v.mean()) < 0.3 and v.min() >= -1.0 and v.max() < 1.0


def test_sbci1_start_noise_reaches_the_lowest_states(h6):
    """R11: with a small full-symmetry component in every start, SBCI1 meets
    the four lowest eigenvalues of the symmetric H6 chain (as a set)."""
    I, sig, H, D = h6
    w = np.linalg.eigvalsh(H)
    run = sbci.SBCI1(sig.apply, D, (20, 20), sbci.SBCIParams(start_noise=1e-2, noise_seed=7))
    res = run.solve(4)
    E = np.sort([r.energy for r in res])
    assert all(r.converged for r in res)
    assert np.abs(E - w[:4]).max() < 1e-8


def test_sbci1_singlet_sector():
    I = inputs.h_chain(6, 1.4)
    sig = sg.StringSigma(I.h1, I.eri, 3, 3)
    H = sc.dense_hamiltonian(I.h1, I.eri, 3, 3)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 3, 3)
    w, V = np.linalg.eigh(H)
    sym = [j for j in range(len(w)) if np.abs(V[:, j].reshape(20, 20) - V[:, j].reshape(20, 20).T).max() < 1e-8]
    run = sbci.SBCI1(sig.apply, D, (20, 20), sbci.SBCIParams(sector=1))
    res = run.solve(3)
    E = np.array([r.energy for r in res])
    assert np.abs(E - w[sym[:3]]).max() < 1e-8
    for r in res:
        assert spin.s_squared(r.vector, 6, 3, 3) < 1e-6


def test_sbci1_matches_davidson_h8():
    I = inputs.h_chain(8, 1.2)
    sig = sg.StringSigma(I.h1, I.eri, 4, 4)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 4, 4)
    wd, _ = eigen.davidson(sig.apply, D, 3, tol=1e-9)
    res = sbci.SBCI1(sig.apply, D, (70, 70)).solve(3)
    assert np.abs(np.array([r.energy for r in res]) - wd).max() < 1e-8


class _Recorder(sbci.SBCI1):
    """Captures (x, y, z, X, Y, Z) and the chosen (E, b, c, k) of each step."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.steps = []

    def _first_step(self, x, X, z, Z):
        out = super()._first_step(x, X, z, Z)
        self.steps.append((x, np.zeros_like(x), z, out))
        return out

    def _later_step(self, x, X, y, Y, z, Z):
        out = super()._later_step(x, X, y, Y, z, Z)
        self.steps.append((x, y, z, out))
        return out


def test_sbci1_step_is_the_lowest_ritz_vector(h6):
    """x_{t+1} = x + b(y - c z) must be parallel to the lowest Ritz vector of H
    in span{x, y, z} (computed generically: QR + eigh), |x_{t+1}| = |k| and
    E_{t+1} = that Ritz value (Eqs. S19/S48, S62b)."""
    I, sig, H, D = h6
    run = _Recorder(sig.apply, D, (20, 20))
    run.solve(2)
    assert len(run.steps) > 10
    for x, y, z, (E, b, c, k, sec) in run.steps:
        vecs = [x, z] if not np.any(y) else [x, y, z]
        Q, _ = np.linalg.qr(np.column_stack(vecs))
        lam, U = np.linalg.eigh(Q.T @ H @ Q)
        u = Q @ U[:, 0]
        xn = x + b * (y - c * z) if np.any(y) else x - c * z
        assert abs(np.linalg.norm(xn) - abs(k)) < 1e-10 * abs(k)
        cosang = abs(u @ xn) / np.linalg.norm(xn)
        assert abs(1 - cosang) < 1e-10
        assert abs(E - lam[0]) < 1e-10 * max(1, abs(lam[0]))
        assert abs(sec[3] - lam[1]) < 1e-8 * max(1, abs(lam[1]))
        # Ritz value cannot exceed the Rayleigh quotient of x_t
        assert E <= x @ H @ x / (x @ x) + 1e-12


def test_sbci1_recurrences_track_h_images():
    """X = H x and Y = H y are carried by recurrences (Eqs. S28, S59); the
    recurrence drift stays at rounding level, and x stays orthogonal to the
    stored states (Eq. S31)."""
    I = inputs.h_chain(6, 1.0)
    sig = sg.StringSigma(I.h1, I.eri, 3, 3)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 3, 3)

    class Check(sbci.SBCI1):
        worst = 0.0
        worst_orth = 0.0
        xc_seen = []

        def _later_step(self, x, X, y, Y, z, Z):
            HX = self.apply(x.reshape(20, 20)).reshape(-1)
            Check.worst = max(Check.worst, np.linalg.norm(X - HX) / np.linalg.norm(HX))
            for u in Check.xc_seen:
                Check.worst_orth = max(Check.worst_orth, abs(u @ x) / np.linalg.norm(x), abs(u @ y) / np.linalg.norm(y))
            return super()._later_step(x, X, y, Y, z, Z)

    run = Check(sig.apply, D, (20, 20))
    orig = run.solve_state

    def wrapped(alpha, x0, X0, E0, xc, Ec):
        Check.xc_seen = list(xc)
        return orig(alpha, x0, X0, E0, xc, Ec)

    run.solve_state = wrapped
    run.solve(3)
    assert Check.worst < 1e-10
    assert Check.worst_orth < 1e-10


def test_energy_conservation_diagnostic_is_close_to_one():
    """Section S4 (Eq. S136): Delta E_t ~ (2/c_{t-2}) Delta T_t with the mass
    M = D - E^0.  A diagnostic without a stated tolerance, whose sign depends on
    the sign convention of z' (Eq. S60 divides by k, Algorithm 1 by |x|), so only the
    magnitude is checked, on consecutive later steps inside one restart cycle
    while the energy still moves (|Delta E| > 1e-5)."""
    I = inputs.h_chain(8, 1.0)
    sig = sg.StringSigma(I.h1, I.eri, 4, 4)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 4, 4)
    rec = []

    class Tr(sbci.SBCI1):
        def _first_step(self, x, X, z, Z):
            out = super()._first_step(x, X, z, Z)
            rec.append((0, x, X, np.zeros_like(x), out))
            return out

        def _later_step(self, x, X, y, Y, z, Z):
            out = super()._later_step(x, X, y, Y, z, Z)
            rec.append((1, x, X, y, out))
            return out

    Tr(sig.apply, D, (70, 70)).solve(1)
    ratios = []
    for t in range(2, len(rec)):
        if rec[t][0] == 0 or rec[t - 1][0] == 0:
            continue
        _, x1, X1, y1, _ = rec[t - 1]
        _, x2, X2, y2, _ = rec[t]
        b2, c2 = rec[t - 2][4][1], rec[t - 2][4][2]
        M = D - rec[t - 1][4][0]
        dE = (x1 @ X1) / (x1 @ x1) - (x2 @ X2) / (x2 @ x2)
        dT = 0.5 * b2 * (y2 @ (M * y2) - y1 @ (M * y1))
        if abs(dE) > 1e-5:
            ratios.append(abs(dE / ((2.0 / c2) * dT)))
    assert len(ratios) >= 5
    assert 0.3 < float(np.median(ratios)) < 3.0


def test_r15_later_step_undefined_and_first_step_fallback():
    """A later step can be undefined (reading R15): with H = diag(1, 2, 0) and
    x = (1, 1, 1), y = (1, -1, 0), z = (-1, -1, 2), the lowest Ritz vector of
    span{x, y, z} is e3 = (x + z) / 3, which has no y component, so no finite
    c reaches it through x + b (y - c z) (Eq. S55 divides by zero).  The
    first-step path from x / |x| on the same z is defined and is the lowest
    Ritz vector of span{x, z}."""
    Hm = np.diag([1.0, 2.0, 0.0])
    H = lambda v: Hm @ v
    run = sbci.SBCI1(H, np.diag(Hm).copy(), (1, 3))
    x = np.array([1.0, 1.0, 1.0])
    y = np.array([1.0, -1.0, 0.0])
    z = np.array([-1.0, -1.0, 2.0])
    with np.errstate(divide="ignore", invalid="ignore"):
        E, b, c, k, _ = run._later_step(x, H(x), y, H(y), z, H(z))
    assert abs(E) < 1e-12  # the Ritz value itself is fine: e3's eigenvalue 0
    # in floating point the zero denominator comes out as 0 (non-finite c: R15)
    # or as a rounding residue (an astronomically large c, and |k| = 3 outside
    # [x_th1, x_th2], so S62b restarts right after the step)
    assert (not np.all(np.isfinite([E, b, c, k]))) or (abs(c) > 1e12 and abs(k) > run.p.x_th2)
    xn = x / np.linalg.norm(x)
    E1, b1, c1, k1, _ = run._first_step(xn, H(xn), z, H(z))
    assert np.all(np.isfinite([E1, b1, c1, k1]))
    B = np.linalg.qr(np.stack([xn, z], axis=1))[0]
    assert abs(E1 - np.linalg.eigvalsh(B.T @ Hm @ B)[0]) < 1e-12


def test_restart_cause_on_constructed_scalars():
    """Section S1.5, Eqs. S62a-c with the paper's thresholds (b_th = 1e-2,
    eps1 = 1e-7, x_th1 = 0.1, x_th2 = 1.2, r1 = 1, max_cycle = 20), each
    condition switched on alone from a base step that triggers none, plus the
    edges the inequalities fix (strict bounds, alpha > 0 in S62a, t > 0 in
    S62c, the max_cycle period of reading R5)."""
    p = sbci.SBCIParams()
    base = dict(alpha=1, b=0.5, k=1.0, dE=1e-3, dz=0.5, t=3)

    def cause(**kw):
        a = dict(base, **kw)
        return sbci.restart_cause(p, a["alpha"], a["b"], a["k"], a["dE"], a["dz"], a["t"])

    assert cause() == ""
    # S62a: needs alpha > 0, |b| < b_th and dE < eps1 together
    assert cause(b=-5e-3, dE=5e-8) == "a"
    assert cause(alpha=0, b=5e-3, dE=5e-8) == ""  # the ground state never restarts by S62a
    assert cause(b=1e-2, dE=5e-8) == ""  # |b| = b_th is not below it
    assert cause(b=5e-3, dE=1e-7) == ""  # dE = eps1 is not below it
    assert cause(b=5e-3) == ""  # large dE
    # S62b: |k| outside [x_th1, x_th2], either sign of k
    assert cause(k=0.05) == "b" and cause(k=-0.05) == "b"
    assert cause(k=1.3) == "b" and cause(k=-1.3) == "b"
    assert cause(k=0.1) == "" and cause(k=1.2) == ""  # the bounds themselves are inside
    # S62c: |z'| > r1 on a later step only
    assert cause(dz=1.5) == "c"
    assert cause(dz=1.5, t=0) == ""
    assert cause(dz=1.0) == ""
    # the max_cycle period: t + 1 reaches max_cycle
    assert cause(t=19) == "max" and cause(t=18) == ""
    # order of the tests when several hold: S62a, then S62b, S62c, max_cycle
    assert cause(b=5e-3, dE=5e-8, k=2.0, dz=2.0, t=19) == "a"
    assert cause(k=2.0, dz=2.0, t=19) == "b"
    assert cause(dz=2.0, t=19) == "c"


def test_energy_conservation_in_the_trace():
    """The trace's per-step Eq. S136 right-hand side (2/c) Delta T against the
    Rayleigh-quotient drop Delta E of the same update (Eq. S134), on H8: the
    paper's Section S4 finds the two close at every step (Fig. S10); here the
    median of |Delta E / ((2/c) Delta T)| over the later steps that still move
    the energy (|Delta E| > 1e-5) lies within a factor 3 of one (the band of
    the diagnostic test above; the sign follows the z' convention of reading
    R1), and first steps carry no value."""
    I = inputs.h_chain(8, 1.0)
    sig = sg.StringSigma(I.h1, I.eri, 4, 4)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 4, 4)
    run = sbci.SBCI1(sig.apply, D, (70, 70))
    run.solve(2)
    tr = run.trace
    ratios = []
    for prev, cur in zip(tr, tr[1:]):
        if cur.t == 0:
            assert np.isnan(cur.s136)
            continue
        if prev.state != cur.state or not np.isfinite(cur.s136):
            continue
        dE = prev.energy - cur.energy
        if abs(dE) > 1e-5:
            ratios.append(dE / cur.s136)
    assert len(ratios) >= 10
    med = float(np.median(np.abs(ratios)))
    assert 0.3 < med < 3.0, med
