"""GPU SBCI1 against the oracle: energies, trajectories, excited states, sectors.

Tolerances: energies within 1e-8 hartree of the oracle (the FP64 target);
step-by-step Ritz energies within 1e-10 and identical restart/convergence
events while both runs take the same decisions.
"""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import eigen, sbci as osb, spin
from oracle import slater_condon as sc

from gpu_common import make_integrals, oracle_sigma, require_lib

pytestmark = pytest.mark.gpu


def _oracle_run(key, nstates, c0=None, **kw):
    I = make_integrals(key)
    ora = oracle_sigma(key)
    D = sc.diagonal_by_occupation(I.h1, I.eri, I.nalpha, I.nbeta)
    run = osb.SBCI1(ora.apply, D, (ora.Na, ora.Nb), osb.SBCIParams(**kw))
    res = run.solve(nstates, c0=c0)
    return run, res


def test_h6_random_start_trajectory_parity():
    """The small-chain workload: H6 at 1.0 A, random c (seed 0), zero momentum."""
    sbci = require_lib()
    key = ("chain", 6, 1.0)
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    c0 = inputs.random_vector(20, 20, 0)
    E, V, R, stt = ctx.solve(1, sbci.params(init=1), c0=c0, want_vectors=True)
    assert stt == sbci.SBCI_OK and R[0].converged
    H = sc.dense_hamiltonian(I.h1, I.eri, 3, 3)
    w = np.linalg.eigvalsh(H)
    assert abs(E[0] - (w[0] + I.e_core)) < 1e-8
    run, res = _oracle_run(key, 1, c0=c0)
    tr = ctx.trace()
    assert len(tr) == len(run.trace)
    for g, o in zip(tr, run.trace):
        assert abs(g.energy - o.energy) < 1e-10
        assert abs(g.b - o.b) < 1e-8 * max(1.0, abs(o.b))
        assert abs(abs(g.k) - abs(o.k)) < 1e-8
        ev = {0: "", 1: "converged", 2: "restart:a", 3: "restart:b", 4: "restart:c", 5: "restart:max"}[g.event]
        assert ev == o.event
        # the Eq. S136 right-hand side of the update: defined on the same steps
        assert np.isfinite(g.s136) == np.isfinite(o.s136)
    v = V[0]
    assert np.linalg.norm(H @ v - (E[0] - I.e_core) * v) < 2e-5


def test_h6_four_states_and_step_api():
    sbci = require_lib()
    key = ("chain", 6, 1.0)
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    E, V, R, stt = ctx.solve(4, want_vectors=True)
    assert stt == sbci.SBCI_OK
    H = sc.dense_hamiltonian(I.h1, I.eri, 3, 3)
    w = np.linalg.eigvalsh(H)[:4] + I.e_core
    # H6 has inversion symmetry: the start of an excited state (S1.4) keeps the
    # symmetry of the previous state up to rounding, so two runs may meet the
    # third and fourth states in either order.  The set found is unique; the
    # order is not, so compare sorted energies and check each is an eigenpair.
    assert np.abs(np.sort(E) - w).max() < 1e-8
    for j in range(4):
        assert np.linalg.norm(H @ V[j] - (E[j] - I.e_core) * V[j]) < 2e-5
    assert np.abs(V @ V.T - np.eye(4)).max() < 1e-8
    _, res = _oracle_run(key, 4)
    assert np.abs(np.sort(E - I.e_core) - np.sort([r.energy for r in res])).max() < 1e-8
    # begin / step / finish give the same as solve
    ctx.begin(4)
    done = False
    n = 0
    while not done:
        rec, done = ctx.step()
        n += 1
    E2, _, R2, _ = ctx.finish()
    assert np.array_equal(E, E2)
    assert n == sum(r.n_step for r in R2)


def test_h10_singlet_sector_four_states():
    """The H10 workload (1.2 A): ground + 3 excited states in the c = c^T sector."""
    sbci = require_lib()
    key = ("chain", 10, 1.2)
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    E, V, R, stt = ctx.solve(4, sbci.params(sector=1), want_vectors=True)
    assert stt == sbci.SBCI_OK
    _, res = _oracle_run(key, 4, sector=1)
    Eo = np.array([r.energy for r in res]) + I.e_core
    assert np.abs(E - Eo).max() < 1e-8
    for j in range(4):
        m = V[j].reshape(252, 252)
        assert np.abs(m - m.T).max() < 1e-10
    assert spin.s_squared(V[0], 10, 5, 5) < 1e-6


def test_h8_three_states_vs_davidson():
    sbci = require_lib()
    key = ("chain", 8, 1.3)
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    E, _, R, stt = ctx.solve(3)
    ora = oracle_sigma(key)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 4, 4)
    wd, _ = eigen.davidson(ora.apply, D, 3, tol=1e-9)
    assert np.abs(E - (wd + I.e_core)).max() < 1e-8


def test_unequal_spins_ground_state():
    sbci = require_lib()
    key = ("rand", 7, 5, 4, 3)
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    E, _, _, stt = ctx.solve(2)
    H = sc.dense_hamiltonian(I.h1, I.eri, 4, 3)
    w = np.linalg.eigvalsh(H)[:2]
    assert np.abs(E - w).max() < 1e-8


def test_random_df_n14_two_states_residual_rows():
    """The 11.8M-determinant random-DF workload in FP64: the oracle checks the
    returned vectors row by row (Slater-Condon residual on sampled rows) and the
    Rayleigh quotient through its own sigma."""
    sbci = require_lib()
    key = ("rand", 14, 14, 7, 7)
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    E, V, R, stt = ctx.solve(2, want_vectors=True)
    assert stt == sbci.SBCI_OK
    rows = np.random.default_rng(3).choice(ctx.ndet, 12, replace=False)
    for j in range(2):
        hx = sc.sampled_sigma_rows(I.h1, I.eri, 7, 7, V[j], rows)
        res = hx - E[j] * V[j][rows]
        assert np.abs(res).max() < 1e-5
    assert abs(float(V[0] @ V[1])) < 1e-8


@pytest.mark.parametrize("key,k,kw", [(("chain", 6, 1.0), 4, {}), (("chain", 10, 1.2), 3, {"sector": 1}),
                                       (("chain", 8, 1.3), 3, {})])
def test_start_noise_matches_oracle(key, k, kw):
    """start_noise (reading R11): the same seeded SplitMix64 vector on both sides;
    the states found must agree with the oracle and be the lowest ones."""
    sbci = require_lib()
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    E, _, R, st = ctx.solve(k, sbci.params(start_noise=1e-2, noise_seed=7, **kw))
    assert st == sbci.SBCI_OK
    _, res = _oracle_run(key, k, start_noise=1e-2, noise_seed=7, **kw)
    Eo = np.array([r.energy for r in res]) + I.e_core
    assert np.abs(np.sort(E) - np.sort(Eo)).max() < 1e-8
    if not kw:
        H = sc.dense_hamiltonian(I.h1, I.eri, I.nalpha, I.nbeta)
        w = np.linalg.eigvalsh(H)[:k] + I.e_core
        assert np.abs(np.sort(E) - w).max() < 1e-8


@pytest.mark.parametrize("key,c0seed,hf", [(("chain", 6, 1.0), 0, False), (("chain", 10, 1.2), 0, True)])
def test_energy_conservation_diagnostic_matches_oracle(key, c0seed, hf):
    """Section S4 (Eq. S136) at run time: the device controller's per-step
    (2/c) Delta T equals the oracle's in magnitude on the same FP64 trajectory
    (1e-8 of its scale, on the records before the two runs part, that is
    while their energies agree to 1e-10; its sign follows that of c, which
    the eigenvector sign decides), and the report's geometric-mean ratio |Delta E / ((2/c) Delta T)|
    is the oracle's own, computed the same way from its trace."""
    sbci = require_lib()
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    c0 = inputs.random_vector(ctx.na, ctx.nb, c0seed)
    if hf:
        # H10: a random start sits mid-spectrum, where D - E_0 nearly vanishes
        # for many determinants and the first steps amplify rounding (the two
        # runs part within a step); start near the lowest determinant instead
        D = sc.diagonal_by_occupation(I.h1, I.eri, I.nalpha, I.nbeta)
        c0 = 0.05 * c0.reshape(-1)
        c0[int(np.argmin(D))] += 1.0
        c0 = (c0 / np.linalg.norm(c0)).reshape(ctx.na, ctx.nb)
    kw = {"init": 1} if c0 is not None else {}
    E, _, R, st = ctx.solve(1, sbci.params(**kw), c0=c0)
    assert st == sbci.SBCI_OK
    run, _ = _oracle_run(key, 1, c0=c0)
    tr = ctx.trace()
    checked = 0
    for g, o in zip(tr, run.trace):
        if abs(g.energy - o.energy) >= 1e-10:  # the two runs have parted (rounding, chaotic SB)
            break
        assert np.isfinite(g.s136) == np.isfinite(o.s136)
        if np.isfinite(o.s136):
            # c (and with it 2/c) takes the sign of the Ritz vector, which either
            # eigen-solver may flip (reading C-11): compare magnitudes
            assert abs(abs(g.s136) - abs(o.s136)) <= 1e-8 * max(abs(o.s136), 1e-6), (g.s136, o.s136)
            checked += 1
    assert checked >= 3
    # the report's summary against the same summary of the oracle's trace
    lsum, cnt = 0.0, 0
    for p_, q in zip(run.trace, run.trace[1:]):
        if q.t > 0 and np.isfinite(q.s136) and q.s136 != 0.0 and abs(p_.energy - q.energy) > 1e-6:
            lsum += np.log(abs((p_.energy - q.energy) / q.s136))
            cnt += 1
    assert R[0].s136_steps > 0
    if len(tr) == len(run.trace):
        assert R[0].s136_steps == cnt
        assert abs(R[0].s136_ratio - np.exp(lsum / cnt)) < 1e-6 * np.exp(lsum / cnt)
    assert 0.1 < R[0].s136_ratio < 10.0
