"""Split-precision sigma on the tensor cores and the mixed -> FP64 refinement solve.

Tolerances (derived from the arithmetic): a TF32 hi/lo pair carries 22 bits,
the three kept products leave ~2^-21 relative per product, D and G are
accumulated in FP32 (2^-24 per add over <= 2*nlink and npair terms), so sigma
stays within 5e-6 of max|sigma|; FP32 SIMT the same.  After FP64 refinement to
the paper's thresholds the energies are held to the FP64 target, 1e-8 hartree.
"""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import sbci as osb
from oracle import slater_condon as sc

from gpu_common import make_integrals, oracle_sigma, rel_err, require_lib

pytestmark = pytest.mark.gpu

SPLIT_TOL = 5e-6


@pytest.mark.parametrize("key", [("chain", 6, 1.0), ("rand", 7, 5, 4, 3), ("chain", 10, 1.2),
                                 ("chain", 12, 1.2)])
@pytest.mark.parametrize("prec", ["TF32X3", "FP32"])
def test_split_sigma_matches_oracle(key, prec):
    sbci = require_lib()
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    c = np.stack([inputs.random_vector(ctx.na, ctx.nb, s) for s in (31, 32)])
    out = ctx.sigma(c, prec=getattr(sbci, "SBCI_" + prec))
    if ctx.ndet <= 100_000:
        ora = oracle_sigma(key)
        for v in range(2):
            assert rel_err(out[v], ora.apply(c[v])) < SPLIT_TOL
    else:  # H12: sampled Slater-Condon rows of the oracle
        rows = np.random.default_rng(1).choice(ctx.ndet, 16, replace=False)
        ref = sc.sampled_sigma_rows(I.h1, I.eri, I.nalpha, I.nbeta, c[0], rows)
        scale = np.abs(out[0]).max()
        assert np.abs(out[0].reshape(-1)[rows] - ref).max() < SPLIT_TOL * scale


def test_tf32x3_random_df_n14_rows():
    import torch

    sbci = require_lib()
    I = make_integrals(("rand", 14, 14, 7, 7))
    ctx = sbci.Context.from_integrals(I)
    u = torch.from_numpy(inputs.random_vector(3432, 3432, 41)).cuda()
    s_tc = ctx.sigma(u, prec=sbci.SBCI_TF32X3)
    rows = np.random.default_rng(2).choice(ctx.ndet, 12, replace=False)
    ref = sc.sampled_sigma_rows(I.h1, I.eri, 7, 7, u.cpu().numpy(), rows)
    got = s_tc.reshape(-1)[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.abs(got - ref).max() < SPLIT_TOL * float(s_tc.abs().max())


def test_tf32x3_rejected_beyond_shared_memory():
    sbci = require_lib()
    I = inputs.random_df(16, 3, 1, 1)  # n = 16: TF32 operands exceed shared memory
    ctx = sbci.Context.from_integrals(I)
    c = inputs.random_vector(ctx.na, ctx.nb, 0)
    with pytest.raises(sbci.SbciError) as e:
        ctx.sigma(c, prec=sbci.SBCI_TF32X3)
    assert e.value.status == sbci.SBCI_ERR_INVALID


@pytest.mark.parametrize("prec", ["TF32X3", "FP32"])
def test_mixed_solve_h10_singlet(prec):
    """The H10 workload with the split-precision stage and FP64 refinement."""
    sbci = require_lib()
    key = ("chain", 10, 1.2)
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    E, V, R, st = ctx.solve(4, sbci.params(sector=1, prec=getattr(sbci, "SBCI_" + prec)),
                            want_vectors=True)
    assert st == sbci.SBCI_OK
    assert all(r.converged for r in R)
    ora = oracle_sigma(key)
    D = sc.diagonal_by_occupation(I.h1, I.eri, 5, 5)
    run = osb.SBCI1(ora.apply, D, (252, 252), osb.SBCIParams(sector=1))
    Eo = np.array([r.energy for r in run.solve(4)]) + I.e_core
    err = np.abs(np.sort(E) - np.sort(Eo))
    assert err.max() < 1e-8, err
    # every state ends with FP64 H-products, and most of the work is low precision
    assert all(r.n_sigma_fp64 >= 1 for r in R)
    assert sum(r.n_sigma_fp64 for r in R) < sum(r.n_sigma for r in R)
    tr = ctx.trace()
    assert any(t.event == 6 for t in tr)


def test_refinement_budget_falls_back_to_fp64():
    """A state whose low-precision refinement spends its budget
    (refine_max_sigma) continues with FP64 sigma from an exact X and meets the
    FP64 target; the trace records the fallback (event 7)."""
    sbci = require_lib()
    I = make_integrals(("chain", 8, 1.3))
    ctx = sbci.Context.from_integrals(I)
    E64, _, _, st = ctx.solve(3, sbci.params(prec=sbci.SBCI_FP64))
    assert st == sbci.SBCI_OK
    p = sbci.params(prec=sbci.SBCI_TF32X3, refine_max_sigma=2)
    E, _, R, st = ctx.solve(3, p)
    assert st == sbci.SBCI_OK and all(r.converged for r in R)
    assert np.abs(E - E64).max() < 1e-8
    assert any(t.event == 7 for t in ctx.trace())
    # the same through the batched engine and the batched server
    ctxs = [sbci.Context.from_integrals(I) for _ in range(3)]
    EB, RB, st = sbci.solve_batch(ctxs, 3, p)
    assert st == sbci.SBCI_OK
    for i in range(3):
        assert np.array_equal(EB[i], E)
    server = sbci.Server(4 << 30, 4, batching=True)
    t = [server.submit(I, 3, p) for _ in range(2)]
    done = {}
    import time
    t0 = time.time()
    while len(done) < 2 and time.time() - t0 < 300:
        server.progress()
        for x in t:
            r = server.poll(x)
            if r is not None:
                done[x] = r
    assert len(done) == 2
    for x in t:
        assert done[x][3] == sbci.SBCI_OK and np.array_equal(done[x][0], E)
    server.close()
    for c in ctxs:
        c.close()


def test_stagnating_refinement_falls_back_to_fp64():
    """Stretched H12 (2.96 A, nearly degenerate) with a seeded start: the
    TF32x3 refinement stalls at its noise floor (|z'| ~ 2e-5, above r0), and
    its large-|b| steps carry low-precision rounding into X.  X is made exact
    after every max_cycle refinement steps and, after two windows without
    convergence, the state goes on with FP64 sigma (before, the refinement
    spent its budget while X drifted from H x until the energies ran away).
    All three states meet the FP64 solve's energies."""
    sbci = require_lib()
    I = inputs.h_chain(12, 2.959854009887736)
    ctx = sbci.Context.from_integrals(I)
    E64, _, _, st = ctx.solve(3, sbci.params(prec=sbci.SBCI_FP64, start_noise=1e-2, noise_seed=2603))
    assert st == sbci.SBCI_OK
    p = sbci.params(prec=sbci.SBCI_TF32X3, start_noise=1e-2, noise_seed=2603)
    E, _, R, st = ctx.solve(3, p)
    assert st == sbci.SBCI_OK and all(r.converged for r in R)
    assert np.abs(E - E64).max() < 1e-8
    tr = ctx.trace()
    assert min(t.energy for t in tr) > E64[0] - I.e_core - 1e-4  # no run-away below the ground state
