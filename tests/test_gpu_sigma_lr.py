"""Low-rank (density-fitting) form of the FP64 SIMT sigma contraction
(lowrank.h): W = F M F^T with F = [L | kappa | delta] from a pivoted Cholesky
of the pair matrix (ij|kl) = L L^T and the one-electron part, G = (F M)(F^T D).
Used beyond the exact-slice kernel's size (npair > 55) when the two-electron
integrals are density-fitted (rank W <= naux + 2 < 0.45 npair: from n = 14
orbitals with naux = 3n).

Tolerance as for the full contraction: FP64 1e-12 of max|sigma| (the
Cholesky remainder is below 1e-13 of the largest diagonal of (ij|kl)).
"""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs

from gpu_common import oracle_sigma, rel_err, require_lib

pytestmark = pytest.mark.gpu


def _stats(ctx, fn):
    ctx.profile(True)
    out = fn()
    st = ctx.profile_read()
    ctx.profile(False)
    return out, st


KEY = ("rand", 14, 7, 3, 2)  # npair = 105, rank(W) <= 3n + 2 = 44; 33,124 determinants


def test_density_fitted_space_uses_low_rank_form():
    sbci = require_lib()
    I = inputs.random_df(14, 7, 3, 2)
    ctx = sbci.Context.from_integrals(I)
    ora = oracle_sigma(KEY)
    c = np.random.default_rng(4).standard_normal((2, ctx.ndet))
    s, st = _stats(ctx, lambda: ctx.sigma(c, prec=sbci.SBCI_FP64))
    assert st["sigma_gather_contract_lr"][0] == 2 and st["sigma_gather_contract"][0] == 0
    ref = np.stack([ora.apply(ci.reshape(ora.Na, ora.Nb)).reshape(-1) for ci in c])
    assert rel_err(s, ref) < 1e-12
    # the FP32 contraction keeps the full form
    s32, st32 = _stats(ctx, lambda: ctx.sigma(c, prec=sbci.SBCI_FP32))
    assert st32["sigma_gather_contract_lr"][0] == 0 and st32["sigma_gather_contract"][0] == 2
    assert rel_err(s32, ref) < 2e-5


def test_full_rank_space_keeps_the_full_contraction():
    sbci = require_lib()
    I = inputs.h_chain(12, 1.2)  # npair = 78, W of full rank
    ctx = sbci.Context.from_integrals(I)
    c = np.random.default_rng(1).standard_normal(ctx.ndet)
    _, st = _stats(ctx, lambda: ctx.sigma(c, prec=sbci.SBCI_FP64))
    assert st["sigma_gather_contract_lr"][0] == 0 and st["sigma_gather_contract"][0] == 1


def test_low_rank_fp64_solve():
    """An FP64 SBCI1 solve on the density-fitted space runs the low-rank
    contraction inside its step loop and reaches the oracle's Lanczos energy."""
    sbci = require_lib()
    from oracle import eigen

    I = inputs.random_df(14, 7, 3, 2)
    ctx = sbci.Context.from_integrals(I)
    (E, _, R, st), stats = _stats(ctx, lambda: ctx.solve(1, sbci.params()))
    assert st == sbci.SBCI_OK and R[0].converged
    assert stats["sigma_gather_contract_lr"][0] > 10
    ora = oracle_sigma(KEY)
    wl, _ = eigen.lowest_lanczos(ora.apply, ora.ndet, 1)
    assert abs(E[0] - (wl[0] + I.e_core)) < 1e-8
