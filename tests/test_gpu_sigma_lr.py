"""Low-rank (density-fitting) form of the FP64 SIMT sigma contraction
(lowrank.h): W = F M F^T with F = [L | kappa | delta] from a pivoted Cholesky
of the pair matrix (ij|kl) = L L^T and the one-electron part, G = (F M)(F^T D).
Used beyond the exact-slice kernel's size (npair > 55) when the two-electron
integrals are density-fitted (rank W <= naux + 2 < 0.45 npair: from n = 14
orbitals with naux = 3n).

Tolerance as for the full contraction: FP64 1e-12 of max|sigma| (the
Cholesky remainder is below 1e-13 of the largest diagonal of (ij|kl)).

The TF32x3 contraction can take the same factor on the tensor cores
(kernels_tclr.cu): T = D F and G = T (F M)^T as two chained tcgen05 products
per tile, T re-split from its FP32 accumulator; selected where the full
form's operands exceed shared memory (n = 15), or everywhere it fits with
SBCI_TC_LOWRANK=1.  Its bound is the TF32x3 split's, 5e-6 of max|sigma| (as
for the full form, test_gpu_mixed).
"""
import os

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
SPLIT_TOL = 5e-6


def _ctx_env(sbci, I, name, value):
    old = os.environ.get(name)
    os.environ[name] = value
    try:
        return sbci.Context.from_integrals(I)
    finally:
        if old is None:
            del os.environ[name]
        else:
            os.environ[name] = old


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


def test_tf32x3_factored_form_on_tensor_cores():
    """TF32x3 on the density-fitted n = 14 space: the full form by default
    (it fits shared memory and is the faster one there), the factored
    tensor-core contraction with SBCI_TC_LOWRANK=1 (259 tiles, the last one
    ragged); both meet the TF32x3 bound against the oracle."""
    sbci = require_lib()
    I = inputs.random_df(14, 7, 3, 2)
    ora = oracle_sigma(KEY)
    c = np.random.default_rng(5).standard_normal((2, ora.ndet))
    ref = np.stack([ora.apply(ci.reshape(ora.Na, ora.Nb)).reshape(-1) for ci in c])
    ctx = sbci.Context.from_integrals(I)
    s, st = _stats(ctx, lambda: ctx.sigma(c, prec=sbci.SBCI_TF32X3))
    assert st["sigma_gather_contract_tc"][0] == 2 and st["sigma_gather_contract_tc_lr"][0] == 0
    assert rel_err(s, ref) < SPLIT_TOL
    ctx.close()
    fac = _ctx_env(sbci, I, "SBCI_TC_LOWRANK", "1")
    s2, st2 = _stats(fac, lambda: fac.sigma(c, prec=sbci.SBCI_TF32X3))
    assert st2["sigma_gather_contract_tc_lr"][0] == 2 and st2["sigma_gather_contract_tc"][0] == 0
    assert rel_err(s2, ref) < SPLIT_TOL
    fac.close()


def test_tf32x3_n15_only_in_factored_form():
    """n = 15 (npair = 120): the full-form TF32 operands exceed shared memory,
    the factored ones fit, so TF32x3 runs on a density-fitted space through
    the factored kernel and meets its bound; with the full form kept the
    precision is refused."""
    sbci = require_lib()
    key = ("rand", 15, 9, 2, 2)  # 105 x 105 strings, rank(W) <= 3n + 2 = 47
    I = inputs.random_df(15, 9, 2, 2)
    ora = oracle_sigma(key)
    c = np.random.default_rng(6).standard_normal(ora.ndet)
    ctx = sbci.Context.from_integrals(I)
    s, st = _stats(ctx, lambda: ctx.sigma(c, prec=sbci.SBCI_TF32X3))
    assert st["sigma_gather_contract_tc_lr"][0] == 1
    assert rel_err(s, ora.apply(c.reshape(ora.Na, ora.Nb)).reshape(-1)) < SPLIT_TOL
    ctx.close()
    full = _ctx_env(sbci, I, "SBCI_TC_LOWRANK", "0")
    with pytest.raises(sbci.SbciError) as e:
        full.sigma(c, prec=sbci.SBCI_TF32X3)
    assert e.value.status == sbci.SBCI_ERR_INVALID
    full.close()


def test_low_rank_tf32x3_solve():
    """A mixed TF32x3 SBCI1 solve on the density-fitted space with the
    factored tensor-core contraction (SBCI_TC_LOWRANK=1) runs it in its step
    loop and, after the FP64 refinement, reaches the oracle's Lanczos
    energy."""
    sbci = require_lib()
    from oracle import eigen

    I = inputs.random_df(14, 7, 3, 2)
    ctx = _ctx_env(sbci, I, "SBCI_TC_LOWRANK", "1")
    (E, _, R, st), stats = _stats(ctx, lambda: ctx.solve(1, sbci.params(prec=sbci.SBCI_TF32X3)))
    assert st == sbci.SBCI_OK and R[0].converged
    assert stats["sigma_gather_contract_tc_lr"][0] > 10
    ora = oracle_sigma(KEY)
    wl, _ = eigen.lowest_lanczos(ora.apply, ora.ndet, 1)
    assert abs(E[0] - (wl[0] + I.e_core)) < 1e-8
