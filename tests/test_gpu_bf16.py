"""The 3-term BF16 split contraction (SBCI_BF16X3) on the tensor cores: sigma
against the oracle, for every orbital count up to 16, and a mixed-precision
solve refined to the FP64 target.

Tolerance (derived from the arithmetic): a BF16 hi / lo pair carries 16 bits,
so each of D and W is represented to about 2^-17 of its value and the dropped
lo * lo product weighs 2^-18; with the FP32 accumulation of G and of the
scatter, sigma stays within 2e-4 of max|sigma| (the TF32x3 bound of 5e-6
scaled by the 2^4 fewer bits of each split half, with a factor 2.5 of room).
After FP64 refinement to the paper's thresholds the energies are held to the
FP64 target, 1e-8 hartree.
"""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import slater_condon as sc

from gpu_common import make_integrals, oracle_sector_energies, oracle_sigma, rel_err, require_lib

pytestmark = pytest.mark.gpu

BF16_TOL = 2e-4


@pytest.mark.parametrize("key", [("chain", 6, 1.0), ("rand", 7, 5, 4, 3), ("chain", 10, 1.2),
                                 ("chain", 12, 1.2), ("rand", 14, 14, 7, 7)])
def test_bf16x3_sigma_matches_oracle(key):
    import torch

    sbci = require_lib()
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    c = torch.from_numpy(inputs.random_vector(ctx.na, ctx.nb, 33)).cuda()
    ctx.profile(False)
    out = ctx.sigma(c, prec=sbci.SBCI_BF16X3)
    assert ctx.profile_read()["sigma_gather_contract_bf16"][0] == 1
    scale = float(out.abs().max())
    if ctx.ndet <= 100_000:
        err = rel_err(out.cpu().numpy(), oracle_sigma(key).apply(c.cpu().numpy()))
    else:  # sampled Slater-Condon rows of the oracle
        rows = np.random.default_rng(3).choice(ctx.ndet, 12, replace=False)
        ref = sc.sampled_sigma_rows(I.h1, I.eri, I.nalpha, I.nbeta, c.cpu().numpy(), rows)
        got = out.reshape(-1)[torch.from_numpy(rows).cuda()].cpu().numpy()
        err = float(np.abs(got - ref).max()) / scale
    assert err < BF16_TOL, err
    # and more accurate than a plain BF16 product would be (2^-9): the split works
    if ctx.ndet <= 100_000:
        assert err < 2e-3 * 0.1


def test_bf16x3_solve_h8_singlet():
    """Mixed-precision SBCI1 with the BF16x3 stage, refined to the FP64 target."""
    sbci = require_lib()
    key = ("chain", 8, 1.3)
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    p = sbci.params(sector=1, prec=sbci.SBCI_BF16X3)
    ctx.profile(False)
    E, _, R, st = ctx.solve(3, p)
    assert st == sbci.SBCI_OK and all(r.converged for r in R)
    launches = ctx.profile_read()
    assert launches["sigma_gather_contract_bf16"][0] > 0
    ref = oracle_sector_energies(key, 3) + I.e_core
    err = np.abs(np.sort(E) - ref)
    assert err.max() < 1e-8, err
    assert sum(r.n_sigma_fp64 for r in R) < sum(r.n_sigma for r in R)
