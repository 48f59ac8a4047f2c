"""FP64 sigma with the contraction on the tensor cores by exact BF16 integer
slices (kernels_os.cu, the error-free splitting of Ozaki, Ogita & Oishi 2012),
against the oracle and against the FP64-FMA kernel.

Tolerance: 2e-14 of max|sigma|.  The slices carry 56 bits of every D row and
W row below its largest element and every product and level sum is exact, so
the result differs from exact arithmetic by the final rounding to FP64 (plus
2^-56 of the row scales); FP64 FMAs differ by about 2^-53 per term.  If the
tensor cores rounded any of the level sums (which stay below 2^23), the error
would be near 2^-24.
"""
import os

import numpy as np
import pytest

from gpu_common import make_integrals, oracle_sigma, rel_err, require_lib

pytestmark = pytest.mark.gpu

TOL = 2e-14

CASES = [
    ("chain", 4, 1.0),        # 36 dets: one ragged tile
    ("chain", 6, 1.0),        # 400 dets, ragged tail
    ("chain", 8, 1.3),        # 4900
    ("rand", 7, 5, 4, 3),     # nalpha != nbeta
    ("rand", 9, 6, 5, 3),     # 10584, ragged
    ("rand", 4, 8, 0, 2),     # no alpha electrons
    ("rand", 10, 11, 5, 5),   # npair = 55, the largest operand the kernel takes
    ("chain", 10, 1.2),       # the H10 workload, 63504
]


def _ctx(key, dfma=False):
    sbci = require_lib()
    old = os.environ.get("SBCI_FP64_CONTRACTION")
    if dfma:
        os.environ["SBCI_FP64_CONTRACTION"] = "dfma"
    else:
        os.environ.pop("SBCI_FP64_CONTRACTION", None)
    try:
        return sbci.Context.from_integrals(make_integrals(key))
    finally:
        if old is None:
            os.environ.pop("SBCI_FP64_CONTRACTION", None)
        else:
            os.environ["SBCI_FP64_CONTRACTION"] = old


@pytest.mark.parametrize("key", CASES)
def test_against_oracle_and_fma_kernel(key):
    sbci = require_lib()
    ctx = _ctx(key)
    ora = oracle_sigma(key)
    rng = np.random.default_rng(11)
    c = rng.standard_normal((2, ctx.ndet))
    ctx.profile(True)
    s = ctx.sigma(c, prec=sbci.SBCI_FP64)
    stats = ctx.profile_read()
    ctx.profile(False)
    assert stats["sigma_gather_contract_os"][0] == 2 and stats["sigma_gather_contract"][0] == 0
    ref = np.stack([ora.apply(ci.reshape(ora.Na, ora.Nb)).reshape(-1) for ci in c])
    assert rel_err(s, ref) < TOL
    s2 = _ctx(key, dfma=True).sigma(c, prec=sbci.SBCI_FP64)
    assert rel_err(s, s2) < TOL


def test_wide_dynamic_range_and_special_vectors():
    """Elements spread over 30 decades (each D row and W row scales itself); a
    zero vector gives exactly zero; one nonzero element."""
    sbci = require_lib()
    key = ("chain", 8, 1.3)
    ctx = _ctx(key)
    ora = oracle_sigma(key)
    rng = np.random.default_rng(5)
    c = rng.standard_normal(ctx.ndet) * 10.0 ** rng.uniform(-30, 0, ctx.ndet)
    s = ctx.sigma(c, prec=sbci.SBCI_FP64)
    ref = ora.apply(c.reshape(ora.Na, ora.Nb)).reshape(-1)
    assert rel_err(s, ref) < TOL
    z = ctx.sigma(np.zeros(ctx.ndet), prec=sbci.SBCI_FP64)
    assert not np.any(z)
    e = np.zeros(ctx.ndet)
    e[1234] = 1.0
    s1 = ctx.sigma(e, prec=sbci.SBCI_FP64)
    ref1 = ora.apply(e.reshape(ora.Na, ora.Nb)).reshape(-1)
    assert rel_err(s1, ref1) < TOL


def test_larger_spaces_keep_the_fma_kernel():
    sbci = require_lib()
    key = ("chain", 12, 1.2)  # npair = 78 > 55
    ctx = _ctx(key)
    c = np.random.default_rng(2).standard_normal(ctx.ndet)
    ctx.profile(True)
    ctx.sigma(c, prec=sbci.SBCI_FP64)
    stats = ctx.profile_read()
    ctx.profile(False)
    assert stats["sigma_gather_contract_os"][0] == 0 and stats["sigma_gather_contract"][0] == 1


def test_non_finite_input_propagates():
    """A NaN in a device input vector reaches sigma as non-finite values (the
    controller's numeric checks rely on it), as with the FMA kernel."""
    torch = pytest.importorskip("torch")
    sbci = require_lib()
    ctx = _ctx(("chain", 6, 1.0))
    c = torch.randn(ctx.ndet, dtype=torch.float64, device="cuda")
    c[37] = float("nan")
    s = torch.empty_like(c)
    ctx.sigma(c, s, prec=sbci.SBCI_FP64)
    assert not bool(torch.isfinite(s).all())
    c[37] = 0.0
    ctx.sigma(c, s, prec=sbci.SBCI_FP64)
    assert bool(torch.isfinite(s).all())
