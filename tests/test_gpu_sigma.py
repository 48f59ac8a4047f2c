"""GPU parity of the string tables, the diagonal and sigma = H c against the oracle.

All calls go through the C ABI (ctypes binding).  Tolerances: tables bit-exact;
FP64 sigma within 1e-12 relative to max|sigma| (rounding of sums of at most
2 nlink * npair products of O(1) numbers); the FP32 contraction within 2e-5.
"""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs
from oracle import slater_condon as sc
from oracle import strings as st

from gpu_common import make_integrals, oracle_sigma, rel_err, require_lib

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def ctx_for(key):
    sbci = require_lib()
    return sbci.Context.from_integrals(make_integrals(key))


@pytest.mark.parametrize("n,m", [(6, 3), (7, 2), (8, 5), (10, 5), (14, 7), (16, 8), (5, 0), (5, 5)])
def test_string_tables_bit_exact(n, m):
    sbci = require_lib()
    I = inputs.random_df(n, 1, m, max(1, n // 2) if m == 0 else m)
    ctx = sbci.Context.from_integrals(I)
    tab = ctx.string_table(0)
    ref = st.excitation_list(n, m)
    assert tab.shape[:2] == ref.shape[:2]
    pair = np.array([[st.pair_index(int(k), int(l)) for k, l, _, _ in row] for row in ref]).reshape(tab.shape[:2])
    assert np.array_equal(tab[..., 0], pair)
    assert np.array_equal(tab[..., 1], ref[..., 2])
    assert np.array_equal(tab[..., 2], ref[..., 3])


@pytest.mark.parametrize("key", [("chain", 6, 1.0), ("rand", 7, 3, 4, 3), ("rand", 9, 4, 5, 3)])
def test_diagonal(key):
    I = make_integrals(key)
    ctx = ctx_for(key)
    d = ctx.diagonal()
    ref = sc.diagonal_by_occupation(I.h1, I.eri, I.nalpha, I.nbeta)
    assert np.abs(d - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    if ctx.ndet <= 1225:
        assert np.abs(d - sc.diagonal(I.h1, I.eri, I.nalpha, I.nbeta)).max() < 1e-12 * np.abs(ref).max()


SIGMA_CASES = [
    ("chain", 4, 1.0),        # 36 dets: one ragged tile
    ("chain", 6, 1.0),        # 400 dets: 7 tiles, ragged tail
    ("chain", 8, 1.3),        # 4900
    ("rand", 7, 5, 4, 3),     # nalpha != nbeta
    ("rand", 9, 6, 5, 3),     # 10584, ragged
    ("rand", 4, 8, 0, 2),     # no alpha electrons
    ("rand", 5, 9, 5, 1),     # full alpha shell
    ("rand", 3, 10, 1, 1),
    ("chain", 10, 1.2),       # the H10 workload size, 63504
]


@pytest.mark.parametrize("key", SIGMA_CASES)
def test_sigma_fp64_matches_oracle(key):
    ctx = ctx_for(key)
    ora = oracle_sigma(key)
    c = np.stack([inputs.random_vector(ctx.na, ctx.nb, s) for s in (11, 12)])
    out = ctx.sigma(c)
    for v in range(2):
        ref = ora.apply(c[v])
        assert rel_err(out[v], ref) < FP64_TOL


def test_sigma_device_pointers_and_determinism():
    import torch

    key = ("chain", 8, 1.3)
    ctx = ctx_for(key)
    c = inputs.random_vector(ctx.na, ctx.nb, 3)
    ct = torch.from_numpy(c).cuda()
    o1 = ctx.sigma(ct)
    o2 = ctx.sigma(ct)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)  # gather form, fixed-order sums: bitwise reproducible
    ref = oracle_sigma(key).apply(c)
    assert rel_err(o1.cpu().numpy(), ref) < FP64_TOL


def test_sigma_fp32_contraction_bound():
    sbci = require_lib()
    key = ("chain", 10, 1.2)
    ctx = ctx_for(key)
    c = inputs.random_vector(ctx.na, ctx.nb, 5)
    s64 = ctx.sigma(c, prec=sbci.SBCI_FP64)
    s32 = ctx.sigma(c, prec=sbci.SBCI_FP32)
    assert rel_err(s32, s64) < 2e-5


def test_sigma_random_df_n14_sampled_rows():
    """The 11.8M-determinant random-DF workload: sampled rows against the
    Slater-Condon rows of the oracle, and Hermiticity u.(Hv) = (Hu).v."""
    import torch

    I = make_integrals(("rand", 14, 14, 7, 7))
    sbci = require_lib()
    ctx = sbci.Context.from_integrals(I)
    assert ctx.ndet == 3432 * 3432
    u = torch.from_numpy(inputs.random_vector(3432, 3432, 21)).cuda()
    v = torch.from_numpy(inputs.random_vector(3432, 3432, 22)).cuda()
    Hu = ctx.sigma(u)
    Hv = ctx.sigma(v)
    rows = np.random.default_rng(7).choice(ctx.ndet, 24, replace=False)
    ref = sc.sampled_sigma_rows(I.h1, I.eri, 7, 7, u.cpu().numpy(), rows)
    got = Hu.reshape(-1)[torch.from_numpy(rows).cuda()].cpu().numpy()
    scale = float(Hu.abs().max())
    assert np.abs(got - ref).max() < FP64_TOL * scale
    a = float((u * Hv).sum())
    b = float((Hu * v).sum())
    assert abs(a - b) < 1e-12 * max(1.0, abs(a))
