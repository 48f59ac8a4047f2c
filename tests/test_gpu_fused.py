"""The column-fused sigma of singlet-sector TF32x3 steps (one CTA builds one
column of the alpha part A: gather, tcgen05 contraction and alpha-only
scatter, with G kept in shared memory).

It forms the same D, the same TF32 split, the same MMAs and the same
summation order of the scatter as the tile kernel + scatter pair, so a solve
with it and the same solve with SBCI_FUSED=0 (tile kernel + scatter, G in
global memory) take the same trajectory: the test requires the same energies
to 1e-12 hartree and the same trace, step by step.  Energies are held to the
oracle's exact sector energies at the FP64 target, 1e-8 hartree.
"""
import os

import numpy as np
import pytest

from gpu_common import make_integrals, oracle_sector_energies, require_lib

pytestmark = pytest.mark.gpu


def _ctx(sbci, I, fused: bool):
    old = os.environ.get("SBCI_FUSED")
    os.environ["SBCI_FUSED"] = "1" if fused else "0"
    try:
        return sbci.Context.from_integrals(I)
    finally:
        if old is None:
            del os.environ["SBCI_FUSED"]
        else:
            os.environ["SBCI_FUSED"] = old


@pytest.mark.parametrize("key,k", [(("chain", 10, 1.2), 4), (("chain", 6, 1.0), 3), (("chain", 8, 1.3), 3),
                                   # edge shapes: 6 strings per spin (one partial tile), 66 strings with
                                   # 78 pairs (Np = 80: the second accumulator at a 128-column offset),
                                   # 220 strings with 78 pairs (two tiles, Kp = 80)
                                   (("chain", 4, 1.1), 2), (("rand", 12, 5, 2, 2), 2), (("rand", 12, 6, 3, 3), 2)])
def test_fused_column_same_trajectory_as_tile_path(key, k):
    sbci = require_lib()
    I = make_integrals(key)
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3)
    out = {}
    for fused in (True, False):
        ctx = _ctx(sbci, I, fused)
        ctx.profile(False)
        E, _, R, st = ctx.solve(k, p)
        assert st == sbci.SBCI_OK and all(r.converged for r in R)
        launches = {n: v[0] for n, v in ctx.profile_read().items() if v[0]}
        out[fused] = (E, [(t.state, t.event, t.energy) for t in ctx.trace()], launches)
        ctx.close()
    Ef, trf, lf = out[True]
    Et, trt, lt = out[False]
    # the fused solve ran the column kernel and neither the tile kernel nor the scatter
    assert lf.get("sigma_fused_column", 0) > 0
    assert "sigma_gather_contract_tc" not in lf
    assert lt.get("sigma_gather_contract_tc", 0) > 0 and "sigma_fused_column" not in lt
    assert np.abs(Ef - Et).max() < 1e-12, np.abs(Ef - Et).max()
    assert len(trf) == len(trt)
    assert [t[:2] for t in trf] == [t[:2] for t in trt]
    assert max(abs(a[2] - b[2]) for a, b in zip(trf, trt)) < 1e-12
    ref = oracle_sector_energies(key, k) + I.e_core
    assert np.abs(np.sort(Ef) - ref).max() < 1e-8


def test_fused_column_step_by_step():
    """sbci_step drives the same kernels one body at a time: the records of
    the first steps of the fused and the tile path agree to 1e-12."""
    sbci = require_lib()
    I = make_integrals(("chain", 10, 1.2))
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3)
    recs = {}
    for fused in (True, False):
        ctx = _ctx(sbci, I, fused)
        ctx.begin(2, p)
        r = []
        for _ in range(40):
            rec, done = ctx.step()
            r.append((rec.state, rec.t, rec.event, rec.energy, rec.b, rec.c, rec.k))
            if done:
                break
        recs[fused] = r
        ctx.close()
    a, b = recs[True], recs[False]
    assert len(a) == len(b) >= 20
    for x, y in zip(a, b):
        assert x[:3] == y[:3]
        assert np.allclose(x[3:], y[3:], rtol=1e-12, atol=1e-14)
