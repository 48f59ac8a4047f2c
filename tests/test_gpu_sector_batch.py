"""The singlet-sector (c = c^T) batched TF32x3 path: the engine that the bench
line times (16 solves of H10 at 1.2 A, 4 states, through sbci_solve_batch),
the same path with uneven sizes, and the batched server in the sector.

Tolerances: the energies after FP64 refinement are held to the FP64 target,
1e-8 hartree, against exact sector energies of the oracle (Lanczos on the
symmetrised oracle sigma); a batched solve and the same solve run alone give
bitwise the same energies (fixed partitions and reduction orders, shared
kernel bodies compiled without implicit contraction).
"""
import time

import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs

from gpu_common import make_integrals, oracle_sector_energies, require_lib

pytestmark = pytest.mark.gpu

E_TOL = 1e-8


def _alone(sbci, I, k, p):
    ctx = sbci.Context.from_integrals(I)
    E, _, R, st = ctx.solve(k, p)
    ctx.close()
    assert st == sbci.SBCI_OK and all(r.converged for r in R)
    return E


def test_bench_config_h10_sector_batch16():
    """The bench workload: 16 H10 contexts, sector 1, TF32x3, k = 4."""
    sbci = require_lib()
    key = ("chain", 10, 1.2)
    I = make_integrals(key)
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3)
    ctxs = [sbci.Context.from_integrals(I) for _ in range(16)]
    E, R, st = sbci.solve_batch(ctxs, 4, p)
    assert st == sbci.SBCI_OK
    assert all(r.converged for r in R)
    Ea = _alone(sbci, I, 4, p)
    ref = oracle_sector_energies(key, 4) + I.e_core
    for i in range(16):
        assert np.array_equal(E[i], Ea), np.abs(E[i] - Ea).max()
        err = np.abs(np.sort(E[i]) - ref)
        assert err.max() < E_TOL, err
    for c in ctxs:
        c.close()


def test_init_stage_h10_sector_batch():
    """init_stage = 1 (the start's H-products in TF32x3): 8 batched H10
    solves equal the solve run alone bit for bit and meet the oracle's exact
    sector energies to the FP64 target after refinement; the start itself
    (sbci_begin) runs its H-products (one per start vector: two here, the
    four lowest determinants being two transposed pairs) on the tensor-core
    kernel instead of the FP64 one."""
    sbci = require_lib()
    key = ("chain", 10, 1.2)
    I = make_integrals(key)
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3, init_stage=1)
    ctxs = [sbci.Context.from_integrals(I) for _ in range(8)]
    E, R, st = sbci.solve_batch(ctxs, 4, p)
    assert st == sbci.SBCI_OK
    assert all(r.converged for r in R)
    Ea = _alone(sbci, I, 4, p)
    ref = oracle_sector_energies(key, 4) + I.e_core
    for i in range(8):
        assert np.array_equal(E[i], Ea), np.abs(E[i] - Ea).max()
        err = np.abs(np.sort(E[i]) - ref)
        assert err.max() < E_TOL, err
    for c in ctxs:
        c.close()
    ctx = sbci.Context.from_integrals(I)
    counts = {}
    for stage in (0, 1):
        ctx.profile(False)  # resets the launch counts
        ctx.begin(4, sbci.params(sector=1, prec=sbci.SBCI_TF32X3, init_stage=stage))
        st = ctx.profile_read()
        counts[stage] = (st.get("sigma_gather_contract_os", (0, 0.0))[0],
                         st.get("sigma_gather_contract_tc", (0, 0.0))[0])
    _, _, R1, st1 = ctx.solve(4, p)
    ctx.close()
    m = counts[0][0]
    assert m >= 1 and counts[0][1] == 0 and counts[1] == (0, m), counts
    assert st1 == sbci.SBCI_OK and all(r.converged for r in R1)
    assert all(r.n_sigma_fp64 >= 1 for r in R1)  # every state ends on FP64 H-products


def test_sector_batch_uneven_sizes():
    """H6 / H8 / H10 / H12 in the sector, one batch: each equals its solve run
    alone bit for bit; H6-H10 meet the oracle's exact sector energies and H12
    (853,776 determinants, beyond a quick oracle eigen-solve) the FP64 solve,
    which the FP64 tests pin to the oracle."""
    sbci = require_lib()
    keys = [("chain", 6, 1.0), ("chain", 8, 1.3), ("chain", 10, 1.2), ("chain", 12, 1.2), ("chain", 10, 2.0)]
    k = 2
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3)
    ints = [make_integrals(key) for key in keys]
    ctxs = [sbci.Context.from_integrals(I) for I in ints]
    E, R, st = sbci.solve_batch(ctxs, k, p)
    assert st == sbci.SBCI_OK
    assert all(r.converged for r in R)
    for i, (key, I) in enumerate(zip(keys, ints)):
        Ea = _alone(sbci, I, k, p)
        assert np.array_equal(E[i], Ea), (key, np.abs(E[i] - Ea).max())
        if key[1] <= 10:
            ref = oracle_sector_energies(key, k) + I.e_core
        else:
            ref = _alone(sbci, I, k, sbci.params(sector=1, prec=sbci.SBCI_FP64))
        err = np.abs(np.sort(E[i]) - np.sort(ref))
        assert err.max() < E_TOL, (key, err)
    for c in ctxs:
        c.close()


def test_sector_server_same_alone_and_in_mix():
    """The batched server with sector 1: requests of uneven sizes arrive while
    others run, and each result equals the solve run alone bit for bit."""
    sbci = require_lib()
    mix = [(6, 1.0, 2), (10, 1.2, 4), (8, 1.3, 3), (10, 2.2, 1), (6, 2.0, 1), (8, 0.9, 2)]
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3)
    ints = [inputs.h_chain(n, R) for n, R, _ in mix]
    alone = [_alone(sbci, I, k, p) for I, (_, _, k) in zip(ints, mix)]
    server = sbci.Server(8 << 30, 3, batching=True)
    tickets, out = [], {}
    t0 = time.time()
    # staggered arrivals: half now, the rest while the first ones are on the GPU
    for I, (_, _, k) in list(zip(ints, mix))[:3]:
        tickets.append(server.submit(I, k, p))
    server.progress()
    for I, (_, _, k) in list(zip(ints, mix))[3:]:
        tickets.append(server.submit(I, k, p))
    while len(out) < len(tickets):
        server.progress()
        for t in tickets:
            if t not in out:
                r = server.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < 300, "server did not finish in time"
    for t, Ea in zip(tickets, alone):
        E, R, _, st = out[t]
        assert st == sbci.SBCI_OK and all(r.converged for r in R)
        assert np.array_equal(E, Ea), np.abs(E - Ea).max()
    server.close()


def test_sector_batch_runs_the_column_kernel():
    """The batched sector H10 loop body is update, projection, column-fused
    sigma, symmetric finish and end: no tile kernel, no scatter, G never in
    global memory.  Same energies under kernel timing as through the graph."""
    sbci = require_lib()
    I = make_integrals(("chain", 10, 1.2))
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3)
    ctxs = [sbci.Context.from_integrals(I) for _ in range(4)]
    E0, _, st = sbci.solve_batch(ctxs, 2, p)
    assert st == sbci.SBCI_OK
    sbci.batch_profile(True)
    E1, _, st = sbci.solve_batch(ctxs, 2, p)
    stats = sbci.batch_profile_read()
    sbci.batch_profile(False)
    assert st == sbci.SBCI_OK and np.array_equal(E0, E1)
    bodies = stats["batch_end"][0]
    assert bodies > 0
    for k in ("batch_update", "batch_project", "batch_fused_column", "batch_symfinish"):
        assert stats[k][0] == bodies and stats[k][1] > 0.0, k
    assert stats["batch_gather_contract_tc"][0] == 0 and stats["batch_scatter"][0] == 0
    # (earlier tests met mixed tables: H12 sector jobs take the tile kernel)
    cls = [c for c in sbci.batch_classes() if "fused_column" in c["ctas"] and "tensor_core" not in c["ctas"]]
    assert cls
    for c in ctxs:
        c.close()
