"""Serving layer (continuous batching): each result is the same alone and in the
mix, admission respects the memory budget, oversize requests are refused.

Tolerance: none — a solve run alone and the same solve run in the mix agree
bit for bit.  Each solve's arithmetic does not depend on what else runs (fixed
virtual-block partitions, fixed-order reductions), and the one-solve and the
batched kernels call the same compiled bodies, so the energies are compared
for exact equality.
"""
import time

import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs

from gpu_common import require_lib

pytestmark = pytest.mark.gpu

MIX = [(6, 1.0, 2), (8, 1.3, 3), (10, 1.2, 1), (6, 2.0, 4), (8, 0.9, 2), (6, 1.5, 1), (10, 2.2, 2)]


def _drain(server, tickets, timeout_s=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        server.progress()
        for t in tickets:
            if t not in out:
                r = server.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout_s, "server did not finish in time"
    return out


@pytest.mark.parametrize("prec,batching", [("TF32X3", True), ("TF32X3", False), ("FP64", True)])
def test_same_alone_and_in_mix(prec, batching):
    """batching = True and TF32X3: the solves share the batched persistent kernels."""
    sbci = require_lib()
    p = sbci.params(prec=getattr(sbci, "SBCI_" + prec))
    ints = [inputs.h_chain(n, R) for n, R, _ in MIX]
    alone = []
    for I, (_, _, k) in zip(ints, MIX):
        ctx = sbci.Context.from_integrals(I)
        E, _, R, st = ctx.solve(k, p)
        assert st == sbci.SBCI_OK
        alone.append(E)
        ctx.close()
    server = sbci.Server(8 << 30, 4, batching=batching)
    tickets = [server.submit(I, k, p) for I, (_, _, k) in zip(ints, MIX)]
    res = _drain(server, tickets)
    for t, Ea in zip(tickets, alone):
        E, R, times, st = res[t]
        assert st == sbci.SBCI_OK
        assert np.array_equal(E, Ea), np.abs(E - Ea).max()
        assert all(r.converged for r in R)
    server.close()


def test_admission_by_memory_budget():
    sbci = require_lib()
    I = inputs.h_chain(10, 1.2)
    p = sbci.params(prec=sbci.SBCI_TF32X3)
    ctx = sbci.Context.from_integrals(I)
    Ea, _, _, _ = ctx.solve(1, p)
    ctx.close()
    # about 40 MB per H10 one-state solve: the budget admits one at a time
    server = sbci.Server(48 << 20, 4)
    tickets = [server.submit(I, 1, p) for _ in range(3)]
    active, queued = server.progress()
    assert active == 1 and queued == 2
    res = _drain(server, tickets)
    queue_times = [res[t][2][0] for t in tickets]
    assert queue_times[2] > 0.0 and queue_times[2] >= queue_times[0]
    for t in tickets:
        assert np.array_equal(res[t][0], Ea)
    server.close()


def test_oversize_request_refused():
    sbci = require_lib()
    server = sbci.Server(1 << 20, 2)
    with pytest.raises(sbci.SbciError) as e:
        server.submit(inputs.h_chain(8, 1.0), 1)
    assert e.value.status == sbci.SBCI_ERR_NOMEM
    server.close()


def test_solve_batch_same_as_alone():
    """sbci_solve_batch: solves of uneven sizes share the batched persistent
    kernels; each result equals the solve run alone."""
    sbci = require_lib()
    p = sbci.params(prec=sbci.SBCI_TF32X3)
    ints = [inputs.h_chain(n, R) for n, R in [(6, 1.0), (10, 1.2), (8, 1.3), (6, 2.0), (12, 1.2)]]
    k = 2
    alone = []
    for I in ints:
        ctx = sbci.Context.from_integrals(I)
        E, _, _, st = ctx.solve(k, p)
        assert st == sbci.SBCI_OK
        alone.append(E)
        ctx.close()
    ctxs = [sbci.Context.from_integrals(I) for I in ints]
    E, R, st = sbci.solve_batch(ctxs, k, p)
    assert st == sbci.SBCI_OK
    for i in range(len(ints)):
        assert np.array_equal(E[i], alone[i]), np.abs(E[i] - alone[i]).max()
    for c in ctxs:
        c.close()


def test_batch_profile_same_result():
    """Kernel timing of the batch engine launches the same kernels one by one:
    same energies as the graph loop, every family counted and timed."""
    sbci = require_lib()
    p = sbci.params(prec=sbci.SBCI_TF32X3)
    ints = [inputs.h_chain(n, R) for n, R in [(8, 1.0), (10, 1.4), (6, 1.1)]]
    ctxs = [sbci.Context.from_integrals(I) for I in ints]
    E0, _, st = sbci.solve_batch(ctxs, 2, p)
    assert st == sbci.SBCI_OK
    n_graph = sbci.solve_batch.last_launches
    sbci.batch_profile(True)
    E1, _, st = sbci.solve_batch(ctxs, 2, p)
    assert st == sbci.SBCI_OK
    stats = sbci.batch_profile_read()
    sbci.batch_profile(False)
    assert np.array_equal(E1, E0)
    assert set(stats) == {"batch_update", "batch_project", "batch_gather_contract_tc", "batch_fused_column",
                          "batch_scatter", "batch_symfinish", "batch_end", "batch_host_halted"}
    assert stats.pop("batch_host_halted")[0] > 0  # (halted solves handled between rounds)
    bodies = stats["batch_end"][0]
    # every solve of this mix is outside the singlet sector: the tile kernel and
    # the scatter run, the column kernel and the symmetric finish do not
    used = {"batch_update", "batch_project", "batch_gather_contract_tc", "batch_scatter", "batch_end"}
    assert bodies > 0 and all(stats[k][0] == bodies and stats[k][1] > 0.0 for k in used)
    assert stats["batch_fused_column"][0] == 0 and stats["batch_symfinish"][0] == 0
    assert n_graph >= 5 * bodies  # the graph loop ran the same bodies (plus host-driven kernels)
    for c in ctxs:
        c.close()
