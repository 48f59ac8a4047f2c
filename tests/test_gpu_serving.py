"""Serving layer (continuous batching): each result is the same alone and in the
mix, admission respects the memory budget, oversize requests are refused.

Tolerance: 1e-10 hartree between a solve run alone and the same solve run in
the mix.  Each solve's arithmetic does not depend on what else runs (fixed
grids, fixed-order reductions), so the two are expected to agree to the last
bit; 1e-10 is the stated bound.
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


@pytest.mark.parametrize("prec", ["TF32X3", "FP64"])
def test_same_alone_and_in_mix(prec):
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
    server = sbci.Server(8 << 30, 4)
    tickets = [server.submit(I, k, p) for I, (_, _, k) in zip(ints, MIX)]
    res = _drain(server, tickets)
    for t, Ea in zip(tickets, alone):
        E, R, times, st = res[t]
        assert st == sbci.SBCI_OK
        assert np.abs(E - Ea).max() <= 1e-10
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
        assert np.abs(res[t][0] - Ea).max() <= 1e-10
    server.close()


def test_oversize_request_refused():
    sbci = require_lib()
    server = sbci.Server(1 << 20, 2)
    with pytest.raises(sbci.SbciError) as e:
        server.submit(inputs.h_chain(8, 1.0), 1)
    assert e.value.status == sbci.SBCI_ERR_NOMEM
    server.close()
