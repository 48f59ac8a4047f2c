"""The library's buffer cache (csrc/pool.cpp, sbci_pool_stats / sbci_pool_trim).

Contexts and solves take their device and pinned host buffers from a cache of
freed blocks; a context created on recycled buffers must compute exactly
what one created on fresh memory computes (sigma and a batched solve of the
bench workload, bitwise), the second round of creations must be served from
the cache, and a trim must return the cache to CUDA.
"""
import numpy as np
import pytest

from gpu_common import make_integrals, require_lib

pytestmark = pytest.mark.gpu


def test_recycled_buffers_give_identical_results():
    sbci = require_lib()
    I = make_integrals(("chain", 10, 1.2))
    sbci.pool_trim()
    c = np.random.default_rng(3).standard_normal(63504)
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3)
    out = []
    for rnd in range(2):
        before = sbci.pool_stats()
        ctxs = [sbci.Context.from_integrals(I) for _ in range(4)]
        s = ctxs[0].sigma(c, prec=sbci.SBCI_FP64)
        E, _, st = sbci.solve_batch(ctxs, 2, p)
        assert st == sbci.SBCI_OK
        for x in ctxs:
            x.close()
        after = sbci.pool_stats()
        out.append((s, E, before, after))
    (s0, E0, b0, a0), (s1, E1, b1, a1) = out
    assert np.array_equal(s0, s1)
    assert np.array_equal(E0, E1)
    # the second round took its buffers from the cache, not from CUDA
    assert a1["hits"] - b1["hits"] > 0
    assert a1["misses"] - b1["misses"] < a0["misses"] - b0["misses"]
    assert a1["cached_bytes"] > 0
    sbci.pool_trim()
    assert sbci.pool_stats()["cached_bytes"] == 0


def test_contexts_made_in_parallel():
    """sbci_init_integrals_many: contexts made on the host worker threads give
    the sigma and the batched energies of contexts made one at a time
    (bitwise); an invalid request leaves no context."""
    sbci = require_lib()
    I = make_integrals(("chain", 10, 1.2))
    c = np.random.default_rng(9).standard_normal(63504)
    p = sbci.params(sector=1, prec=sbci.SBCI_TF32X3)
    many = sbci.Context.many(I.norb, I.nalpha, I.nbeta, I.h1, I.eri, I.e_core, n=4)
    one = [sbci.Context.from_integrals(I) for _ in range(4)]
    assert all(np.array_equal(a.sigma(c, prec=sbci.SBCI_FP64), b.sigma(c, prec=sbci.SBCI_FP64))
               for a, b in zip(many, one))
    Em, _, st1 = sbci.solve_batch(many, 2, p)
    Eo, _, st2 = sbci.solve_batch(one, 2, p)
    assert st1 == st2 == sbci.SBCI_OK and np.array_equal(Em, Eo)
    for x in many + one:
        x.close()
    with pytest.raises(sbci.SbciError) as e:
        sbci.Context.many(17, 1, 1, np.zeros((17, 17)), np.zeros((17,) * 4), 0.0, n=3)
    assert e.value.status == sbci.SBCI_ERR_INVALID
