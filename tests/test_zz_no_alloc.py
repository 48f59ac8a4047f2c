"""sbci_sigma_noalloc: the FP64 sigma with a fixed static scratch, for callers
that cannot allocate (stream captures, pool-owning frameworks, latency loops).

Collected last on purpose.  Checks, through the C ABI, that two calls in a row
give what sbci_sigma gives (same FP64 tolerance as the other sigma tests),
that device free memory does not shrink across them once the first (set-up)
call on the device has been made, and that an oversized space is rejected with
a clear error.
"""
import numpy as np
import pytest

from paper_2603_06101_gb300 import inputs

from gpu_common import make_integrals, require_lib

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("key", [("chain", 6, 1.0), ("chain", 10, 1.2)])
def test_noalloc_matches_sigma_twice(key):
    import torch

    sbci = require_lib()
    I = make_integrals(key)
    ctx = sbci.Context.from_integrals(I)
    c1 = torch.from_numpy(inputs.random_vector(ctx.na, ctx.nb, 51)).cuda()
    c2 = torch.from_numpy(inputs.random_vector(ctx.na, ctx.nb, 52)).cuda()
    ref1 = ctx.sigma(c1)
    ref2 = ctx.sigma(c2)
    out1 = torch.empty_like(c1)
    out2 = torch.empty_like(c2)
    # the first call on a device is the set-up: it looks up the scratch address,
    # which (with lazy module loading) commits the static array itself
    ctx.sigma_noalloc(c2, out1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx.sigma_noalloc(c1, out1)
    ctx.sigma_noalloc(c2, out2)  # second call in a row on the shared scratch
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert _rel(out1, ref1) < FP64_TOL
    assert _rel(out2, ref2) < FP64_TOL
    assert free1 >= free0  # no device allocation happened during the calls


def test_noalloc_rejects_oversized_space():
    import torch

    sbci = require_lib()
    I = make_integrals(("chain", 12, 1.2))  # 78 * 853,776 * 8 B > 32 MiB
    ctx = sbci.Context.from_integrals(I)
    c = torch.zeros(ctx.ndet, dtype=torch.float64, device="cuda")
    out = torch.empty_like(c)
    with pytest.raises(sbci.SbciError) as e:
        ctx.sigma_noalloc(c, out)
    assert e.value.status == sbci.SBCI_ERR_INVALID
    assert "use sbci_sigma" in str(e.value)
