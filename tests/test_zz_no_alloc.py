"""The allocation-free ||X||^2 entry point (planc_sqnorm_noalloc) against the
context-based planc_sqnorm and the FP64 oracle, through the C ABI.

It exists for callers that cannot allocate device memory when they need the
reduction (graph capture, externally owned memory pools, latency-critical
loops); its scratch is a fixed array inside the library, reused by every
call.  Two calls in a row on different inputs must each match the context
result and the oracle's sum over the stored values within the tolerance the
sqnorm parity test uses (1e-7 relative), so a stale scratch array, or a
mistake in the reduction both entry points share, would show.  This file is
collected last on purpose.
"""

import ctypes as C

import numpy as np
import pytest
import torch

import oracle as o
from helpers import planc, x_to_device

pytestmark = pytest.mark.gpu


def _noalloc(p, Xd, alpha):
    stream = torch.cuda.current_stream().cuda_stream
    return p.lib.planc_sqnorm_noalloc(p._DT[Xd.dtype], Xd.data_ptr(), Xd.numel(),
                                      alpha.data_ptr(), C.c_void_p(stream))


def test_noalloc_sqnorm_matches_context_twice():
    p = planc()
    cases = [((257, 129, 63), "f32", 11), ((96, 200, 41), "bf16", 12)]
    for dims, dt, seed in cases:
        X = np.random.default_rng(seed).random(dims)
        Xd, stored = x_to_device(X, dt)
        exact = o.sqnorm(stored)
        with p.Context(Xd, dims, 4) as ctx:
            ref = float(ctx.sqnorm().cpu()[0])
        alpha = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(p, Xd, alpha) == 0
        got = float(alpha.cpu()[0])
        assert abs(got - ref) <= 1e-7 * ref, (dt, got, ref)
        assert abs(got - exact) <= 1e-7 * exact, (dt, got, exact)


def test_noalloc_sqnorm_rejects_bad_sizes():
    p = planc()
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    X = torch.ones(8, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # n beyond the supported maximum is refused before any launch
    assert p.lib.planc_sqnorm_noalloc(1, X.data_ptr(), 1 << 41, alpha.data_ptr(), stream) == 2
    assert p.lib.planc_sqnorm_noalloc(1, X.data_ptr(), 0, alpha.data_ptr(), stream) == 2
    assert p.lib.planc_sqnorm_noalloc(1, None, 8, alpha.data_ptr(), stream) == 1
