"""GPU parity of the fused per-mode update (one thread-block-cluster launch per
mode for factors of at most 1024 rows and R <= 32, MU / HALS / PGD) against
the FP64 oracle and against the multi-kernel path on the same inputs.

Tolerances: FP64 solves, the relative error of every outer iteration within
1e-10 of the oracle's and lambda within 1e-9 relative; FP32 solves, the final
relative error within 1e-5 (the same bars as the other solve tests).  The two
device paths run the same arithmetic in a different reduction order, so they
are compared with the oracle's tolerance, not bit for bit.
"""

import numpy as np
import pytest
import torch

import oracle as o
from paper_1909_01149_gb300 import synth
from helpers import factors_to_device, planc, x_to_device

pytestmark = pytest.mark.gpu


def _solve(monkeypatch, fused, X, dims, R, alg, iters, dt, seed):
    monkeypatch.setenv("PLANC_FUSED_MODES", "1" if fused else "0")
    p = planc()
    Xd, _ = x_to_device(X, dt)
    fdt = "f64" if dt == "f64" else "f32"
    Hd, _ = factors_to_device(synth.init_factors(dims, R, seed + 1), fdt)
    with p.Context(Xd, dims, R) as ctx:
        res = ctx.solve(Hd, alg=alg, iters=iters)
    return res, Hd


CASES = [
    # (dims, R): rows per mode across the cluster's row split, padding of R
    ((30, 41, 52), 6),
    ((30, 41, 52), 17),
    ((64, 9, 33), 32),
    ((1, 40, 33), 5),            # a one-row factor
    ((1024, 6, 5), 8),           # the largest fused factor
    ((1025, 6, 5), 8),           # one row more: that mode takes the multi-kernel path
    ((12, 9, 14, 11), 16),
]


@pytest.mark.parametrize("alg", ["hals", "mu", "pgd"])
@pytest.mark.parametrize("dims,R", CASES)
def test_fused_fp64_per_iteration(monkeypatch, alg, dims, R):
    X, _ = synth.planted(dims, R, 4, noise=0.02)
    _, Xs = x_to_device(X, "f64")
    H0 = synth.init_factors(dims, R, 5)
    ref = o.nncp(Xs, [np.asarray(h, dtype=np.float64) for h in H0], alg, iters=6)
    fused, Hf = _solve(monkeypatch, True, X, dims, R, alg, 6, "f64", 4)
    multi, Hm = _solve(monkeypatch, False, X, dims, R, alg, 6, "f64", 4)
    for res in (fused, multi):
        np.testing.assert_allclose(res["rel_err"], ref["rel_err"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(res["lam"], ref["lam"], rtol=1e-9, atol=1e-300)
    for a, b in zip(Hf, Hm):
        np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=1e-9, atol=1e-13)
    # the fused path launches fewer kernels whenever some mode is eligible
    if min(dims) <= 1024:
        assert fused["launches"] < multi["launches"]


@pytest.mark.parametrize("alg", ["hals", "mu", "pgd"])
@pytest.mark.parametrize("dims,R", [((30, 41, 52), 6), ((200, 130, 97), 32),
                                    ((512, 40, 64), 32)])
def test_fused_fp32_final_fit(monkeypatch, alg, dims, R):
    X, _ = synth.planted(dims, R, 6, noise=0.05)
    _, Xs = x_to_device(X, "f32")
    H0 = synth.init_factors(dims, R, 7)
    Hs = [torch.from_numpy(np.asarray(h)).float().double().numpy() for h in H0]
    ref = o.nncp(Xs, Hs, alg, iters=8)
    fused, _ = _solve(monkeypatch, True, X, dims, R, alg, 8, "f32", 6)
    assert abs(fused["rel_err"][-1] - ref["rel_err"][-1]) <= 1e-5


def test_fused_repeatable(monkeypatch):
    """Fixed reduction order: two runs give bit-identical histories."""
    dims, R = (300, 200, 100), 32
    X, _ = synth.planted(dims, R, 8, noise=0.05)
    a, _ = _solve(monkeypatch, True, X, dims, R, "hals", 5, "f32", 8)
    b, _ = _solve(monkeypatch, True, X, dims, R, "hals", 5, "f32", 8)
    assert a["rel_err"] == b["rel_err"]
    assert a["lam"] == b["lam"]
