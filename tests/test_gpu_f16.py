"""FP16 storage on the tensor cores: both partial MTTKRPs as one tcgen05 GEMM
each against the Khatri-Rao image split into three FP16 terms, every column
scaled by a power of two into FP16's range (undone exactly after the sum).

Tolerances as for BF16 storage: per-entry relative <= 1e-5 against the FP64
oracle run on the FP16-rounded tensor (three FP16 terms carry about 33 bits of
each scaled entry; accumulation in FP32); the tensor-core and CUDA-core
partial MTTKRPs within 2e-6 of each other; a HALS solve's final error within
1e-5 of the oracle's, a BPP solve's within 1e-3 (the mixed-precision bar).
"""

import numpy as np
import pytest

import oracle as o
from paper_1909_01149_gb300 import synth
from helpers import factors_to_device, max_rel, planc, x_to_device

pytestmark = pytest.mark.gpu

# shapes whose branches are eligible (R <= 32, the row stride of X_(1:S) a
# multiple of 16 bytes): ragged row tiles, padded ranks, long reductions,
# 4-way, R = 1 and R = 17 (padded to 32)
F16_CASES = [
    ((64, 48, 80), 16, -1),
    ((16, 16, 5000), 24, 2),
    ((40, 40, 40, 40), 16, 2),
    ((24, 40, 130), 1, 2),
    ((16, 24, 200), 17, 2),
    ((8, 8, 9, 3), 32, 2),
    ((32, 128, 333), 12, 2),
]


def _inputs(dims, R, seed, spread=None):
    rng = np.random.default_rng(seed)
    X = rng.random(dims)
    if spread is None:
        H = [rng.random((d, R)) for d in dims]
    else:  # entries 10^U[-spread, spread): products far outside FP16's range
        H = [10.0 ** rng.uniform(-spread, spread, (d, R)) for d in dims]
    Xd, Xs = x_to_device(X, "f16")
    Hd, Hs = factors_to_device(H, "f32")
    return Xd, Xs, Hd, Hs


@pytest.mark.parametrize("dims,R,split", F16_CASES)
def test_f16_mttkrp_on_tensor_cores_matches_oracle(dims, R, split):
    p = planc()
    Xd, Xs, Hd, Hs = _inputs(dims, R, 11)
    with p.Context(Xd, dims, R, split) as ctx:
        assert ctx.tc_mask == 3, "expected both partial MTTKRPs on the tensor cores"
        for n in range(len(dims)):
            M = ctx.mttkrp(Hd, n).double().cpu().numpy()
            ref = o.mttkrp(Xs, Hs, n)
            assert max_rel(M, ref) <= 1e-5, (n, max_rel(M, ref))


@pytest.mark.parametrize("dims,R,split", [((64, 48, 80), 16, -1), ((16, 24, 200), 17, 2)])
def test_f16_factor_entries_spanning_twelve_decades(dims, R, split):
    """Factor entries 10^U[-6, 6): Khatri-Rao entries from 1e-18 to 1e18, each
    column with its own scale; every MTTKRP entry still within 1e-5."""
    p = planc()
    Xd, Xs, Hd, Hs = _inputs(dims, R, 12, spread=6)
    with p.Context(Xd, dims, R, split) as ctx:
        assert ctx.tc_mask == 3
        for n in range(len(dims)):
            M = ctx.mttkrp(Hd, n).double().cpu().numpy()
            ref = o.mttkrp(Xs, Hs, n)
            assert max_rel(M, ref) <= 1e-5, (n, max_rel(M, ref))


@pytest.mark.parametrize("dims,R,split", F16_CASES[:3])
def test_f16_tensor_cores_match_cuda_cores(dims, R, split, monkeypatch):
    p = planc()
    Xd, Xs, Hd, Hs = _inputs(dims, R, 13)
    with p.Context(Xd, dims, R, split) as ctx:
        assert ctx.tc_mask == 3
        T_tc = [ctx.partial_mttkrp(Hd, s).double().cpu().numpy() for s in (0, 1)]
    monkeypatch.setenv("PLANC_PM_KRP", "0")  # FP16 then has no tensor-core kernel
    with p.Context(Xd, dims, R, split) as ctx:
        assert ctx.tc_mask == 0
        T_simt = [ctx.partial_mttkrp(Hd, s).double().cpu().numpy() for s in (0, 1)]
    for a, b in zip(T_tc, T_simt):
        assert max_rel(a, b) <= 2e-6


def test_f16_rank_above_32_stays_on_cuda_cores():
    p = planc()
    dims, R = (32, 24, 40), 40
    Xd, Xs, Hd, Hs = _inputs(dims, R, 14)
    with p.Context(Xd, dims, R) as ctx:
        assert ctx.tc_mask == 0
        for n in range(3):
            M = ctx.mttkrp(Hd, n).double().cpu().numpy()
            assert max_rel(M, o.mttkrp(Xs, Hs, n)) <= 1e-5


def test_f16_hals_solve_matches_oracle():
    p = planc()
    dims, R = (64, 40, 36), 8
    X, _ = synth.planted(dims, R, 15, noise=0.05)
    Xd, Xs = x_to_device(X, "f16")
    Hd, Hs = factors_to_device(synth.init_factors(dims, R, 16), "f32")
    with p.Context(Xd, dims, R) as ctx:
        assert ctx.tc_mask == 3
        res = ctx.solve(Hd, "hals", 15)
    ref = o.nncp(Xs, Hs, "hals", iters=15)
    np.testing.assert_allclose(res["rel_err"], ref["rel_err"], rtol=0, atol=1e-5)


def test_f16_mouse_like_bpp_solve_matches_oracle():
    p = planc()
    dims, R = (24, 32, 30, 10), 4
    X, _ = synth.mouse_like(dims, R, data_seed=3)
    Xd, Xs = x_to_device(X, "f16")
    Hd, Hs = factors_to_device(synth.init_factors(dims, R, 17), "f32")
    with p.Context(Xd, dims, R) as ctx:
        assert ctx.tc_mask != 0
        res = ctx.solve(Hd, "bpp", 10)
    ref = o.nncp(Xs, Hs, "bpp", iters=10)
    assert abs(res["rel_err"][-1] - ref["rel_err"][-1]) <= 1e-3
