"""Parity of the tcgen05 tensor-core partial MTTKRP against the FP64 oracle and
against the CUDA-core path, across shapes that exercise ragged row tiles,
ragged reduction stages, reduction splits, padded ranks and both root
branches.

Tolerance: per-entry relative <= 1e-5 (BF16 storage: the Khatri-Rao operand
is carried in three BF16 terms, about 2^-26 relative; FP32 storage: X and
the Khatri-Rao operand in two TF32 terms each, dropped term below 2^-22;
accumulation in FP32).
"""

import os

import numpy as np
import pytest
import torch

import oracle as o
from helpers import factors_to_device, max_rel, planc, x_to_device

pytestmark = pytest.mark.gpu

TC_CASES = [
    ((64, 48, 80), 16, -1),        # both branches on tensor cores
    ((8, 37, 300), 32, 2),         # L = 296: ragged last row tile
    ((256, 3, 1000), 7, 2),        # R = 7 padded to 16
    ((16, 16, 5000), 24, 2),       # long right reduction: many k-splits
    ((128, 8, 97, 5), 64, 2),      # R = 64 (MMA N = 192), 4-way
    ((512, 1030), 5, 1),           # N = 2: both branches are leaves
    ((40, 40, 40, 40), 16, 2),     # 4-way, L = 1600
    # right branch in 32-row block mode (L / I_1 a multiple of 32, not of 128)
    ((40, 96, 50), 16, 2),         # L / I_1 = 96, ragged last row tile
    ((16, 32, 7, 9), 32, 2),       # L / I_1 = 32, 4-way
    ((24, 160, 33), 64, 2),        # L / I_1 = 160, R = 64
    # right branch with L / I_1 = 128 and R <= 16: BF16 X reduces two output
    # rows per epilogue round (more items than CTAs, pairs and an odd last item)
    ((32, 128, 400), 16, 2),
    ((32, 128, 333), 12, 2),       # R = 12 padded to 16
    # BF16 right branch as one GEMM against the split Khatri-Rao image:
    # R = 1, R = 17 (padded to 32), a single row tile with fewer units than SMs
    ((24, 40, 130), 1, 2),
    ((16, 24, 200), 17, 2),
    ((8, 8, 9, 3), 32, 2),
    # FP32 right branch as the converter GEMM with R = 64 (trailing part 2304)
    ((16, 16, 48, 48), 64, 2),
]


def _ctx_and_refs(dims, R, split, dt="bf16", seed=0):
    rng = np.random.default_rng(seed)
    X = rng.random(dims)
    H = [rng.random((d, R)) for d in dims]
    Xd, Xs = x_to_device(X, dt)
    Hd, Hs = factors_to_device(H, "f32")
    return Xd, Xs, Hd, Hs


@pytest.mark.parametrize("dt", ["bf16", "f32"])
@pytest.mark.parametrize("dims,R,split", TC_CASES)
def test_tc_mttkrp_matches_oracle(dims, R, split, dt):
    p = planc()
    Xd, Xs, Hd, Hs = _ctx_and_refs(dims, R, split, dt)
    with p.Context(Xd, dims, R, split) as ctx:
        assert ctx.tc_mask == 3, "expected both partial MTTKRPs on the tensor cores"
        for n in range(len(dims)):
            M = ctx.mttkrp(Hd, n).double().cpu().numpy()
            assert max_rel(M, o.mttkrp(Xs, Hs, n)) <= 1e-5, (n, max_rel(M, o.mttkrp(Xs, Hs, n)))


@pytest.mark.parametrize("dt", ["bf16", "f32"])
@pytest.mark.parametrize("dims,R,split", TC_CASES[:4])
def test_tc_partials_match_cuda_core_path(dims, R, split, dt, monkeypatch):
    p = planc()
    Xd, Xs, Hd, Hs = _ctx_and_refs(dims, R, split, dt, seed=1)
    with p.Context(Xd, dims, R, split) as ctx:
        assert ctx.tc_mask == 3
        T_tc = [ctx.partial_mttkrp(Hd, s).double().cpu().numpy() for s in (0, 1)]
    monkeypatch.setenv("PLANC_PM_PATH", "simt")
    with p.Context(Xd, dims, R, split) as ctx:
        assert ctx.tc_mask == 0
        T_simt = [ctx.partial_mttkrp(Hd, s).double().cpu().numpy() for s in (0, 1)]
    for a, b in zip(T_tc, T_simt):
        assert max_rel(a, b) <= 2e-5


@pytest.mark.parametrize("dt", ["bf16", "f32"])
def test_tc_not_used_when_rows_are_not_16_byte_strided(dt):
    p = planc()
    dims, R = (33, 65, 17), 5  # split 1: L = 33 elements is not a multiple of 16 bytes
    Xd, Xs, Hd, Hs = _ctx_and_refs(dims, R, 1, dt)
    with p.Context(Xd, dims, R, 1) as ctx:
        assert ctx.tc_mask & 1 == 0
        for n in range(3):
            M = ctx.mttkrp(Hd, n).double().cpu().numpy()
            assert max_rel(M, o.mttkrp(Xs, Hs, n)) <= 1e-5


def test_tc_fp32_solve_matches_oracle():
    """FP32 storage on the tensor cores: final error of a HALS solve within
    1e-5 of the oracle's."""
    p = planc()
    import oracle as o
    from paper_1909_01149_gb300 import synth
    dims, R = (64, 40, 36), 8  # L = 2560 -> both branches eligible
    X, _ = synth.planted(dims, R, 3, noise=0.05)
    Xd, Xs = x_to_device(X, "f32")
    H0 = synth.init_factors(dims, R, 4)
    Hd, Hs = factors_to_device(H0, "f32")
    with p.Context(Xd, dims, R) as ctx:
        assert ctx.tc_mask == 3
        res = ctx.solve(Hd, "hals", 15)
    ref = o.nncp(Xs, Hs, "hals", iters=15)
    assert abs(res["rel_err"][-1] - ref["rel_err"][-1]) <= 1e-5


def test_tc_solve_matches_cuda_core_solve(monkeypatch):
    """A whole BPP solve on BF16 storage: tensor-core and CUDA-core partial
    MTTKRPs give the same relative-error trajectory to 1e-6."""
    p = planc()
    from paper_1909_01149_gb300 import synth
    dims, R = (48, 40, 30, 12), 8
    X, _ = synth.mouse_like(dims, R, data_seed=5)
    Xd, _ = x_to_device(X, "bf16")
    out = []
    for path in ("auto", "simt"):
        if path == "simt":
            monkeypatch.setenv("PLANC_PM_PATH", "simt")
        Hd, _ = factors_to_device(synth.init_factors(dims, R, 6), "f32")
        with p.Context(Xd, dims, R) as ctx:
            assert (ctx.tc_mask != 0) == (path == "auto")
            out.append(ctx.solve(Hd, "bpp", 8)["rel_err"])
    np.testing.assert_allclose(out[0], out[1], rtol=0, atol=1e-6)


@pytest.mark.parametrize("dims,R,split", [((64, 48, 80), 16, -1), ((16, 24, 200), 17, 2),
                                          ((32, 128, 400), 16, 2), ((128, 8, 97, 5), 32, 2)])
def test_bf16_gemm_branches_match_weighted_rows(dims, R, split, monkeypatch):
    """Both BF16 partial MTTKRPs as one GEMM against the split Khatri-Rao
    image and the weighted-row kernels (PLANC_PM_KRP=0) agree, and both
    match the oracle to 1e-5 per entry."""
    p = planc()
    Xd, Xs, Hd, Hs = _ctx_and_refs(dims, R, split, "bf16", seed=3)
    outs = []
    for krp in ("1", "0"):
        monkeypatch.setenv("PLANC_PM_KRP", krp)
        with p.Context(Xd, dims, R, split) as ctx:
            assert ctx.tc_mask == 3
            outs.append([ctx.partial_mttkrp(Hd, s).double().cpu().numpy() for s in (0, 1)])
            for n in range(len(dims)):
                M = ctx.mttkrp(Hd, n).double().cpu().numpy()
                assert max_rel(M, o.mttkrp(Xs, Hs, n)) <= 1e-5, n
    for a, b in zip(outs[0], outs[1]):
        assert max_rel(a, b) <= 2e-6


@pytest.mark.parametrize("dims,R,split", [((256, 3, 1000), 7, 2), ((16, 16, 5000), 24, 2),
                                          ((16, 16, 48, 48), 64, 2), ((40, 40, 40, 40), 16, 2)])
def test_fp32_right_branch_gemm_matches_weighted_rows(dims, R, split, monkeypatch):
    """FP32 storage, right branch with a long trailing part (the Khatri-Rao
    image small next to X): the converter GEMM and the weighted-row kernel
    (PLANC_PM_KRP=0) agree, and every mode matches the oracle to 1e-5."""
    p = planc()
    Xd, Xs, Hd, Hs = _ctx_and_refs(dims, R, split, "f32", seed=5)
    outs = []
    for krp in ("1", "0"):
        monkeypatch.setenv("PLANC_PM_KRP", krp)
        with p.Context(Xd, dims, R, split) as ctx:
            assert ctx.tc_mask == 3
            outs.append(ctx.partial_mttkrp(Hd, 1).double().cpu().numpy())
            for n in range(len(dims)):
                M = ctx.mttkrp(Hd, n).double().cpu().numpy()
                assert max_rel(M, o.mttkrp(Xs, Hs, n)) <= 1e-5, n
    assert max_rel(outs[0], outs[1]) <= 2e-6

