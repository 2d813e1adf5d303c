"""GPU parity of the Nesterov-type update and the outer acceleration
(Sec. 4.3.5) against the FP64 oracle.

Tolerances: the standalone update within 1e-10 (FP64) / 2e-5 (FP32) of the
row scale, with the same number of inner steps; FP64 solves: the relative
error of every outer iteration within 1e-10, the same inner step counts and
the same acceleration decisions; FP32 solves: every iteration within 1e-4 and
the last within 1e-5 (5 % noise keeps the FP32 error identity, which moves
eps by about u_32 / eps, well inside that).
"""

import numpy as np
import pytest
import torch

import oracle as o
from helpers import factors_to_device, planc, x_to_device
from paper_1909_01149_gb300 import synth

pytestmark = pytest.mark.gpu


def _nls_problem(rows, R, seed, well_conditioned):
    rng = np.random.default_rng(seed)
    if well_conditioned:
        A = rng.standard_normal((4 * R + 3, R))
        S = A.T @ A
    else:  # Hadamard of Grams of uniform factors: eigenvalues spread widely
        G = [(lambda h: h.T @ h)(rng.random((d, R))) for d in (9, 11)]
        S = G[0] * G[1]
    H0 = rng.random((rows, R))
    M = (rng.random((rows, R)) - 0.2) @ S
    return S, M, H0


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("rows,R,well", [(1, 1, True), (37, 5, True), (200, 16, False),
                                         (65, 33, False), (130, 64, True), (40, 64, False)])
def test_nes_update(dt, rows, R, well):
    p = planc()
    S, M, H0 = _nls_problem(rows, R, rows * 10 + R, well)
    (Md, Hd), (Ms, Hs) = factors_to_device([M, H0], dt)
    Sd = torch.from_numpy(S).cuda()
    inner = torch.zeros(1, dtype=torch.int32, device="cuda")
    X = torch.ones(rows * 2, dtype=torch.float64 if dt == "f64" else torch.float32, device="cuda")
    with p.Context(X, (rows, 2), R) as ctx:
        ctx.nls_update("nes", Sd, Md, Hd, inner=inner)
        got = Hd.double().cpu().numpy()
    ref, k = o.nls_nes(S, Ms, Hs, return_state=True)
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-30)
    tol = 1e-10 if dt == "f64" else 2e-5
    err = float(np.max(np.abs(got - ref) / scale))
    assert err <= tol, err
    assert int(inner.item()) == k
    assert (got >= 0).all()


def test_nes_update_zero_gram_keeps_warm_start():
    p = planc()
    rows, R = 20, 4
    rng = np.random.default_rng(3)
    (Md, Hd), (_, Hs) = factors_to_device([rng.random((rows, R)), rng.random((rows, R))], "f64")
    inner = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    X = torch.ones(rows * 2, dtype=torch.float64, device="cuda")
    with p.Context(X, (rows, 2), R) as ctx:
        ctx.nls_update("nes", torch.zeros(R, R, dtype=torch.float64, device="cuda"), Md, Hd,
                       inner=inner)
        got = Hd.cpu().numpy()
    np.testing.assert_array_equal(got, Hs)
    assert int(inner.item()) == 0


def _planted(dims, R, seed, noise):
    X, _ = synth.planted(dims, R, seed, noise=noise)
    return X, synth.init_factors(dims, R, seed + 1)


@pytest.mark.parametrize("dims,R,accel", [((20, 24, 18), 4, True), ((9, 8, 10, 7), 3, True),
                                          ((20, 24, 18), 4, False), ((30, 5, 40), 8, True)])
def test_nes_solve_fp64_per_iteration(dims, R, accel):
    p = planc()
    X, H0 = _planted(dims, R, 41, 0.05)
    Xd, Xs = x_to_device(X, "f64")
    Hd, Hs = factors_to_device(H0, "f64")
    iters = 12
    with p.Context(Xd, dims, R) as ctx:
        res = ctx.solve(Hd, "nes", iters, nes_accel=accel)
    ref = o.nncp(Xs, Hs, "nes", iters=iters, nes_accel=accel)
    np.testing.assert_allclose(res["rel_err"], ref["rel_err"], rtol=0, atol=1e-10)
    assert res["inner"] == ref["inner"]
    if accel:
        assert res["accepted"][1:] == ref["accepted"]
        assert res["accel_accepted"] == sum(ref["accepted"])
    else:
        assert res["accel_accepted"] == 0
    np.testing.assert_allclose(res["lam"], ref["lam"], rtol=1e-9)
    for hd, hr in zip(Hd, ref["H"]):
        np.testing.assert_allclose(hd.cpu().numpy(), hr, rtol=0, atol=1e-9)


def test_nes_solve_fp32():
    p = planc()
    dims, R = (64, 48, 56), 8
    X, H0 = _planted(dims, R, 42, 0.05)
    Xd, Xs = x_to_device(X, "f32")
    Hd, Hs = factors_to_device(H0, "f32")
    with p.Context(Xd, dims, R) as ctx:
        res = ctx.solve(Hd, "nes", 10)
    ref = o.nncp(Xs, Hs, "nes", iters=10)
    np.testing.assert_allclose(res["rel_err"], ref["rel_err"], rtol=0, atol=1e-4)
    assert abs(res["rel_err"][-1] - ref["rel_err"][-1]) <= 1e-5


def test_nes_graph_and_stream_agree():
    p = planc()
    dims, R = (33, 17, 25), 6
    X, H0 = _planted(dims, R, 43, 0.05)
    Xd, _ = x_to_device(X, "f32")
    out = []
    for graph in (True, False):
        Hd, _ = factors_to_device(H0, "f32")
        with p.Context(Xd, dims, R) as ctx:
            out.append(ctx.solve(Hd, "nes", 8, use_graph=graph))
    assert out[0]["rel_err"] == out[1]["rel_err"]
    assert out[0]["accepted"] == out[1]["accepted"]
