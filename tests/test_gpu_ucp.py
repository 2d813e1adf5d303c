"""GPU parity of the unconstrained update (UCP, CP-ALS) against the FP64
oracle: the standalone update (FP64 1e-10, FP32 1e-4 of the row scale: the
update multiplies by S^{-1}, whose condition number on these inputs is
~1e2), whole solves (FP64 relative error of every outer iteration within
1e-10, FP32 the last one within 1e-5) and the singular-S error."""

import numpy as np
import pytest
import torch

import oracle as o
from helpers import factors_to_device, planc, x_to_device

pytestmark = pytest.mark.gpu


def _normal_problem(dims, R, seed, noise=0.01):
    rng = np.random.default_rng(seed)
    A = [rng.standard_normal((d, R)) for d in dims]
    X = o.cp_full(A)
    X = X + noise * np.abs(X).mean() * rng.standard_normal(X.shape)
    H0 = [a + 0.3 * rng.standard_normal(a.shape) for a in A]
    return X, H0


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("rows,R", [(1, 1), (37, 5), (200, 16), (65, 33)])
def test_ucp_update(dt, rows, R):
    p = planc()
    rng = np.random.default_rng(rows * 10 + R)
    A = rng.standard_normal((3 * R + 2, R))
    S = A.T @ A
    M = rng.standard_normal((rows, R))
    (Md, Hd), (Ms, _) = factors_to_device([M, np.zeros((rows, R))], dt)
    Sd = torch.from_numpy(S).cuda()
    X = torch.ones(rows * 2, dtype=torch.float64 if dt == "f64" else torch.float32, device="cuda")
    with p.Context(X, (rows, 2), R) as ctx:
        ctx.nls_update("ucp", Sd, Md, Hd)
        got = Hd.double().cpu().numpy()
    ref = o.nls_ucp(S, Ms)
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-30)
    tol = 1e-10 if dt == "f64" else 1e-4
    assert float(np.max(np.abs(got - ref) / scale)) <= tol


@pytest.mark.parametrize("dims,R", [((20, 24, 18), 4), ((9, 8, 10, 7), 3)])
def test_ucp_solve_fp64_per_iteration(dims, R):
    p = planc()
    X, H0 = _normal_problem(dims, R, 31)
    Xd, Xs = x_to_device(X, "f64")
    Hd, Hs = factors_to_device(H0, "f64")
    with p.Context(Xd, dims, R) as ctx:
        res = ctx.solve(Hd, "ucp", 15)
    ref = o.nncp(Xs, Hs, "ucp", iters=15)
    np.testing.assert_allclose(res["rel_err"], ref["rel_err"], rtol=0, atol=1e-10)


def test_ucp_solve_fp32():
    """FP32: the error identity subtracts O(1) terms to get eps^2, so its
    FP32 rounding moves eps by about u_32 / eps; 5 % noise (eps ~ 0.03) keeps
    that well under the 1e-5 bar of the other FP32 solves."""
    p = planc()
    dims, R = (64, 48, 56), 8
    X, H0 = _normal_problem(dims, R, 32, noise=0.05)
    Xd, Xs = x_to_device(X, "f32")
    Hd, Hs = factors_to_device(H0, "f32")
    with p.Context(Xd, dims, R) as ctx:
        res = ctx.solve(Hd, "ucp", 10)
    ref = o.nncp(Xs, Hs, "ucp", iters=10)
    assert ref["rel_err"][-1] > 0.02
    np.testing.assert_allclose(res["rel_err"], ref["rel_err"], rtol=0, atol=1e-4)
    assert abs(res["rel_err"][-1] - ref["rel_err"][-1]) <= 1e-5


def test_ucp_singular_gram_is_a_numeric_error():
    """A zero column in two factors makes S^(n) singular for the third mode."""
    p = planc()
    dims, R = (6, 7, 8), 3
    X, H0 = _normal_problem(dims, R, 33)
    H0[1][:, 2] = 0.0
    H0[2][:, 2] = 0.0
    Xd, _ = x_to_device(X, "f64")
    Hd, _ = factors_to_device(H0, "f64")
    with p.Context(Xd, dims, R) as ctx:
        with pytest.raises(p.PlancError) as ei:
            ctx.solve(Hd, "ucp", 2)
    assert ei.value.status == 6  # PLANC_E_NUMERIC
