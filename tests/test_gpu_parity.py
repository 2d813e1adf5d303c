"""GPU parity: every step of the hot path through the C ABI against the FP64
oracle on the same seeded inputs.

Tolerances (written where used):
  MTTKRP, FP32 storage/accumulation: per-entry relative <= 1e-5 (all entries
  are positive, so relative error is well defined); FP64: 1e-12.
  BF16/F16 storage: per-entry relative <= 1e-5 against the oracle run on the
  rounded tensor (the Khatri-Rao operand stays FP32).
  Grams/normalisation: FP32 products summed in FP32 over at most a few dozen
  rows then in FP64: relative 1e-6 (FP32) / 1e-13 (FP64).
  NNLS updates: relative 2e-5 of the row scale (FP32 arithmetic over R-term
  dot products, compounded over one HALS sweep).
  Full FP32 solves: final relative error within 1e-5; FP64: 1e-10 per
  iteration; BF16-storage solves: within 1e-3.
"""

import numpy as np
import pytest
import torch

import oracle as o
from paper_1909_01149_gb300 import synth
from helpers import factors_to_device, max_rel, planc, x_to_device

pytestmark = pytest.mark.gpu

MTTKRP_CASES = [
    ((37, 29, 41), 1), ((37, 29, 41), 2),
    ((13, 11, 17, 9), 1), ((13, 11, 17, 9), 2), ((13, 11, 17, 9), 3),
    ((5, 7, 3, 6, 4), 1), ((5, 7, 3, 6, 4), 2), ((5, 7, 3, 6, 4), 3), ((5, 7, 3, 6, 4), 4),
    ((300, 5, 200), 1), ((300, 5, 200), 2),
    ((1, 5, 7), 1), ((6, 1, 1), 2), ((130, 257), 1),
]


@pytest.mark.parametrize("dims,split", MTTKRP_CASES)
@pytest.mark.parametrize("R", [1, 8, 17, 32])
@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_mttkrp_every_mode(dims, split, R, dt):
    p = planc()
    rng = np.random.default_rng(hash((dims, split, R)) % 2**32)
    X = rng.random(dims)
    H = [rng.random((d, R)) for d in dims]
    Xd, Xs = x_to_device(X, dt)
    Hd, Hs = factors_to_device(H, dt)
    tol = 1e-5 if dt == "f32" else 1e-12
    with p.Context(Xd, dims, R, split) as ctx:
        assert ctx.split == split
        for n in range(len(dims)):
            M = ctx.mttkrp(Hd, n).double().cpu().numpy()
            ref = o.mttkrp(Xs, Hs, n)
            assert max_rel(M, ref) <= tol, (n, max_rel(M, ref))


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("dims,R", [((64, 48, 80), 16), ((24, 20, 30, 10), 8), ((33, 65, 17), 5)])
def test_mttkrp_16bit_storage(dims, R, dt):
    p = planc()
    rng = np.random.default_rng(7)
    X = rng.random(dims)
    H = [rng.random((d, R)) for d in dims]
    Xd, Xs = x_to_device(X, dt)
    Hd, Hs = factors_to_device(H, "f32")
    with p.Context(Xd, dims, R) as ctx:
        for n in range(len(dims)):
            M = ctx.mttkrp(Hd, n).double().cpu().numpy()
            assert max_rel(M, o.mttkrp(Xs, Hs, n)) <= 1e-5


@pytest.mark.parametrize("dims,split,R", [((37, 29, 41), 2, 32), ((13, 11, 17, 9), 2, 16),
                                          ((40, 700, 3), 1, 8)])
def test_partial_mttkrp_both_sides(dims, split, R):
    """T^{1:S} = X_(1:S) K^{S+1:N} and T^{S+1:N} = X_(1:S)^T K^{1:S}
    (Sec. 4.2.2), R-slowest layout."""
    p = planc()
    rng = np.random.default_rng(3)
    X = rng.random(dims)
    H = [rng.random((d, R)) for d in dims]
    Xd, Xs = x_to_device(X, "f32")
    Hd, Hs = factors_to_device(H, "f32")
    L = int(np.prod(dims[:split]))
    Cc = int(np.prod(dims[split:]))
    X12 = np.reshape(Xs, (L, Cc), order="F")
    with p.Context(Xd, dims, R, split) as ctx:
        T0 = ctx.partial_mttkrp(Hd, 0).double().cpu().numpy().reshape(R, L).T
        T1 = ctx.partial_mttkrp(Hd, 1).double().cpu().numpy().reshape(R, Cc).T
    K_right = o.khatri_rao([Hs[k] for k in range(len(dims) - 1, split - 1, -1)])
    K_left = o.khatri_rao([Hs[k] for k in range(split - 1, -1, -1)])
    assert max_rel(T0, X12 @ K_right) <= 1e-5
    assert max_rel(T1, X12.T @ K_left) <= 1e-5


def test_sqnorm():
    p = planc()
    for dt, tol in (("f32", 1e-7), ("f64", 1e-13), ("bf16", 1e-7)):
        X = np.random.default_rng(1).random((101, 37, 53))
        Xd, Xs = x_to_device(X, dt)
        with p.Context(Xd, X.shape, 4) as ctx:
            a = float(ctx.sqnorm().cpu()[0])
        assert abs(a - o.sqnorm(Xs)) <= tol * o.sqnorm(Xs)


@pytest.mark.parametrize("R", [1, 8, 32, 64])
def test_gram_hadamard_bit_exact(R):
    p = planc()
    N = 4
    rng = np.random.default_rng(R)
    G = rng.random((N, R, R))
    Gd = torch.from_numpy(G).cuda()
    X = torch.ones(2 * 3 * 4 * 5, dtype=torch.float64, device="cuda")
    with p.Context(X, (2, 3, 4, 5), R) as ctx:
        for n in range(N):
            S = ctx.gram_hadamard(Gd, n).cpu().numpy()
            np.testing.assert_array_equal(S, o.gram_hadamard(list(G), n))


@pytest.mark.parametrize("dt,rows,R", [("f32", 512, 32), ("f32", 77, 5), ("f64", 64, 8),
                                       ("f32", 1000, 64), ("f32", 1, 3)])
def test_gram_and_normalize(dt, rows, R):
    p = planc()
    rng = np.random.default_rng(rows + R)
    Hh = rng.random((rows, R))
    if R > 3:
        Hh[:, 2] = 0.0  # a zero column keeps lambda = 0 and stays zero
    X = torch.ones(rows * 2, dtype=torch.float64 if dt == "f64" else torch.float32,
                   device="cuda")
    tol = 1e-6 if dt == "f32" else 1e-13
    with p.Context(X, (rows, 2), R) as ctx:
        Hd, Hs = factors_to_device([Hh], dt)
        G = ctx.gram(Hd[0]).cpu().numpy()
        np.testing.assert_allclose(G, o.gram(Hs[0]), rtol=tol, atol=tol * np.abs(G).max())
        Gn = torch.empty((R, R), dtype=torch.float64, device="cuda")
        Hn, lam = ctx.normalize(Hd[0], G=Gn)
        H_ref, lam_ref = o.normalize_columns(Hs[0])
        np.testing.assert_allclose(lam.cpu().numpy(), lam_ref, rtol=tol)
        np.testing.assert_allclose(Hn.double().cpu().numpy(), H_ref, rtol=tol * 10,
                                   atol=1e-7 if dt == "f32" else 1e-15)
        Gr = o.gram(Hn.double().cpu().numpy())
        np.testing.assert_allclose(Gn.cpu().numpy(), Gr, rtol=tol, atol=tol)


def _nls_problem(rows, R, seed, dims_other=(9, 11)):
    """S and M from real Khatri-Rao structure: S = *_k G^(k), M = X_(n) K."""
    rng = np.random.default_rng(seed)
    dims = (rows,) + dims_other
    X = rng.random(dims)
    H = [rng.random((d, R)) for d in dims]
    S = o.gram_hadamard([o.gram(h) for h in H], 0)
    M = o.mttkrp(X, H, 0)
    return S, M, H[0]


@pytest.mark.parametrize("alg", ["mu", "hals", "pgd", "admm", "bpp"])
@pytest.mark.parametrize("dt,rows,R", [("f32", 512, 32), ("f32", 77, 5), ("f64", 64, 8),
                                       ("f32", 130, 16), ("f32", 40, 64)])
def test_nls_update(alg, dt, rows, R):
    p = planc()
    S, M, H0 = _nls_problem(rows, R, rows * 100 + R)
    X = torch.ones(rows * 2, dtype=torch.float64 if dt == "f64" else torch.float32,
                   device="cuda")
    (Md, Hd), (Ms, Hs) = factors_to_device([M, H0], dt)
    Sd = torch.from_numpy(S).cuda()
    inner = torch.zeros(1, dtype=torch.int32, device="cuda")
    with p.Context(X, (rows, 2), R) as ctx:
        ctx.nls_update(alg, Sd, Md, Hd, inner=inner)
        got = Hd.double().cpu().numpy()
    if alg == "mu":
        ref = o.nls_mu(S, Ms, Hs)
    elif alg == "hals":
        ref = o.nls_hals(S, Ms, Hs)
    elif alg == "pgd":
        ref = o.nls_pgd(S, Ms, Hs)
    elif alg == "admm":
        ref, _, k = o.nls_admm(S, Ms, Hs, return_state=True)
        assert int(inner.item()) == k
    else:
        ref, k, ok = o.nls_bpp(S, Ms, Hs)
        assert ok
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-30)
    tol = 2e-5 if dt == "f32" else 1e-11
    err = float(np.max(np.abs(got - ref) / scale))
    assert err <= tol, err
    assert (got >= 0).all()


def test_bpp_kkt_on_device():
    p = planc()
    S, M, H0 = _nls_problem(200, 16, 5)
    M = M - 0.4 * M.mean()  # activate constraints in many rows
    X = torch.ones(400, dtype=torch.float64, device="cuda")
    (Md, Hd), _ = factors_to_device([M, H0], "f64")
    with p.Context(X, (200, 2), 16) as ctx:
        ctx.nls_update("bpp", torch.from_numpy(S).cuda(), Md, Hd)
        x = Hd.cpu().numpy()
    y = x @ S - M
    assert x.min() >= 0 and y.min() > -1e-9 and np.abs(x * y).max() < 1e-9
    ref, _, _ = o.nls_bpp(S, M, H0)
    np.testing.assert_allclose(x, ref, rtol=1e-9, atol=1e-12)


def test_fit_identity_on_device():
    p = planc()
    dims, R = (30, 22, 26), 5
    X, _ = synth.planted(dims, R, 4, noise=0.1)
    Xd, Xs = x_to_device(X, "f64")
    H = synth.init_factors(dims, R, 5)
    Hn = [o.normalize_columns(h)[0] for h in H]
    lam = np.linspace(0.5, 2.0, R)
    Hd, Hs = factors_to_device(Hn, "f64")
    with p.Context(Xd, dims, R) as ctx:
        eps, fit = ctx.fit(Hd, torch.from_numpy(lam).cuda())
    ref, _ = o.fit_explicit(Xs, Hs, lam)
    assert abs(eps - ref) < 1e-10
    assert abs(fit - (1 - ref)) < 1e-10


def _solve_both(dims, R, alg, iters, dt, seed=1, noise=0.05, split=-1, Xgen=None):
    p = planc()
    if Xgen is None:
        X, _ = synth.planted(dims, R, seed, noise=noise)
    else:
        X = Xgen
    Xd, Xs = x_to_device(X, dt)
    H0 = synth.init_factors(dims, R, seed + 1)
    fdt = "f64" if dt == "f64" else "f32"
    Hd, Hs = factors_to_device(H0, fdt)
    with p.Context(Xd, dims, R, split) as ctx:
        res = ctx.solve(Hd, alg=alg, iters=iters)
    ref = o.nncp(Xs, Hs, alg, iters=iters)
    return res, ref, Hd


def test_solve_fp64_hals_config_small_per_iteration():
    """64^3 FP64, R = 8, HALS, 20 outer iterations, 1% noise: the relative
    error of every outer iteration within 1e-10 of the oracle's."""
    res, ref, Hd = _solve_both((64, 64, 64), 8, "hals", 20, "f64", noise=0.01)
    assert res["iters"] == 20
    np.testing.assert_allclose(res["rel_err"], ref["rel_err"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(res["lam"], ref["lam"], rtol=1e-9)
    for h, hr in zip(Hd, ref["H"]):
        np.testing.assert_allclose(h.cpu().numpy(), hr, rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("alg", ["mu", "hals", "admm", "bpp", "pgd"])
@pytest.mark.parametrize("dims,split", [((30, 41, 52), -1), ((12, 9, 14, 11), 2),
                                        ((12, 9, 14, 11), 1)])
def test_solve_fp32_final_fit(alg, dims, split):
    res, ref, _ = _solve_both(dims, 6, alg, 12, "f32", split=split)
    assert abs(res["rel_err"][-1] - ref["rel_err"][-1]) <= 1e-5
    # the inner-step counts of ADMM/BPP follow the oracle's for the first sweep
    if alg == "admm":
        assert res["inner"][:len(dims)] == ref["inner"][:len(dims)]


def test_solve_bf16_mouse_like_bpp():
    dims, R = (24, 20, 30, 10), 4
    X, _ = synth.mouse_like(dims, R, data_seed=3)
    res, ref, _ = _solve_both(dims, R, "bpp", 10, "bf16", Xgen=X)
    assert abs(res["rel_err"][-1] - ref["rel_err"][-1]) <= 1e-3


def test_solve_graph_and_stream_paths_agree():
    p = planc()
    dims, R = (20, 24, 28), 5
    X, _ = synth.planted(dims, R, 2, noise=0.05)
    Xd, _ = x_to_device(X, "f32")
    outs = []
    for graph in (True, False):
        Hd, _ = factors_to_device(synth.init_factors(dims, R, 3), "f32")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with p.Context(Xd, dims, R, stream=s) as ctx:
                outs.append(ctx.solve(Hd, "hals", 8, use_graph=graph)["rel_err"])
    assert outs[0] == outs[1]  # bit-identical: same kernels, fixed reduction order


def test_zero_tensor_and_degenerate_columns():
    """All-zero X: MU keeps zeros, lambda = 0, eps = 0 (guarded alpha = 0)."""
    p = planc()
    dims, R = (6, 7, 8), 3
    Xd = torch.zeros(int(np.prod(dims)), dtype=torch.float32, device="cuda")
    Hd, _ = factors_to_device(synth.init_factors(dims, R, 1), "f32")
    with p.Context(Xd, dims, R) as ctx:
        res = ctx.solve(Hd, "mu", 3)
    assert res["rel_err"][-1] == 0.0
    assert all(l == 0.0 for l in res["lam"])


def test_invalid_arguments_are_errors_not_crashes():
    p = planc()
    X = torch.ones(24, device="cuda")
    with pytest.raises((ValueError, p.PlancError)):
        p.Context(X, (2, 3, 0), 4)
    with pytest.raises(p.PlancError):
        p.Context(X, (24,), 4)
    with pytest.raises(p.PlancError):
        p.Context(X, (2, 3, 4), 0)
    with pytest.raises(p.PlancError):
        p.Context(X, (2, 3, 4), 4, split=3)
    with p.Context(X, (2, 3, 4), 4) as ctx:
        Hd, _ = factors_to_device([np.ones((2, 4)), np.ones((3, 4)), np.ones((4, 4))], "f32")
        with pytest.raises(p.PlancError):
            ctx.mttkrp(Hd, 5)
