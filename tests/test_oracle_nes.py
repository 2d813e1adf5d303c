"""Pins for the oracle's Nesterov-type update and outer acceleration
(Sec. 4.3.5, Eq. nesnls, Eq. nesinnerupd, Eq. nesouterupd).

The parameters are checked against closed forms; the uncapped inner
iteration against SciPy's Lawson-Hanson NNLS of the plain problem (no
proximal term) and of the proximal problem written as one stacked least
squares problem; the momentum against the linear-rate bound of the
accelerated projected gradient method for strongly convex objectives (which
the method without momentum breaks); the outer acceleration against an
explicit reconstruction of the extrapolated model.
"""

import importlib
import math

import numpy as np
import pytest

import oracle as o

onn = importlib.import_module("oracle.nncp")


def _rotated(eigs, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((len(eigs), len(eigs))))
    return Q @ np.diag(eigs) @ Q.T


def test_nes_params_closed_forms():
    # well conditioned: no proximal term, beta from mu0 / L0
    lam_p, L, beta = o.nes_params(np.diag([2.0, 1.0]))
    q = 0.5
    assert lam_p == 0.0 and L == 2.0
    assert beta == pytest.approx((1 - math.sqrt(q)) / (1 + math.sqrt(q)), rel=1e-15)
    # condition 1e4: lam_p = (1 - 100e-4) / 99 = 0.01, then L / mu = 100 exactly
    lam_p, L, beta = o.nes_params(np.diag([1.0, 1e-4, 0.5]))
    assert lam_p == pytest.approx(0.01, rel=1e-13)
    assert L == pytest.approx(1.01, rel=1e-13)
    assert beta == pytest.approx(0.9 / 1.1, rel=1e-12)
    # eigenvalues, not diagonal entries, decide: a rotated S gives the same
    got = o.nes_params(_rotated([1.0, 1e-4, 0.5], 3))
    for a, b in zip(got, (0.01, 1.01, 0.9 / 1.1)):
        assert a == pytest.approx(b, rel=1e-10)
    # singular S: mu0 = 0, lam_p = L0 / 99
    lam_p, L, beta = o.nes_params(np.diag([3.0, 0.0]))
    assert lam_p == pytest.approx(3.0 / 99, rel=1e-14)
    assert L == pytest.approx(3.0 + 3.0 / 99, rel=1e-14)
    # S = 0: no step
    assert o.nes_params(np.zeros((3, 3)))[1] == 0.0


def _stacked_nnls(A, b):
    scipy_opt = pytest.importorskip("scipy.optimize")
    return scipy_opt.nnls(A, b, maxiter=1000)[0]


def test_nes_uncapped_reaches_nnls_solution():
    """Well-conditioned S (lam_p = 0): the iteration converges to the NNLS
    minimiser of each row, min 1/2||A x - b||^2, x >= 0."""
    rng = np.random.default_rng(5)
    R, rows = 6, 9
    A = rng.random((4 * R, R)) + np.eye(4 * R, R) * 2.0
    B = rng.standard_normal((4 * R, rows))
    S = A.T @ A
    assert o.nes_params(S)[0] == 0.0
    M = (A.T @ B).T
    H0 = rng.random((rows, R))
    got = o.nls_nes(S, M, H0, max_inner=5000, tol=0.0)
    ref = np.stack([_stacked_nnls(A, B[:, i]) for i in range(rows)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)
    assert (ref == 0).any()  # some constraints are active


def test_nes_uncapped_reaches_proximal_solution():
    """Ill-conditioned S (lam_p > 0): the limit is the minimiser of f_p, i.e.
    NNLS of the stacked problem [A; sqrt(lam_p) I] x = [b; sqrt(lam_p) x*]."""
    rng = np.random.default_rng(6)
    R, rows = 5, 7
    S = _rotated([4.0, 1.0, 0.3, 1e-3, 1e-6], 7)
    lam_p, L, _ = o.nes_params(S)
    assert lam_p > 0
    A = np.linalg.cholesky(S).T  # S = A^T A
    B = rng.standard_normal((R, rows))
    M = (A.T @ B).T
    Hs = rng.random((rows, R))
    got = o.nls_nes(S, M, Hs, max_inner=20000, tol=0.0)
    As = np.vstack([A, math.sqrt(lam_p) * np.eye(R)])
    ref = np.stack([_stacked_nnls(As, np.concatenate([B[:, i], math.sqrt(lam_p) * Hs[i]]))
                    for i in range(rows)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)


def _fp(S, M, Hs, lam_p, X):
    return (0.5 * np.sum((X @ S) * X) - np.sum(M * X)
            + 0.5 * lam_p * np.sum((X - Hs) ** 2))


def _rate_check(beta_override=None):
    """Largest ratio, over k, of f_p(X_k) - f* to the accelerated bound
    (f_p(X_0) - f* + mu/2 ||X_0 - X*||^2) (1 - sqrt(mu/L))^k."""
    rng = np.random.default_rng(8)
    R, rows = 8, 4
    S = _rotated(np.geomspace(1.0, 1e-2, R), 9)  # condition 100: lam_p = 0
    M = rng.standard_normal((rows, R)) * 0.5
    Hs = rng.random((rows, R))
    lam_p, L, beta = o.nes_params(S)
    assert lam_p == pytest.approx(0.0, abs=1e-12)
    mu = np.linalg.eigvalsh(S)[0] + lam_p
    Xs = o.nls_nes(S, M, Hs, max_inner=20000, tol=0.0)
    fstar = _fp(S, M, Hs, lam_p, Xs)
    c0 = _fp(S, M, Hs, lam_p, Hs) - fstar + 0.5 * mu * np.sum((Hs - Xs) ** 2)
    worst = 0.0
    orig = onn.nes_params
    try:
        if beta_override is not None:
            onn.nes_params = lambda S_, kappa=o.NES_KAPPA: orig(S_, kappa)[:2] + (beta_override,)
        for k in range(1, 80):
            Xk = onn.nls_nes(S, M, Hs, max_inner=k, tol=0.0)
            bound = c0 * (1 - math.sqrt(mu / L)) ** k
            worst = max(worst, (_fp(S, M, Hs, lam_p, Xk) - fstar) / bound)
    finally:
        onn.nes_params = orig
    return worst


def test_nes_momentum_meets_the_accelerated_rate():
    assert _rate_check() <= 1.0 + 1e-9


def test_rate_check_catches_dropped_momentum():
    # planted mistake in the oracle (CPU only): no momentum breaks the bound
    assert _rate_check(beta_override=0.0) > 1.0


def test_nes_fixed_point_stops_after_one_step():
    """A warm start that already solves the (lam_p = 0) problem: X_1 = Y_0,
    so the stopping rule holds after the first step and H* is returned."""
    rng = np.random.default_rng(10)
    R, rows = 4, 6
    A = rng.random((3 * R, R)) + np.eye(3 * R, R)
    S = A.T @ A
    X = np.abs(rng.standard_normal((rows, R)))
    X[:, 0] = 0.0
    M = X @ S
    M[:, 0] -= 1.0  # column 0 active: gradient +1 at the bound
    got, k = o.nls_nes(S, M, X, return_state=True)
    assert k == 1
    np.testing.assert_allclose(got, X, rtol=0, atol=1e-13)


def test_nes_inner_cap_and_zero_gram():
    rng = np.random.default_rng(11)
    S = _rotated([1.0, 1e-3, 1e-5], 12)
    M = rng.standard_normal((5, 3))
    H = rng.random((5, 3))
    _, k = o.nls_nes(S, M, H, return_state=True)
    assert 1 <= k <= o.NES_MAX_INNER
    got, k = o.nls_nes(np.zeros((3, 3)), M, H, return_state=True)
    assert k == 0
    np.testing.assert_array_equal(got, H)


def _model(dims, R, seed):
    rng = np.random.default_rng(seed)
    H = [rng.random((d, R)) for d in dims]
    Hn, lam = [], np.ones(R)
    for h in H:
        a, nu = o.normalize_columns(h)
        Hn.append(a)
        lam = lam * nu
    return Hn, lam


@pytest.mark.parametrize("dims", [(5, 6, 7), (3, 4, 2, 5)])
def test_extrapolated_model_is_projected_weighted_extrapolation(dims):
    R = 3
    H, lam = _model(dims, R, 13)
    Hp, lamp = _model(dims, R, 14)
    s = 1.7
    Hc, lamc = o.nes_extrapolate(H, lam, Hp, lamp, s)
    N = len(dims)
    F = [H[n] * (lam if n == N - 1 else 1.0) for n in range(N)]
    Fp = [Hp[n] * (lamp if n == N - 1 else 1.0) for n in range(N)]
    Fc = [np.maximum(0.0, f + s * (f - fp)) for f, fp in zip(F, Fp)]
    np.testing.assert_allclose(o.cp_full(Hc, lamc), o.cp_full(Fc), rtol=1e-12, atol=1e-14)
    for h in Hc:
        nz = np.linalg.norm(h, axis=0) > 0
        np.testing.assert_allclose(np.linalg.norm(h, axis=0)[nz], 1.0, rtol=1e-14)
    # s = 0 keeps the model
    H0, lam0 = o.nes_extrapolate(H, lam, Hp, lamp, 0.0)
    np.testing.assert_allclose(o.cp_full(H0, lam0), o.cp_full(H, lam), rtol=1e-12)


@pytest.mark.parametrize("dims", [(5, 6, 7), (3, 4, 2, 5)])
def test_model_error_matches_explicit_residual(dims):
    rng = np.random.default_rng(15)
    X = rng.random(dims)
    H, lam = _model(dims, 4, 16)
    got = o.model_error(X, H, lam, o.sqnorm(X))
    ref = o.fit_explicit(X, H, lam)[0]
    assert got == pytest.approx(ref, rel=1e-11)


def test_nncp_nes_acceleration_decision():
    """Two outer iterations: the second one's error is the candidate's when
    the candidate is better, else the plain iterate's."""
    from paper_1909_01149_gb300 import synth
    X, _ = synth.planted((8, 9, 10), 3, 17, noise=0.05)
    H0 = synth.init_factors(X.shape, 3, 18)
    plain = o.nncp(X, H0, "nes", iters=2, nes_accel=False)
    one = o.nncp(X, H0, "nes", iters=1)
    acc = o.nncp(X, H0, "nes", iters=2)
    assert acc["rel_err"][0] == one["rel_err"][0] == plain["rel_err"][0]
    s = 2 ** (1 / 3)
    Hc, lamc = o.nes_extrapolate(plain["H"], plain["lam"], one["H"], one["lam"], s)
    eps_c = o.model_error(X, Hc, lamc, o.sqnorm(X))
    assert acc["accepted"] == [eps_c < plain["rel_err"][1]]
    assert acc["rel_err"][1] == pytest.approx(min(eps_c, plain["rel_err"][1]), rel=1e-12)


def test_nncp_nes_recovers_planted_tensor():
    from paper_1909_01149_gb300 import synth
    X, _ = synth.planted((10, 11, 12), 3, 19, noise=0.0)
    H0 = synth.init_factors(X.shape, 3, 20)
    res = o.nncp(X, H0, "nes", iters=150)
    assert res["rel_err"][-1] < 1e-3
    assert any(res["accepted"])
