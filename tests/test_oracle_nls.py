"""Pins for the oracle's NNLS updates (Sec. 4.3).

BPP is checked against SciPy's Lawson-Hanson NNLS on an explicit A, b with
A^T A = S and A^T b = m, against brute-force enumeration of every passive
set, and against the KKT conditions.  HALS, MU, ADMM and PGD are checked by
the properties the paper states or that fix them: monotone objective, the
exact 1-D minimiser of each HALS column step, and convergence to the unique
BPP solution when S is positive definite.
"""

import itertools

import numpy as np
import pytest

import oracle as o


def _problem(rows, R, seed, m_rows=None):
    """Random NNLS instance in Gram form: A (m x R), B (m x rows)."""
    rng = np.random.default_rng(seed)
    m_rows = m_rows or 3 * R
    A = rng.random((m_rows, R))
    B = rng.random((m_rows, rows)) - 0.3  # some rows have active constraints
    S = A.T @ A
    M = (A.T @ B).T  # rows x R
    return A, B, S, M


def _kkt(S, m, x):
    y = S @ x - m
    return x.min(), y.min(), np.abs(x * y).max()


@pytest.mark.parametrize("R", [1, 3, 6, 12])
def test_bpp_matches_lawson_hanson(R):
    scipy_opt = pytest.importorskip("scipy.optimize")
    A, B, S, M = _problem(8, R, R)
    X, _, ok = o.nls_bpp(S, M)
    assert ok
    for i in range(M.shape[0]):
        ref, _ = scipy_opt.nnls(A, B[:, i])
        np.testing.assert_allclose(X[i], ref, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("R", [2, 4, 6])
def test_bpp_matches_passive_set_enumeration(R):
    _, _, S, M = _problem(5, R, 40 + R)
    X, _, _ = o.nls_bpp(S, M)
    for i in range(M.shape[0]):
        m = M[i]
        found = []
        for mask in itertools.product([False, True], repeat=R):
            F = np.array(mask)
            x = np.zeros(R)
            if F.any():
                x[F] = np.linalg.solve(S[np.ix_(F, F)], m[F])
            y = S @ x - m
            if x.min() >= -1e-12 and y[~F].min(initial=0) >= -1e-12:
                found.append(np.maximum(x, 0))
        assert found, "no KKT point found by enumeration"
        for f in found:
            np.testing.assert_allclose(X[i], f, rtol=1e-9, atol=1e-12)


def test_bpp_kkt_and_warm_start_independence():
    _, _, S, M = _problem(20, 10, 7)
    X0, _, _ = o.nls_bpp(S, M)
    rng = np.random.default_rng(1)
    X1, _, _ = o.nls_bpp(S, M, rng.random(M.shape) - 0.5)
    np.testing.assert_allclose(X0, X1, rtol=1e-10, atol=1e-13)
    for i in range(M.shape[0]):
        xmin, ymin, comp = _kkt(S, M[i], X0[i])
        assert xmin >= 0 and ymin > -1e-10 and comp < 1e-10


def test_bpp_row_zero_rhs():
    S = np.eye(3) * 2
    x, it, ok = o.nls_bpp_row(S, np.zeros(3))
    assert ok and it == 0 and not x.any()


@pytest.mark.parametrize("alg", ["mu", "hals", "admm", "pgd"])
def test_objective_non_increasing(alg):
    _, _, S, M = _problem(30, 8, 11)
    M = np.abs(M)  # MU needs a non-negative numerator
    H = np.random.default_rng(3).random(M.shape)
    f0 = o.nls_objective(S, M, H)
    fn = {"mu": o.nls_mu, "hals": o.nls_hals, "pgd": o.nls_pgd,
          "admm": lambda S, M, H: o.nls_admm(S, M, H)}[alg]
    for _ in range(20):
        H = fn(S, M, H)
        f1 = o.nls_objective(S, M, H)
        if alg != "admm":  # ADMM is not a descent method step by step
            assert f1 <= f0 + 1e-12 * abs(f0)
        f0 = f1
    assert (H >= 0).all()


def test_hals_column_step_is_exact_minimiser():
    _, _, S, M = _problem(6, 5, 13)
    H = np.random.default_rng(4).random(M.shape)
    R = S.shape[0]
    # one column step in isolation: only column 0 changes
    H1 = H.copy()
    H1[:, 0] = np.maximum(0, H[:, 0] + (M[:, 0] - H @ S[:, 0]) / S[0, 0])
    Hs = o.nls_hals(S, M, H)
    np.testing.assert_allclose(Hs[:, 0], H1[:, 0], rtol=1e-14)
    f1 = o.nls_objective(S, M, H1)
    for delta in (1e-3, -1e-3, 0.1, -0.1):
        Hp = H1.copy()
        Hp[:, 0] = np.maximum(0, Hp[:, 0] + delta)
        assert o.nls_objective(S, M, Hp) >= f1 - 1e-14
    assert R == 5


@pytest.mark.parametrize("alg", ["hals", "admm", "pgd"])
def test_iterations_reach_bpp_solution(alg):
    _, _, S, M = _problem(10, 6, 17)
    X, _, _ = o.nls_bpp(S, M)
    H = np.random.default_rng(5).random(M.shape)
    if alg == "hals":
        for _ in range(3000):
            H = o.nls_hals(S, M, H)
    elif alg == "pgd":
        H = o.nls_pgd(S, M, H, steps=40000)
    else:
        H = o.nls_admm(S, M, H, max_inner=3000, tol=0.0)
    np.testing.assert_allclose(H, X, rtol=1e-6, atol=1e-8)


def test_mu_fixed_point_and_eps():
    S = np.array([[2.0, 0.5], [0.5, 1.0]])
    x = np.array([[0.3, 0.7]])
    M = x @ S  # unconstrained optimum is x itself, strictly positive
    np.testing.assert_allclose(o.nls_mu(S, M, x), x, rtol=1e-14)
    # zero denominator is protected by eps and keeps zero entries at zero
    z = o.nls_mu(S, M, np.zeros((1, 2)))
    assert np.all(z == 0)


def test_hals_skips_zero_diagonal():
    S = np.array([[0.0, 0.0], [0.0, 1.0]])
    M = np.array([[5.0, 2.0]])
    H = np.array([[0.7, 0.1]])
    out = o.nls_hals(S, M, H)
    assert out[0, 0] == 0.7 and out[0, 1] == 2.0


def test_admm_first_step_by_hand():
    """One ADMM step from H = 0, U = 0 is the projected ridge solution with
    rho = trace(S) / R."""
    S = np.array([[4.0, 1.0], [1.0, 2.0]])
    M = np.array([[1.0, -3.0]])
    rho = 3.0
    Htil = M @ np.linalg.inv(S + rho * np.eye(2))
    H, U, k = o.nls_admm(S, M, np.zeros((1, 2)), max_inner=1,
                         return_state=True)
    np.testing.assert_allclose(H, np.maximum(Htil, 0), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(U, H - Htil, rtol=1e-14, atol=1e-15)
    assert k == 1


def test_normalize_columns():
    rng = np.random.default_rng(9)
    Hh = rng.random((7, 4))
    Hh[:, 2] = 0.0
    H, lam = o.normalize_columns(Hh)
    np.testing.assert_allclose(np.linalg.norm(H[:, [0, 1, 3]], axis=0), 1.0)
    assert lam[2] == 0 and not H[:, 2].any()
    np.testing.assert_allclose(H * lam, Hh, rtol=1e-15)


def test_ucp_is_the_unfolded_least_squares_solution():
    """The UCP update solves min ||X_(n) - H K^T|| (least squares on the
    explicit unfolding and Khatri-Rao product, not the normal equations)."""
    rng = np.random.default_rng(21)
    dims, R = (7, 6, 8), 4
    X = rng.random(dims)
    H = [rng.random((d, R)) for d in dims]
    for n in range(3):
        K = o.krp_except(H, n)
        ref, *_ = np.linalg.lstsq(K, o.unfold(X, n).T, rcond=None)
        S = o.gram_hadamard([o.gram(h) for h in H], n)
        np.testing.assert_allclose(o.nls_ucp(S, o.mttkrp(X, H, n)), ref.T, rtol=1e-9, atol=1e-12)


def test_ucp_als_objective_non_increasing_and_exact_recovery():
    """CP-ALS: each block update is the exact block minimiser, so the loss
    never increases; on a noiseless rank-R tensor it converges to zero."""
    rng = np.random.default_rng(22)
    dims, R = (9, 8, 7), 3
    # zero-mean factors (well-conditioned S; UCP has no sign constraint)
    A = [rng.standard_normal((d, R)) for d in dims]
    X = o.cp_full(A)
    H0 = [a + 0.2 * rng.standard_normal(a.shape) for a in A]
    res = o.nncp(X, H0, "ucp", iters=60, record_objective=True)
    obj = res["objective"]
    assert all(b <= a * (1 + 1e-10) + 1e-14 for a, b in zip(obj, obj[1:]))
    assert res["rel_err"][-1] < 1e-6


# ADMM stop rule (reading of Sec. 4.3.4; the paper defers it to its
# reference).  Hand-worked family: S = I (R = 2), so rho = trace(S)/R = 1 and
# the two columns decouple; one row M = [b, -a] with a, b > 0, H = U = 0.
# Each step is Htil = (M + H + U)/2, H = [Htil - U]_+, U = U + H - Htil.
#   column 1 (b > 0): U stays 0, H_k = Htil_k = b (1 - 2^-k);
#   column 2 (-a < 0): H stays 0, Htil_k = -a 2^-k, U_k = a (1 - 2^-k).
# After step k:
#   ||H - Htil||^2 = a^2 4^-k,      ||H||^2 = b^2 (1 - 2^-k)^2,
#   ||H - H_prev||^2 = b^2 4^-k,    ||U||^2 = a^2 (1 - 2^-k)^2.
# With rho = a / b and tol = t^2 the primal test holds iff
# 2^-k < t / (rho + t) and the dual test iff 2^-k < t / (1/rho + t).
# tol = 1e-2 (t = 0.1):
#   a = 4, b = 1: primal from k = 6 (2^-6 < 0.1/4.1 = 0.0244 < 2^-5), dual
#                 from k = 2 (2^-2 < 0.1/0.35 = 0.286 < 2^-1): stop at 6;
#   a = 1, b = 4: the mirror image: stop at 6;
#   a = b:        both from k = 4 (2^-4 < 0.1/1.1 = 0.0909 < 2^-3): stop at 4.
# tol = 4e-2 (t = 0.2), a = 4, b = 1: primal from k = 5 (0.2/4.2 = 0.0476),
#   dual from k = 2: stop at 5.
# A rule with "or" would stop at 2, 2, 4, 2; one that swaps the two
# denominators (||U|| for the primal, ||H|| for the dual) at 4, 4, 4, 4.
@pytest.mark.parametrize("a,b,tol,stop", [(4.0, 1.0, 1e-2, 6), (1.0, 4.0, 1e-2, 6),
                                          (2.0, 2.0, 1e-2, 4), (4.0, 1.0, 4e-2, 5)])
def test_admm_stop_rule_by_hand(a, b, tol, stop):
    S = np.eye(2)
    M = np.array([[b, -a]])
    H, U, k = o.nls_admm(S, M, np.zeros((1, 2)), max_inner=20, tol=tol,
                         return_state=True)
    assert k == stop
    np.testing.assert_allclose(H, [[b * (1 - 2.0 ** -stop), 0.0]], rtol=1e-14, atol=0)
    np.testing.assert_allclose(U, [[0.0, a * (1 - 2.0 ** -stop)]], rtol=1e-14, atol=1e-15)
    # the default cap of 5 steps ends the 6-step cases early
    _, _, k5 = o.nls_admm(S, M, np.zeros((1, 2)), tol=tol, return_state=True)
    assert k5 == min(stop, 5)


def test_admm_zero_gram_uses_rho_one():
    """S = 0 (every other factor has a zero column): trace(S) = 0, the reading
    takes rho = 1, so one step from H = [0.5, 0.5], U = 0 with M = [1, -1] is
    Htil = M + H = [1.5, -0.5], H = [1.5, 0], U = [0, 0.5] (rho = 2 would give
    Htil = [1, 0])."""
    S = np.zeros((2, 2))
    M = np.array([[1.0, -1.0]])
    H, U, k = o.nls_admm(S, M, np.array([[0.5, 0.5]]), max_inner=1, return_state=True)
    assert k == 1
    np.testing.assert_array_equal(H, [[1.5, 0.0]])
    np.testing.assert_array_equal(U, [[0.0, 0.5]])


def test_fit_identity_zero_tensor():
    """alpha = 0 (an all-zero tensor) reports eps = 0 and fit = 1 (reading)."""
    z = np.zeros((3, 2))
    eps, fit = o.fit_identity(0.0, z, z, np.ones((2, 2)), np.eye(2), np.zeros(2))
    assert eps == 0.0 and fit == 1.0
