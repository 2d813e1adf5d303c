"""Pins for the oracle's matricization, Khatri-Rao product, MTTKRP and Grams.

Each check is independent of the code it tests: brute-force element sums,
the closed form of a CP tensor's MTTKRP, the plain GEMM of the N=2 case, the
two-stage 3-way equations of Sec. 4.2.1, and S = K^T K with K built row by
row from its definition.
"""

import itertools

import numpy as np
import pytest

import oracle as o
from paper_1909_01149_gb300 import synth

SHAPES = [(2, 3), (3, 2, 4), (2, 3, 4, 2), (3, 2, 2, 3, 2)]


def _rand(shape, seed):
    return np.random.default_rng(seed).random(shape)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("R", [1, 3, 5])
def test_mttkrp_matches_bruteforce(shape, R):
    X = _rand(shape, 10 + R)
    H = [_rand((d, R), 100 + k) for k, d in enumerate(shape)]
    for n in range(len(shape)):
        np.testing.assert_allclose(o.mttkrp(X, H, n),
                                   o.mttkrp_bruteforce(X, H, n),
                                   rtol=1e-13, atol=0)


@pytest.mark.parametrize("shape", SHAPES)
def test_unfold_index_formula(shape):
    """X_(n)[i_n, j] with j = sum_{k != n} i_k prod_{m<k, m != n} I_m."""
    X = _rand(shape, 3)
    N = len(shape)
    for n in range(N):
        U = o.unfold(X, n)
        assert U.shape == (shape[n], X.size // shape[n])
        for idx in itertools.product(*[range(s) for s in shape]):
            j, stride = 0, 1
            for k in range(N):
                if k == n:
                    continue
                j += idx[k] * stride
                stride *= shape[k]
            assert U[idx[n], j] == X[idx]


def test_khatri_rao_last_factor_fastest():
    A = _rand((3, 2), 1)
    B = _rand((4, 2), 2)
    K = o.khatri_rao([A, B])
    for i in range(3):
        for j in range(4):
            np.testing.assert_array_equal(K[i * 4 + j], A[i] * B[j])


@pytest.mark.parametrize("shape", [(4, 5, 6), (3, 4, 2, 5), (2, 3, 2, 2, 3)])
def test_mttkrp_cp_closed_form(shape):
    """For X = [[A_1..A_N]]: M^(n) = A_n (*_{k != n} A_k^T H_k)."""
    R, Rx = 3, 4
    A = [_rand((d, Rx), 20 + k) for k, d in enumerate(shape)]
    H = [_rand((d, R), 40 + k) for k, d in enumerate(shape)]
    X = synth._cp_dense(A)
    for n in range(len(shape)):
        W = np.ones((Rx, R))
        for k in range(len(shape)):
            if k != n:
                W *= A[k].T @ H[k]
        np.testing.assert_allclose(o.mttkrp(X, H, n), A[n] @ W, rtol=1e-12)


def test_mttkrp_two_way_is_gemm():
    X = _rand((7, 5), 5)
    H = [_rand((7, 3), 6), _rand((5, 3), 7)]
    np.testing.assert_allclose(o.mttkrp(X, H, 0), X @ H[1], rtol=1e-14)
    np.testing.assert_allclose(o.mttkrp(X, H, 1), X.T @ H[0], rtol=1e-14)


def test_three_way_partial_mttkrp_equations():
    """Sec. 4.2.1: T_ijr = sum_k X_ijk W_kr;  M1_ir = sum_j V_jr T_ijr;
    M2_jr = sum_i U_ir T_ijr."""
    I, J, K, R = 4, 3, 5, 2
    X = _rand((I, J, K), 8)
    U, V, W = _rand((I, R), 9), _rand((J, R), 10), _rand((K, R), 11)
    T = np.zeros((I, J, R))
    for i in range(I):
        for j in range(J):
            for r in range(R):
                T[i, j, r] = sum(X[i, j, k] * W[k, r] for k in range(K))
    M1 = np.array([[sum(V[j, r] * T[i, j, r] for j in range(J))
                    for r in range(R)] for i in range(I)])
    M2 = np.array([[sum(U[i, r] * T[i, j, r] for i in range(I))
                    for r in range(R)] for j in range(J)])
    np.testing.assert_allclose(o.mttkrp(X, [U, V, W], 0), M1, rtol=1e-13)
    np.testing.assert_allclose(o.mttkrp(X, [U, V, W], 1), M2, rtol=1e-13)


@pytest.mark.parametrize("shape", [(3, 4, 2), (2, 3, 2, 3)])
def test_gram_hadamard_is_krp_gram(shape):
    """S^(n) = K^T K, K = krp of the other factors built row by row."""
    R = 3
    H = [_rand((d, R), 60 + k) for k, d in enumerate(shape)]
    G = [o.gram(h) for h in H]
    N = len(shape)
    for n in range(N):
        rows = []
        others = [k for k in range(N) if k != n]
        for idx in itertools.product(*[range(shape[k]) for k in others]):
            row = np.ones(R)
            for k, i in zip(others, idx):
                row = row * H[k][i]
            rows.append(row)
        K = np.array(rows)
        np.testing.assert_allclose(o.gram_hadamard(G, n), K.T @ K, rtol=1e-13)


def test_sqnorm_and_cp_full():
    X = _rand((3, 4, 5), 12)
    assert abs(o.sqnorm(X) - float(np.sum(X ** 2))) < 1e-12
    A = [_rand((d, 2), 70 + k) for k, d in enumerate((3, 4, 5))]
    lam = np.array([2.0, 0.5])
    F = o.cp_full(A, lam)
    for i, j, k in itertools.product(range(3), range(4), range(5)):
        ref = sum(lam[r] * A[0][i, r] * A[1][j, r] * A[2][k, r]
                  for r in range(2))
        assert abs(F[i, j, k] - ref) < 1e-14


@pytest.mark.parametrize("dims,S", [((512, 512, 512), 2), ((64, 64, 64), 2),
                                    ((128, 128, 200, 100), 2),
                                    ((96, 96, 96, 96), 2), ((10, 1000), 1),
                                    ((1000, 10), 1), ((2, 3, 4, 5, 6), 3)])
def test_choose_split(dims, S):
    """Root split: products of the two contiguous mode groups nearly equal,
    ties to the larger S (agrees with the literal rule on 3-way cubes)."""
    assert o.choose_split(dims) == S


def _rows_bruteforce(X, H, n, rows):
    """Element sums of Sec. 4.2.1 restricted to the listed rows of mode n,
    with Python loops (independent of the matricization path)."""
    R = H[0].shape[1]
    out = np.zeros((len(rows), R))
    for q, i in enumerate(rows):
        for idx in itertools.product(*[range(s) for s in X.shape]):
            if idx[n] != i:
                continue
            for r in range(R):
                p = X[idx]
                for k in range(X.ndim):
                    if k != n:
                        p *= H[k][idx[k], r]
                out[q, r] += p
    return out


@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 4, 2, 3), (2, 3, 2, 3, 2)])
def test_mttkrp_rows_is_the_row_restricted_definition(shape):
    """mttkrp_rows (the sampled checker of the full-size GPU tests) returns
    exactly the requested rows of M^(n), in the requested order: unsorted,
    duplicate-free row lists in every mode, checked against element sums."""
    R = 3
    X = _rand(shape, 50 + len(shape))
    H = [_rand((d, R), 60 + k) for k, d in enumerate(shape)]
    rng = np.random.default_rng(len(shape))
    for n, d in enumerate(shape):
        rows = rng.permutation(d)[: max(1, d - 1)]
        if len(rows) > 1 and np.all(np.diff(rows) > 0):
            rows = rows[::-1].copy()  # keep the list unsorted
        got = o.mttkrp_rows(X, H, n, rows)
        np.testing.assert_allclose(got, _rows_bruteforce(X, H, n, rows), rtol=1e-13, atol=0)
        np.testing.assert_allclose(got, o.mttkrp(X, H, n)[rows], rtol=1e-13, atol=0)


def test_mttkrp_rows_single_row_and_float32_input():
    """One row of a float32 tensor is summed in float64 (the full-size tests
    pass the stored float32 tensor)."""
    shape, R = (5, 4, 3), 2
    X = _rand(shape, 71).astype(np.float32)
    H = [_rand((d, R), 80 + k) for k, d in enumerate(shape)]
    Xd = X.astype(np.float64)
    for n, d in enumerate(shape):
        got = o.mttkrp_rows(X, H, n, [d - 1])
        assert got.dtype == np.float64 and got.shape == (1, R)
        np.testing.assert_allclose(got, _rows_bruteforce(Xd, H, n, [d - 1]), rtol=1e-13)
