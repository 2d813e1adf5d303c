"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module only draws numbers and assembles planted CP tensors; it holds
none of the NNCP method's arithmetic (no MTTKRP, NNLS, normalisation or fit),
so the CUDA library and the FP64 oracle can both be fed from it.

All tensors are returned as NumPy arrays of shape (I_1, ..., I_N) whose
Fortran-order ravel is the "mode-1 fastest" buffer of the paper's layout
(Sec. 4.1.2).  ``flat(X)`` gives that buffer.

Recipes (one per workload):
  planted(dims, R, noise)   U[0,1) factors, X = [[A]] + noise * mean * U[0,1)
                            (the paper's exact-low-rank synthetic data,
                            Sec. 6.1.2, with optional non-negative noise)
  mouse_like(...)           pixel x pixel x time x trial stand-in for the
                            calcium-imaging data of Sec. 6.1.1: Gaussian blob
                            spatial maps, exponential-decay traces, U[0.5,1.5)
                            trial gains, Poisson-like noise at 10 dB SNR
  batch(count)              many small uneven 3-way planted problems
  init_factors(dims, R)     U[0,1) initial factors, drawn in mode order
  perturbed_factors(A)      planted factors times 1 + 10% U[-1,1) (start
                            near the solution)
  decaying(dims, R)         planted tensor whose mode-1 factor columns decay
                            exponentially (fibres spanning orders of magnitude)
"""

from __future__ import annotations

import numpy as np


def flat(X: np.ndarray) -> np.ndarray:
    """Mode-1-fastest flat buffer of X (a contiguous 1-D array)."""
    return np.ascontiguousarray(np.ravel(X, order="F"))


def _cp_dense(A, dtype=np.float64, chunk_elems=1 << 25):
    """Dense sum_r a1_r o a2_r o ... o aN_r, built slab by slab along the last
    mode so that large tensors need little temporary memory."""
    dims = tuple(a.shape[0] for a in A)
    R = A[0].shape[1]
    N = len(dims)
    out = np.empty(dims, dtype=dtype, order="F")
    # Rows of the first N-1 modes combined; row index = i_1 + I_1 (i_2 + ...).
    W = np.ones((1, R))
    for a in A[:-1]:
        W = (W[None, :, :] * a[:, None, :]).reshape(-1, R)
    lead = W.shape[0]
    last = A[-1]
    step = max(1, chunk_elems // max(lead, 1))
    flat_out = out.reshape(-1, order="F")
    for k0 in range(0, dims[-1], step):
        k1 = min(dims[-1], k0 + step)
        blk = W @ last[k0:k1].T  # lead x (k1-k0), column-major = mode-1 fastest
        flat_out[k0 * lead:k1 * lead] = blk.ravel(order="F").astype(dtype)
    return out


def init_factors(dims, R, init_seed=2, dtype=np.float64):
    """U[0,1) initial factors H^(1..N), drawn in mode order from init_seed."""
    rng = np.random.default_rng(init_seed)
    return [rng.random((d, R)).astype(dtype) for d in dims]


def planted(dims, R, data_seed=1, noise=0.0, dtype=np.float64):
    """Planted non-negative CP tensor: A_n ~ U[0,1) (I_n x R), drawn in mode
    order; X = [[A]] + noise * mean([[A]]) * U[0,1) element-wise.

    Returns (X, A) with X of the requested dtype."""
    rng = np.random.default_rng(data_seed)
    A = [rng.random((d, R)) for d in dims]
    M = _cp_dense(A, dtype=np.float64)
    if noise > 0:
        level = noise * float(M.mean())
        flat_m = M.reshape(-1, order="F")
        n = flat_m.size
        step = 1 << 24
        for i0 in range(0, n, step):
            i1 = min(n, i0 + step)
            flat_m[i0:i1] += level * rng.random(i1 - i0)
    return M.astype(dtype, order="F"), A


def mouse_like(dims=(128, 128, 200, 100), R=16, data_seed=1,
               snr_db=10.0, dtype=np.float32):
    """Stand-in for the calcium-imaging tensor (pixel-x, pixel-y, time,
    trial): spatial maps are separable Gaussian blobs with centres uniform over
    each axis and sigma ~ U[3, 8] px; temporal traces exp(-(t - t0)/tau) for
    t >= t0 (0 before), t0 ~ U{0..T-1}, tau ~ U[10, 50]; trial gains
    U[0.5, 1.5).  Noise is Poisson-like, X = c * Poisson(M / c) with
    c = ||M||^2 / (10^(snr/10) * sum(M)), so E||X - M||^2 = ||M||^2 / 10^(snr/10).

    Returns (X, A)."""
    rng = np.random.default_rng(data_seed)
    I1, I2, T, K = dims
    A1 = np.empty((I1, R))
    A2 = np.empty((I2, R))
    x1 = np.arange(I1)[:, None]
    x2 = np.arange(I2)[:, None]
    c1 = rng.uniform(0, I1, R)
    c2 = rng.uniform(0, I2, R)
    s1 = rng.uniform(3, 8, R)
    s2 = rng.uniform(3, 8, R)
    A1[:] = np.exp(-((x1 - c1) ** 2) / (2 * s1 ** 2))
    A2[:] = np.exp(-((x2 - c2) ** 2) / (2 * s2 ** 2))
    t = np.arange(T)[:, None]
    t0 = rng.integers(0, T, R)
    tau = rng.uniform(10, 50, R)
    A3 = np.where(t >= t0, np.exp(-(t - t0) / tau), 0.0)
    A4 = rng.uniform(0.5, 1.5, (K, R))
    A = [A1, A2, A3, A4]
    M = _cp_dense(A, dtype=np.float64)
    flat_m = M.reshape(-1, order="F")
    c = float(flat_m @ flat_m) / (10 ** (snr_db / 10.0) * float(flat_m.sum()))
    n = flat_m.size
    step = 1 << 24
    for i0 in range(0, n, step):
        i1 = min(n, i0 + step)
        flat_m[i0:i1] = c * rng.poisson(flat_m[i0:i1] / c)
    return M.astype(dtype, order="F"), A


def batch(count=256, data_seed=1, noise=0.02, lo=32, hi=160, rlo=8, rhi=32,
          dtype=np.float32):
    """Many uneven 3-way planted problems: each I_n ~ U{lo..hi}, R ~
    U{rlo..rhi}; instance i is planted(..., data_seed * 1000 + i)."""
    rng = np.random.default_rng(data_seed)
    out = []
    for i in range(count):
        dims = tuple(int(v) for v in rng.integers(lo, hi + 1, 3))
        R = int(rng.integers(rlo, rhi + 1))
        X, A = planted(dims, R, data_seed * 1000 + i, noise, dtype)
        out.append((X, A, R))
    return out


def perturbed_factors(A, level=0.1, seed=3, dtype=np.float64):
    """Start factors near planted ones: A_n * (1 + level * U[-1, 1)) entry
    by entry, drawn in mode order from `seed` (a start close to the
    solution, for runs that should reach the noise floor)."""
    rng = np.random.default_rng(seed)
    return [(a * (1.0 + level * (2.0 * rng.random(a.shape) - 1.0))).astype(dtype) for a in A]


def decaying(dims, R, data_seed=1, noise=0.01, tau=(5.0, 40.0), dtype=np.float32):
    """Planted tensor whose mode-1 factor columns decay, A_1[i, r] =
    exp(-i / tau_r) with tau_r ~ U[tau): along mode 1 every fibre falls by
    orders of magnitude (rows whose scale drifts inside a reduction); the
    other factors U[0, 1); noise as in planted().  Returns (X, A)."""
    rng = np.random.default_rng(data_seed)
    taus = rng.uniform(tau[0], tau[1], R)
    A = [np.exp(-np.arange(dims[0])[:, None] / taus[None, :])]
    A += [rng.random((d, R)) for d in dims[1:]]
    M = _cp_dense(A, dtype=np.float64)
    if noise > 0:
        level = noise * float(M.mean())
        flat_m = M.reshape(-1, order="F")
        flat_m += level * rng.random(flat_m.size)
    return M.astype(dtype, order="F"), A


# ----------------------------------------------------------------------------
# 16-bit storage: FP32 -> BF16 / FP16 by round-to-nearest-even, once.
# ----------------------------------------------------------------------------


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """uint16 BF16 bit patterns of float32 x, round-to-nearest-even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    rounding = ((u >> 16) & 1) + np.uint32(0x7FFF)
    return ((u + rounding) >> 16).astype(np.uint16)


def from_bf16_bits(b: np.ndarray) -> np.ndarray:
    """float32 values of uint16 BF16 bit patterns (exact)."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def to_f16(x: np.ndarray) -> np.ndarray:
    """float16 of x by round-to-nearest-even (NumPy's cast)."""
    return np.asarray(x, dtype=np.float32).astype(np.float16)
