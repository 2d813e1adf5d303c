"""The seeded input recipes (paper_1909_01149_gb300/synth.py) against their
stated definitions: the planted CP tensor and its noise bounds, the
mode-1-fastest layout, the slab-wise dense construction (ragged last slab
included), the mouse-like stand-in's factor shapes and signal-to-noise
ratio, and the batch's size ranges and per-instance seeds."""

import numpy as np
import pytest

from paper_1909_01149_gb300 import synth


def _cp(A):
    letters = "abcdefgh"[:len(A)]
    return np.einsum(",".join(l + "r" for l in letters) + "->" + letters, *A)


def test_planted_noiseless_is_the_cp_model_of_its_factors():
    X, A = synth.planted((5, 6, 7, 3), 4, data_seed=3)
    assert [a.shape for a in A] == [(5, 4), (6, 4), (7, 4), (3, 4)]
    np.testing.assert_allclose(X, _cp(A), rtol=1e-14, atol=0)
    assert all((a >= 0).all() and (a < 1).all() for a in A)


def test_planted_noise_is_nonnegative_uniform_scaled_by_the_mean():
    noise = 0.05
    X, A = synth.planted((40, 30, 20), 3, data_seed=4, noise=noise)
    M = _cp(A)
    d = (X - M) / (noise * M.mean())
    assert d.min() >= 0.0 and d.max() < 1.0 + 1e-12
    assert abs(d.mean() - 0.5) < 0.01  # U[0,1): mean 1/2 over 24000 draws


def test_flat_is_mode_one_fastest():
    X, _ = synth.planted((3, 4, 5), 2, data_seed=5)
    f = synth.flat(X)
    assert f.flags["C_CONTIGUOUS"] and f.shape == (60,)
    for i, j, k in [(0, 0, 0), (2, 0, 0), (0, 3, 0), (1, 2, 4), (2, 3, 4)]:
        assert f[i + 3 * (j + 4 * k)] == X[i, j, k]


@pytest.mark.parametrize("chunk", [1, 7, 30, 1 << 25])
def test_slabwise_construction_matches_one_slab(chunk):
    rng = np.random.default_rng(6)
    A = [rng.random((d, 3)) for d in (4, 5, 11)]  # lead = 20 rows, 11 slabs of the last mode
    got = synth._cp_dense(A, chunk_elems=chunk)
    np.testing.assert_allclose(got, _cp(A), rtol=1e-14, atol=0)


def test_mouse_like_factors_and_signal_to_noise():
    dims, R = (32, 32, 40, 20), 5
    X, A = synth.mouse_like(dims, R, data_seed=7, dtype=np.float64)
    A1, A2, A3, A4 = A
    assert [a.shape for a in A] == [(d, R) for d in dims]
    # Gaussian blobs peak at most 1; traces are 0 before onset, 1 at onset, decaying
    assert A1.max() <= 1.0 and A2.max() <= 1.0 and A1.min() > 0.0
    for r in range(R):
        t0 = int(np.argmax(A3[:, r] > 0))
        assert (A3[:t0, r] == 0).all() and A3[t0, r] == 1.0
        assert (np.diff(A3[t0:, r]) <= 0).all()
    assert (A4 >= 0.5).all() and (A4 < 1.5).all()
    M = _cp(A)
    assert (X >= 0).all()
    snr = float((M * M).sum() / ((X - M) ** 2).sum())
    assert abs(10 * np.log10(snr) - 10.0) < 0.1


def test_batch_ranges_and_instance_seeds():
    inst = synth.batch(count=6, data_seed=2, noise=0.02, lo=8, hi=12, rlo=2, rhi=4,
                       dtype=np.float64)
    assert len(inst) == 6
    for i, (X, A, R) in enumerate(inst):
        assert all(8 <= d <= 12 for d in X.shape) and 2 <= R <= 4
        assert [a.shape for a in A] == [(d, R) for d in X.shape]
        Xi, _ = synth.planted(X.shape, R, 2 * 1000 + i, 0.02, np.float64)
        np.testing.assert_array_equal(X, Xi)


def test_init_factors_drawn_in_mode_order():
    H = synth.init_factors((3, 5, 2), 4, init_seed=9)
    rng = np.random.default_rng(9)
    for h, d in zip(H, (3, 5, 2)):
        np.testing.assert_array_equal(h, rng.random((d, 4)))
