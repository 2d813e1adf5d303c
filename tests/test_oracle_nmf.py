"""Pins for the N = 2 case of the oracle's outer loop, which is NMF
(X ~ W H^T): with BPP, every half-step is an exact non-negative least
squares solve, so the model after each outer iteration must equal the one
of a textbook alternating NNLS (ANLS) written with SciPy's Lawson-Hanson
NNLS; a noiseless non-negative low-rank matrix is recovered; the error
identity equals the explicit residual.
"""

import numpy as np
import pytest

import oracle as o
from paper_1909_01149_gb300 import synth


def _anls(X, H, iters):
    """Textbook ANLS for X ~ W H^T with SciPy NNLS, one row at a time."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    for _ in range(iters):
        W = np.stack([scipy_opt.nnls(H, X[i], maxiter=2000)[0] for i in range(X.shape[0])])
        H = np.stack([scipy_opt.nnls(W, X[:, j], maxiter=2000)[0] for j in range(X.shape[1])])
    return W, H


@pytest.mark.parametrize("shape,R", [((30, 20), 4), ((12, 41), 6)])
def test_nmf_bpp_is_textbook_anls(shape, R):
    X, _ = synth.planted(shape, R, 11, noise=0.1)
    H0 = synth.init_factors(shape, R, 12)
    for iters in (1, 3):
        res = o.nncp(X, H0, "bpp", iters=iters)
        W, H = _anls(X, H0[1], iters)
        np.testing.assert_allclose(o.cp_full(res["H"], res["lam"]), W @ H.T, rtol=0, atol=1e-9)


@pytest.mark.parametrize("alg", ["hals", "bpp"])
def test_nmf_noiseless_recovery(alg):
    X, _ = synth.planted((25, 30), 3, 13, noise=0.0)
    res = o.nncp(X, synth.init_factors((25, 30), 3, 14), alg, iters=2000)
    assert o.fit_explicit(X, res["H"], res["lam"])[0] < 1e-6


def test_nmf_error_identity_is_explicit_residual():
    X, _ = synth.planted((17, 23), 5, 15, noise=0.2)
    res = o.nncp(X, synth.init_factors((17, 23), 5, 16), "hals", iters=4)
    W = res["H"][0] * res["lam"]
    ref = np.linalg.norm(X - W @ res["H"][1].T) / np.linalg.norm(X)
    assert res["rel_err"][-1] == pytest.approx(ref, rel=1e-10)
