"""GPU: the all-mode MTTKRP through one dimension-tree pass (planc_mttkrp_all)
equals the per-mode MTTKRP (same kernels, same order: bit for bit) and the
FP64 oracle (FP32 1e-5 per entry relative, FP64 1e-12)."""

import numpy as np
import pytest
import torch

import oracle as o
from helpers import factors_to_device, max_rel, planc, x_to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,R,split", [((30, 24, 28), 8, -1), ((12, 9, 14, 11), 5, 2),
                                          ((12, 9, 14, 11), 5, 1), ((5, 7, 3, 6, 4), 3, 3),
                                          ((64, 48, 80), 16, -1), ((96, 96, 96, 96), 64, 2)])
@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_mttkrp_all_matches_per_mode_and_oracle(dims, R, split, dt):
    if dt == "f64" and np.prod(dims) > 2e6:
        pytest.skip("FP64 case kept small")
    p = planc()
    rng = np.random.default_rng(4)
    X = rng.random(dims)
    Xd, Xs = x_to_device(X, dt)
    Hd, Hs = factors_to_device([rng.random((d, R)) for d in dims], dt)
    with p.Context(Xd, dims, R, split) as ctx:
        M_all = [m.cpu().numpy() for m in ctx.mttkrp_all(Hd)]
        M_one = [ctx.mttkrp(Hd, n).cpu().numpy() for n in range(len(dims))]
    tol = 1e-12 if dt == "f64" else 1e-5
    for n in range(len(dims)):
        assert np.array_equal(M_all[n], M_one[n]), n
        if np.prod(dims) <= 2e6:
            assert max_rel(M_all[n], o.mttkrp(Xs, Hs, n)) <= tol, n
        else:
            rows = np.array([0, dims[n] // 2, dims[n] - 1])
            assert max_rel(M_all[n][rows], o.mttkrp_rows(Xs, Hs, n, rows)) <= tol, n
