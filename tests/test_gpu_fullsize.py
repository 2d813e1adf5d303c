"""Parity at the benchmark's full size (512^3 FP32, R = 32, the split the
benchmark uses) on sampled outputs the oracle computes row by row, plus
properties that hold at any size.

Tolerance: per-entry relative <= 1e-5 for the FP32 MTTKRP rows (all entries
positive); the solve's error identity is compared with the explicit
residual computed on the device in FP64 chunks.
"""

import numpy as np
import pytest
import torch

import oracle as o
from paper_1909_01149_gb300 import synth
from helpers import max_rel, planc

pytestmark = pytest.mark.gpu

DIMS, R = (512, 512, 512), 32


@pytest.fixture(scope="module")
def full():
    X, _ = synth.planted(DIMS, R, 1, noise=0.05, dtype=np.float32)
    Xd = torch.from_numpy(synth.flat(X)).cuda()
    H0 = synth.init_factors(DIMS, R, 2, dtype=np.float32)
    yield X, Xd, H0
    del Xd
    torch.cuda.empty_cache()


def test_full_size_mttkrp_sampled_rows(full):
    X, Xd, H0 = full
    p = planc()
    Hd = [torch.from_numpy(h).cuda() for h in H0]
    Hs = [h.astype(np.float64) for h in H0]
    rng = np.random.default_rng(0)
    with p.Context(Xd, DIMS, R) as ctx:
        assert ctx.split == 2
        for n in range(3):
            M = ctx.mttkrp(Hd, n).double().cpu().numpy()
            rows = np.sort(rng.choice(DIMS[n], 6, replace=False))
            rows = np.unique(np.concatenate([rows, [0, DIMS[n] - 1]]))
            ref = o.mttkrp_rows(X, Hs, n, rows)
            assert max_rel(M[rows], ref) <= 1e-5, (n, max_rel(M[rows], ref))
            assert np.isfinite(M).all() and (M > 0).all()


def test_full_size_solve_error_identity(full):
    """After a few HALS iterations the identity-based error equals the
    explicit residual ||X - [[lambda; H]]|| / ||X|| (computed on the device in
    FP64 slabs, independent of the library)."""
    X, Xd, H0 = full
    p = planc()
    Hd = [torch.from_numpy(h).cuda() for h in H0]
    with p.Context(Xd, DIMS, R) as ctx:
        res = ctx.solve(Hd, alg="hals", iters=3)
    lam = torch.tensor(res["lam"], dtype=torch.float64, device="cuda")
    H = [h.double() for h in Hd]
    num = 0.0
    den = 0.0
    Xv = Xd.view(DIMS[2], DIMS[1], DIMS[0])  # [k][j][i]: mode 1 fastest
    for k0 in range(0, DIMS[2], 64):
        k1 = k0 + 64
        # model slab: sum_r lam_r a_ir b_jr c_kr
        M = torch.einsum("r,ir,jr,kr->kji", lam, H[0], H[1], H[2][k0:k1])
        D = Xv[k0:k1].double() - M
        num += float((D * D).sum())
        den += float((Xv[k0:k1].double() ** 2).sum())
    eps = (num / den) ** 0.5
    assert abs(res["rel_err"][-1] - eps) < 2e-5
