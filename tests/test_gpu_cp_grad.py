"""GPU parity of the CP-loss gradient (planc_cp_grad and the CPLoss autograd
node) against the FP64 oracle, central finite differences and gradcheck.

Tolerances: FP64 loss and gradient within 1e-10 relative of the oracle's
(same arithmetic up to summation order); FP32 gradient entries within
1e-4 of the scale max(|2 H S|, |2 M|) of their own terms (the gradient is a
difference of two FP32 quantities of that size, each accurate to ~1e-6);
finite differences in FP64 with step 1e-6 agree to 1e-6 relative.
"""

import numpy as np
import pytest
import torch

import oracle as o
from paper_1909_01149_gb300 import synth
from helpers import factors_to_device, planc, x_to_device

pytestmark = pytest.mark.gpu


def _setup(dims, R, dt, seed=3, noise=0.05):
    p = planc()
    X, _ = synth.planted(dims, R, seed, noise=noise)
    Xd, Xs = x_to_device(X, dt)
    fdt = "f64" if dt == "f64" else "f32"
    Hd, Hs = factors_to_device(synth.init_factors(dims, R, seed + 1), fdt)
    return p, Xd, Xs, Hd, Hs


@pytest.mark.parametrize("dims,split", [((12, 12, 12, 12), -1), ((12, 12, 12, 12), 1),
                                        ((12, 12, 12, 12), 3), ((9, 14, 11), 1),
                                        ((9, 14, 11), 2), ((20, 17), 1)])
def test_cp_grad_fp64_matches_oracle(dims, split):
    R = 4
    p, Xd, Xs, Hd, Hs = _setup(dims, R, "f64")
    with p.Context(Xd, dims, R, split) as ctx:
        loss, dH = ctx.cp_grad(Hd)
    ref = o.cp_loss(Xs, Hs)
    gref = o.cp_loss_grad(Xs, Hs)
    assert abs(loss - ref) <= 1e-10 * ref
    for g, gr in zip(dH, gref):
        np.testing.assert_allclose(g.cpu().numpy(), gr, rtol=1e-10,
                                   atol=1e-10 * np.abs(gr).max())


def test_cp_grad_fp64_central_differences():
    """Central differences of the GPU loss reproduce the GPU gradient."""
    dims, R = (12, 12, 12, 12), 4
    p, Xd, Xs, Hd, Hs = _setup(dims, R, "f64")
    rng = np.random.default_rng(7)
    with p.Context(Xd, dims, R) as ctx:
        _, dH = ctx.cp_grad(Hd)
        for _ in range(12):
            n = int(rng.integers(len(dims)))
            i, r = int(rng.integers(dims[n])), int(rng.integers(R))
            h = 1e-6 * max(1.0, abs(float(Hd[n][i, r])))
            Hp = [t.clone() for t in Hd]
            Hm = [t.clone() for t in Hd]
            Hp[n][i, r] += h
            Hm[n][i, r] -= h
            fp, _ = ctx.cp_grad(Hp)
            fm, _ = ctx.cp_grad(Hm)
            fd = (fp - fm) / (2 * h)
            g = float(dH[n][i, r])
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (n, i, r, fd, g)


def test_cp_loss_autograd_and_gradcheck():
    dims, R = (6, 5, 7), 3
    p, Xd, Xs, Hd, Hs = _setup(dims, R, "f64")
    with p.Context(Xd, dims, R) as ctx:
        H = [h.clone().requires_grad_(True) for h in Hd]
        loss = p.CPLoss.apply(ctx, *H)
        loss.backward()
        gref = o.cp_loss_grad(Xs, Hs)
        for h, gr in zip(H, gref):
            np.testing.assert_allclose(h.grad.cpu().numpy(), gr, rtol=1e-10,
                                       atol=1e-10 * np.abs(gr).max())
        # a scaled upstream gradient scales every factor gradient
        H2 = [h.detach().clone().requires_grad_(True) for h in Hd]
        (3.0 * p.CPLoss.apply(ctx, *H2)).backward()
        np.testing.assert_allclose(H2[0].grad.cpu().numpy(), 3.0 * gref[0], rtol=1e-10,
                                   atol=1e-10 * np.abs(gref[0]).max())
        Hg = tuple(h.detach().clone().requires_grad_(True) for h in Hd)
        assert torch.autograd.gradcheck(lambda *hs: p.CPLoss.apply(ctx, *hs), Hg,
                                        eps=1e-6, atol=1e-5, rtol=1e-6)


@pytest.mark.parametrize("dims,R", [((20, 24, 16, 18), 8), ((40, 36, 44), 17)])
def test_cp_grad_fp32(dims, R):
    p, Xd, Xs, Hd, Hs = _setup(dims, R, "f32")
    with p.Context(Xd, dims, R) as ctx:
        loss, dH = ctx.cp_grad(Hd)
    ref = o.cp_loss(Xs, Hs)
    assert abs(loss - ref) <= 1e-5 * ref
    G = [o.gram(h) for h in Hs]
    for n, g in enumerate(dH):
        HS = 2.0 * Hs[n] @ o.gram_hadamard(G, n)
        M2 = 2.0 * o.mttkrp(Xs, Hs, n)
        scale = np.maximum(np.abs(HS), np.abs(M2))
        err = np.abs(g.cpu().numpy() - (HS - M2))
        assert np.all(err <= 1e-4 * scale + 1e-30), (n, float(np.max(err / scale)))


def test_cp_grad_full_size_sampled_rows():
    """96^4 FP32, R = 64: sampled gradient rows against the oracle's rows."""
    dims, R = (96, 96, 96, 96), 64
    p, Xd, Xs, Hd, Hs = _setup(dims, R, "f32", noise=0.01)
    with p.Context(Xd, dims, R) as ctx:
        loss, dH = ctx.cp_grad(Hd)
    G = [o.gram(h) for h in Hs]
    rng = np.random.default_rng(11)
    for n in range(4):
        rows = np.sort(rng.choice(dims[n], size=6, replace=False))
        M2 = 2.0 * o.mttkrp_rows(Xs, Hs, n, rows)
        HS = 2.0 * Hs[n][rows] @ o.gram_hadamard(G, n)
        got = dH[n].cpu().numpy()[rows]
        scale = np.maximum(np.abs(HS), np.abs(M2))
        assert np.all(np.abs(got - (HS - M2)) <= 1e-4 * scale), n
    assert np.isfinite(loss) and loss > 0


def test_cp_grad_rejects_bad_arguments():
    p = planc()
    dims, R = (6, 7, 8), 3
    X = torch.rand(int(np.prod(dims)), device="cuda")
    Hd = [torch.rand(d, R, device="cuda") for d in dims]
    with p.Context(X, dims, R) as ctx:
        with pytest.raises((ValueError, p.PlancError)):
            ctx.cp_grad(Hd[:2])
        with pytest.raises((ValueError, p.PlancError)):
            ctx.cp_grad(Hd, [torch.rand(d, R + 1, device="cuda") for d in dims])


def test_cp_grad_repeated_calls_reuse_the_norm():
    """||X||^2 is computed on the first call with a loss and reused: later
    calls, also after a solve on the same context, give the oracle's loss."""
    dims, R = (10, 13, 9), 3
    p, Xd, Xs, Hd, Hs = _setup(dims, R, "f64", seed=11)
    ref = o.cp_loss(Xs, Hs)
    with p.Context(Xd, dims, R) as ctx:
        l1, _ = ctx.cp_grad(Hd)
        l2, g2 = ctx.cp_grad(Hd)
        Hs2 = [h.clone() for h in Hd]
        ctx.solve(Hs2, "hals", 2)
        l3, g3 = ctx.cp_grad(Hd)
    assert abs(l1 - ref) <= 1e-10 * abs(ref) and l2 == l1 and l3 == l1
    for a, b in zip(g2, g3):
        assert torch.equal(a, b)
