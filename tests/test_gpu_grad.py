"""Gradient of the log-likelihood on the GPU (sbv_loglik_grad, FP64) against
the gradient oracle and against central differences of the GPU likelihood.

- Small problems, every nu: per-block gradients agree with oracle/grad.py
  (dense inverses and traces, pinned by central differences of the likelihood
  oracle) to 1e-8 of the gradient's scale; the block terms are bit for bit
  those of sbv_loglik in FP64.
- sine10d shape (20,000 points; and the full 1M-point workload on sampled
  blocks): the total gradient matches central differences of the FP64
  likelihood (a property at any size), and sampled blocks match the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import grad as og
from oracle import sbv
from synth.inputs import uniform_points, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


def structure(ctx, X, beta_scale, bc, m, seed=11):
    Xd = torch.from_numpy(X).cuda()
    b = ctx.sbv_blocking(Xd, beta_scale, bc, 3, seed)
    nbr, cnt = ctx.sbv_knn(Xd, beta_scale, b["ptr"], b["pts"], b["rank"], b["centres"], m)
    return Xd, b, nbr.contiguous(), cnt


@pytest.mark.parametrize("nu2", [1, 3, 5, 7])
def test_block_gradients_match_oracle(ctx, nu2):
    n, d, bc, m = 600, 3, 60, 15
    X = uniform_points(n, d, 21)
    y = np.sin(5 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.1 * np.random.default_rng(2).standard_normal(n)
    Xd, b, nbr, cnt = structure(ctx, X, np.full(d, 0.3), bc, m)
    yd = torch.from_numpy(y).cuda()
    th = np.array([[1.2, 0.03, 0.2, 0.35, 0.5], [0.7, 0.1, 0.5, 0.25, 0.3]])
    bt = torch.empty(2, bc, dtype=torch.float64, device="cuda")
    bg = torch.empty(2, bc, d + 2, dtype=torch.float64, device="cuda")
    ll, g = ctx.sbv_loglik_grad(Xd, yd, b["ptr"], b["pts"], nbr, cnt, th, nu2, block_terms=bt,
                                block_grads=bg)
    bt0 = torch.empty(2, bc, dtype=torch.float64, device="cuda")
    ll0 = ctx.sbv_loglik(Xd, yd, b["ptr"], b["pts"], nbr, cnt, th, nu2, precision="fp64",
                         block_terms=bt0)
    assert torch.equal(bt, bt0) and torch.equal(ll, ll0)
    ptr, pts = b["ptr"].cpu().numpy(), b["pts"].cpu().numpy()
    nb, cn = nbr.cpu().numpy(), cnt.cpu().numpy()
    bg = bg.cpu().numpy()
    for r in range(2):
        want = og.grad_terms(X, y, ptr, pts, nb, cn, th[r], nu2)
        scale = np.abs(want).max(axis=0) + 1.0
        assert np.all(np.abs(bg[r] - want) <= 1e-8 * scale), (r, np.abs(bg[r] - want).max(axis=0))
        assert np.allclose(g.cpu().numpy()[r], want.sum(axis=0), rtol=1e-9, atol=1e-8)


def fd_check(ctx, Xd, yd, b, nbr, cnt, th, g, rel=1e-4, tol=1e-4):
    for k in range(th.size):
        h = rel * th[k]
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        lp = ctx.sbv_loglik(Xd, yd, b["ptr"], b["pts"], nbr, cnt, tp, 5, precision="fp64").item()
        lm = ctx.sbv_loglik(Xd, yd, b["ptr"], b["pts"], nbr, cnt, tm, 5, precision="fp64").item()
        fd = (lp - lm) / (2 * h)
        assert abs(g[k] - fd) <= tol * (abs(fd) + abs(g).max() * 1e-3), (k, g[k], fd)


def test_total_gradient_matches_central_differences(ctx):
    w = workload("sine10d", n=20000, bc=400, m=60)
    Xd, b, nbr, cnt = structure(ctx, w["X"], w["beta_scale"], w["bc"], w["m"])
    yd = torch.from_numpy(w["y"]).cuda()
    th = np.asarray(w["theta"], dtype=np.float64).reshape(-1, 12)[0]
    ll, g = ctx.sbv_loglik_grad(Xd, yd, b["ptr"], b["pts"], nbr, cnt, th, 5)
    fd_check(ctx, Xd, yd, b, nbr, cnt, th, g.cpu().numpy()[0])


def test_full_size_sampled_blocks_and_differences(ctx):
    w = workload("sine10d")
    Xd, b, nbr, cnt = structure(ctx, w["X"], w["beta_scale"], w["bc"], w["m"])
    yd = torch.from_numpy(w["y"]).cuda()
    th = np.asarray(w["theta"], dtype=np.float64).reshape(-1, 12)[0]
    bc = cnt.numel()
    nmax = ctx.max_block_size(b["ptr"], cnt)
    bg = torch.empty(1, bc, 12, dtype=torch.float64, device="cuda")
    ll, g = ctx.sbv_loglik_grad(Xd, yd, b["ptr"], b["pts"], nbr, cnt, th, 5, block_grads=bg,
                                nmax=nmax)
    torch.cuda.synchronize()
    ctx.sbv_sync_status()
    ptr, pts = b["ptr"].cpu().numpy(), b["pts"].cpu().numpy()
    nb, cn = nbr.cpu().numpy(), cnt.cpu().numpy()
    sample = np.random.default_rng(3).choice(bc, 5, replace=False)
    want = og.grad_terms(w["X"], w["y"], ptr, pts, nb, cn, th, 5, blocks=sample)
    got = bg.cpu().numpy()[0][sample]
    scale = np.abs(want).max(axis=0) + 1.0
    assert np.all(np.abs(got - want) <= 1e-8 * scale), np.abs(got - want).max(axis=0)
    fd_check(ctx, Xd, yd, b, nbr, cnt, th, g.cpu().numpy()[0])
