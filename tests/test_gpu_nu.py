"""General smoothness nu = nu2/2 on the FP64 paths (Matern through the Bessel
function K_nu) against the oracle (scipy's K_nu): block terms, prediction and
the analytic gradient; the mixed precisions keep the four closed forms and
reject other nu2.
"""
import numpy as np
import pytest
import torch

from oracle import grad as og
from oracle import sbv
from synth.inputs import uniform_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


@pytest.fixture(scope="module")
def prob(ctx):
    n, d, bc, m = 600, 3, 60, 15
    X = uniform_points(n, d, 31)
    y = np.sin(5 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.1 * np.random.default_rng(3).standard_normal(n)
    Xd = torch.from_numpy(X).cuda()
    b = ctx.sbv_blocking(Xd, np.full(d, 0.3), bc, 3, 11)
    nbr, cnt = ctx.sbv_knn(Xd, np.full(d, 0.3), b["ptr"], b["pts"], b["rank"], b["centres"], m)
    return dict(X=X, y=y, Xd=Xd, yd=torch.from_numpy(y).cuda(), b=b, nbr=nbr.contiguous(), cnt=cnt)


@pytest.mark.parametrize("nu2", [2, 4, 9])
def test_block_terms_and_gradient(ctx, prob, nu2):
    th = np.array([1.1, 0.02, 0.2, 0.35, 0.5])
    b, nbr, cnt = prob["b"], prob["nbr"], prob["cnt"]
    bc = cnt.numel()
    bt = torch.empty(1, bc, dtype=torch.float64, device="cuda")
    ll = ctx.sbv_loglik(prob["Xd"], prob["yd"], b["ptr"], b["pts"], nbr, cnt, th, nu2,
                        precision="fp64", block_terms=bt)
    ptr, pts = b["ptr"].cpu().numpy(), b["pts"].cpu().numpy()
    nb, cn = nbr.cpu().numpy(), cnt.cpu().numpy()
    want = sbv.loglik_terms(prob["X"], prob["y"], ptr, pts, nb, cn, th, nu2)
    assert np.max(np.abs(bt.cpu().numpy()[0] - want)) <= 1e-8 * (1 + np.abs(want).max())
    assert abs(ll.item() - want.sum()) / 600 <= 1e-9
    bg = torch.empty(1, bc, 5, dtype=torch.float64, device="cuda")
    _, g = ctx.sbv_loglik_grad(prob["Xd"], prob["yd"], b["ptr"], b["pts"], nbr, cnt, th, nu2,
                               block_grads=bg)
    gw = og.grad_terms(prob["X"], prob["y"], ptr, pts, nb, cn, th, nu2)
    scale = np.abs(gw).max(axis=0) + 1.0
    assert np.all(np.abs(bg.cpu().numpy()[0] - gw) <= 1e-7 * scale), np.abs(bg.cpu().numpy()[0] - gw).max(axis=0)


def test_prediction(ctx, prob):
    Xt = uniform_points(60, 3, 32)
    th = np.array([1.1, 0.02, 0.2, 0.35, 0.5])
    mean, var, var_lat, _ = ctx.sbv_predict(prob["Xd"], prob["yd"], torch.from_numpy(Xt).cuda(),
                                            np.full(3, 0.3), 40, th, 4, precision="fp64")
    om, ov, ol, _ = sbv.predict(prob["X"], prob["y"], Xt, np.full(3, 0.3), 40, th, 4)
    assert np.max(np.abs(mean.cpu().numpy() - om)) <= 1e-9
    assert np.max(np.abs(var.cpu().numpy() - ov)) <= 1e-9
    assert np.max(np.abs(var_lat.cpu().numpy() - ol)) <= 1e-9


def test_mixed_rejects_general_nu(ctx, prob):
    from paper_2504_12004_gb300 import SBVError
    th = np.array([1.1, 0.02, 0.2, 0.35, 0.5])
    b = prob["b"]
    with pytest.raises(SBVError):
        ctx.sbv_loglik(prob["Xd"], prob["yd"], b["ptr"], b["pts"], prob["nbr"], prob["cnt"], th, 4,
                       precision="mixed")
    with pytest.raises(SBVError):
        ctx.sbv_loglik(prob["Xd"], prob["yd"], b["ptr"], b["pts"], prob["nbr"], prob["cnt"], th, 41,
                       precision="fp64")
