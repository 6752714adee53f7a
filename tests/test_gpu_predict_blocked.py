"""Block prediction (Sec. 5.5; sbv_predict_blocked) against the oracle: the
test blocking and every block's neighbour set bit for bit, means and
variances within the precision's bar; one-point blocks reproduce the
per-point prediction; blocks larger than the planned capacity go through the
FP64 hand-over; argument errors.
"""
import numpy as np
import pytest
import torch

from oracle import sbv
from synth.inputs import standard_normal, uniform_points, workload

pytestmark = pytest.mark.gpu

# relative to sqrt(var) for the mean and to var for the variance
TOL = {"fp64": 1e-9, "mixed": 1e-6, "mixed_bf16": 1e-6}


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


@pytest.fixture(scope="module")
def gp5d():
    w = workload("gp5d")
    idx = np.arange(w["n"])
    y = np.linalg.cholesky(sbv.cov_points(w["X"], idx, idx, w["theta"][0], 5)) @ w["z"]
    return w, y


def check(got, want, tol):
    m, v, vl = (t.cpu().numpy() for t in got[:3])
    om, ov, ovl = want[:3]
    sd = np.sqrt(ov)
    assert np.all(np.abs(m - om) <= tol * sd), np.max(np.abs(m - om) / sd)
    assert np.all(np.abs(v - ov) <= tol * ov), np.max(np.abs(v - ov) / ov)
    assert np.all(np.abs(vl - ovl) <= tol * ov)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("use_blocks", [False, True])
def test_block_prediction_matches_oracle(ctx, gp5d, precision, use_blocks):
    w, y = gp5d
    X, Xt, beta, th = w["X"], w["Xtest"], w["beta_scale"], w["theta"][0]
    bc_test, m_pred, T, seed = 50, w["m"], 3, 17
    Xd = torch.from_numpy(X).cuda()
    blocks = ctx.sbv_blocking(Xd, beta, w["bc"], 3, 11) if use_blocks else None
    got = ctx.sbv_predict_blocked(Xd, torch.from_numpy(y).cuda(), torch.from_numpy(Xt).cuda(),
                                  beta, m_pred, bc_test, th, 5, precision, T, seed, blocks=blocks)
    want = sbv.predict_blocked(X, y, Xt, beta, m_pred, bc_test, T, seed, th, 5)
    assert np.array_equal(got[3].cpu().numpy(), want[3])          # test blocks
    assert np.array_equal(got[4].cpu().numpy(), want[4])          # neighbour sets
    check(got, want, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_point_blocks_equal_per_point_prediction(ctx, gp5d, precision):
    w, y = gp5d
    Xd, yd = torch.from_numpy(w["X"]).cuda(), torch.from_numpy(y).cuda()
    Xt = torch.from_numpy(w["Xtest"][:80]).cuda()
    a = ctx.sbv_predict_blocked(Xd, yd, Xt, w["beta_scale"], 40, 80, w["theta"][0], 5, precision)
    b = ctx.sbv_predict(Xd, yd, Xt, w["beta_scale"], 40, w["theta"][0], 5, precision)
    for x, z in zip(a[:3], b[:3]):
        assert torch.equal(x, z)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_test_blocks(ctx, precision):
    """Blocks of ~100-250 test points with 150 neighbours (N up to ~400); the
    mixed kernel plans for the largest block and hands over nothing."""
    n, d = 3000, 4
    X, y = uniform_points(n, d, 41), standard_normal(n, 42)
    Xt = uniform_points(700, d, 43)
    beta, th = np.array([0.3, 0.5, 0.7, 0.9]), np.array([1.0, 0.01, 0.3, 0.5, 0.7, 0.9])
    got = ctx.sbv_predict_blocked(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(),
                                  torch.from_numpy(Xt).cuda(), beta, 150, 4, th, 5, precision, 2, 3)
    want = sbv.predict_blocked(X, y, Xt, beta, 150, 4, 2, 3, th, 5)
    assert np.array_equal(got[3].cpu().numpy(), want[3])
    check(got, want, TOL[precision])


def test_block_prediction_rejects_bad_arguments(ctx, gp5d):
    from paper_2504_12004_gb300 import SBVError
    w, y = gp5d
    Xd, yd = torch.from_numpy(w["X"]).cuda(), torch.from_numpy(y).cuda()
    Xt = torch.from_numpy(w["Xtest"][:10]).cuda()
    for bc_test in (0, 11):
        with pytest.raises(SBVError):
            ctx.sbv_predict_blocked(Xd, yd, Xt, w["beta_scale"], 20, bc_test, w["theta"][0])
    with pytest.raises(SBVError):     # general nu is FP64 only
        ctx.sbv_predict_blocked(Xd, yd, Xt, w["beta_scale"], 20, 2, w["theta"][0], 4, "mixed")
