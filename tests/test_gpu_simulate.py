"""Conditional simulation (Sec. 5.5) on the GPU against the oracle: every draw
element by element, the sample means, variances and interval ends; ragged draw
counts, zero variances, chunking by index_base, argument errors; the predictive
means and variances of a real prediction; and the 1M-test-point case (1000
draws each) on sampled points and through the sampling law of the means.
"""
import numpy as np
import pytest
import torch

from oracle import sbv
from oracle import simulate as osim
from synth.inputs import workload

pytestmark = pytest.mark.gpu

# FP64 on both sides; the GPU takes sincospi(2 u) where the oracle takes
# cos(2 pi u) and merges Welford partial moments where the oracle sums twice,
# so results agree to a few units in the last place of the draws' scale
RTOL = 1e-13


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


def check(ctx, mean, var, ndraws, seed, index_base=0, draws=True):
    md, vd = torch.from_numpy(mean).cuda(), torch.from_numpy(var).cuda()
    mu, s2, lo, hi, dr = ctx.sbv_simulate(md, vd, ndraws, seed, index_base, want_draws=draws)
    torch.cuda.synchronize()
    o_dr, o_mu, o_s2, o_lo, o_hi = osim.simulate(mean, var, ndraws, seed, index_base=index_base)
    scale = np.abs(mean) + np.sqrt(var) + 1e-300
    if draws:
        err = np.abs(dr.cpu().numpy() - o_dr) / scale[:, None]
        assert err.max() < RTOL, err.max()
    assert np.all(np.abs(mu.cpu().numpy() - o_mu) <= RTOL * scale)
    assert np.all(np.abs(s2.cpu().numpy() - o_s2) <= RTOL * (o_s2 + var * 1e-3 + 1e-300))
    assert np.all(np.abs(lo.cpu().numpy() - o_lo) <= 2 * RTOL * scale)
    assert np.all(np.abs(hi.cpu().numpy() - o_hi) <= 2 * RTOL * scale)
    return mu, s2, lo, hi, dr


@pytest.mark.parametrize("ndraws", [2, 3, 5, 37, 128, 1000])
def test_simulate_matches_oracle(ctx, ndraws):
    rng = np.random.default_rng(ndraws)
    nt = 97
    mean = rng.normal(0.0, 5.0, nt)
    var = rng.uniform(1e-4, 3.0, nt)
    check(ctx, mean, var, ndraws, seed=0xDEADBEEF12345678)


def test_simulate_edge_cases(ctx):
    # zero variance: every draw is the mean; a negative variance gives NaN
    mean = np.array([1.5, -2.0, 0.0])
    var = np.array([0.0, 0.0, 1.0])
    mu, s2, lo, hi, dr = check(ctx, mean, var, 11, seed=3)
    assert torch.all(dr[:2] == torch.from_numpy(mean[:2, None]).cuda())
    assert torch.all(s2[:2] == 0) and torch.all(lo[:2] == mu[:2]) and torch.all(hi[:2] == mu[:2])
    md = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    out = ctx.sbv_simulate(md, -md, 10, 1)
    assert torch.isnan(out[0]).all() and torch.isnan(out[1]).all()
    # no test points: a no-op
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    out = ctx.sbv_simulate(e, e, 1000, 1)
    assert out[0].numel() == 0
    # the statistics do not depend on whether the draws are written
    rng = np.random.default_rng(2)
    m, v = rng.normal(size=40), rng.uniform(0.1, 1, 40)
    a = ctx.sbv_simulate(torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda(), 333, 9)
    b = ctx.sbv_simulate(torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda(), 333, 9,
                         want_draws=True)
    for x, y in zip(a[:4], b[:4]):
        assert torch.equal(x, y)
    # repeat calls are bit-identical; another seed gives other draws
    c = ctx.sbv_simulate(torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda(), 333, 9)
    d = ctx.sbv_simulate(torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda(), 333, 10)
    assert torch.equal(a[0], c[0]) and not torch.equal(a[0], d[0])


def test_simulate_rejects_bad_arguments(ctx):
    from paper_2504_12004_gb300 import SBVError
    md = torch.ones(4, dtype=torch.float64, device="cuda")
    for nd in (1, 0, -5):
        with pytest.raises(SBVError):
            ctx.sbv_simulate(md, md, nd, 1)


def test_simulate_chunks_by_index_base(ctx):
    rng = np.random.default_rng(12)
    mean, var = rng.normal(size=50), rng.uniform(0.2, 2.0, 50)
    whole = ctx.sbv_simulate(torch.from_numpy(mean).cuda(), torch.from_numpy(var).cuda(), 64, 77,
                             want_draws=True)[4]
    part = ctx.sbv_simulate(torch.from_numpy(mean[30:]).cuda(), torch.from_numpy(var[30:]).cuda(),
                            64, 77, index_base=30, want_draws=True)[4]
    assert torch.equal(whole[30:], part)
    check(ctx, mean[30:], var[30:], 64, 77, index_base=30)


def test_simulate_from_prediction(ctx):
    """The Sec. 5.5 pipeline on the 4,000-point gp5d workload: predictive mean
    and variance at its 500 test points (FP64), then 1000 draws each."""
    w = workload("gp5d")
    idx = np.arange(w["n"])
    y = np.linalg.cholesky(sbv.cov_points(w["X"], idx, idx, w["theta"][0], 5)) @ w["z"]
    Xd = torch.from_numpy(w["X"]).cuda()
    Xt = torch.from_numpy(w["Xtest"]).cuda()
    mean, var, _, _ = ctx.sbv_predict(Xd, torch.from_numpy(y).cuda(), Xt, w["beta_scale"], w["m"],
                                      w["theta"][0], 5, "fp64")
    check(ctx, mean.cpu().numpy(), var.cpu().numpy(), 1000, seed=2025)


def test_simulate_one_million_test_points(ctx):
    """1,000,000 test points x 1000 draws (the paper's draw count): sampled
    points against the oracle, and the standardised sample means and variances
    of all points against their sampling laws."""
    nt, nd = 1_000_000, 1000
    g = torch.Generator(device="cuda").manual_seed(5)
    mean = torch.randn(nt, dtype=torch.float64, device="cuda", generator=g) * 2.0
    var = torch.rand(nt, dtype=torch.float64, device="cuda", generator=g) * 2.0 + 0.05
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.sbv_simulate(mean, var, nd, 31)
    start.record()
    mu, s2, lo, hi, _ = ctx.sbv_simulate(mean, var, nd, 31)
    end.record()
    torch.cuda.synchronize()
    print(f"1M test points x 1000 draws: {start.elapsed_time(end):.2f} ms")
    t = ((mu - mean) / torch.sqrt(var / nd)).cpu().numpy()
    assert abs(t.mean()) < 5 / np.sqrt(nt) and abs(t.var() - 1) < 0.01
    q = ((nd - 1) * s2 / var).cpu().numpy()
    assert abs(q.mean() - (nd - 1)) < 5 * np.sqrt(2 * (nd - 1) / nt)
    rows = np.random.default_rng(1).choice(nt, 24, replace=False)
    m, v = mean.cpu().numpy(), var.cpu().numpy()
    _, o_mu, o_s2, o_lo, o_hi = osim.simulate(m, v, nd, 31, rows=rows)
    scale = np.abs(m[rows]) + np.sqrt(v[rows])
    assert np.all(np.abs(mu.cpu().numpy()[rows] - o_mu) <= RTOL * scale)
    assert np.all(np.abs(s2.cpu().numpy()[rows] - o_s2) <= RTOL * o_s2)
    assert np.all(np.abs(lo.cpu().numpy()[rows] - o_lo) <= 2 * RTOL * scale)
    assert np.all(np.abs(hi.cpu().numpy()[rows] - o_hi) <= 2 * RTOL * scale)
