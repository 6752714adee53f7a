"""Synthetic accuracy study (Sec. 7.1, Fig. maternsimu) through the GPU path.

Data as the paper sets it: x uniform on [0,1]^10, y an exact draw of the
zero-mean GP with the Matern kernel at nu = 3.5, sigma^2 = 1, tau^2 = 0,
beta = (0.05, 0.05, 5, ..., 5); n = 2,000 training and 500 test points (the
draw by dense Cholesky of the joint covariance); the true parameters are
given to every method.  The four Vecchia variants are the SBV pipeline with
one-point blocks (bc = n) and/or no input scaling (beta_scale = 1):
CV (unscaled, one point per block), BV (unscaled, blocks of ~10),
SV (scaled, one point), SBV (scaled, blocks of ~10).

Fitting accuracy is KL(p || q) = -l_q(0) - n/2 log 2 pi - 1/2 log det Sigma
(the KL identity pinned in tests/test_oracle_kl.py), with l_q(0) the FP64
log-likelihood of y = 0; prediction accuracy is the MSPE at the test points
(per-point prediction for CV/SV, block prediction with ~10 test points per
block for BV/SBV).  Asserted, as in the paper: scaling makes SV and SBV fit
and predict far better than CV and BV; SBV fits better than SV; every
variant's KL falls as m grows; RAC blocking gives log-likelihood errors
(against the exact GP) comparable to K-means, and both the error and its
spread over five anchor draws fall as m grows.  Measured and not asserted
(they differ from the paper at this size): BV fits worse than CV for
m >= 30; SV predicts better than SBV (the block's neighbours are those of
its centre); blocks of ~12 beat blocks of ~50 only at m = 60.
"""
import numpy as np
import pytest
import torch

from oracle import sbv
from synth.inputs import standard_normal, uniform_points

pytestmark = pytest.mark.gpu

N, NT, D, NU2 = 2000, 500, 10, 7
BETA = np.r_[0.05, 0.05, np.full(8, 5.0)]
THETA = np.r_[1.0, 0.0, BETA]
MS = (10, 30, 60)


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


@pytest.fixture(scope="module")
def data():
    X = uniform_points(N + NT, D, 77)
    idx = np.arange(N + NT)
    K = sbv.cov_points(X, idx, idx, THETA, NU2)
    y = np.linalg.cholesky(K) @ standard_normal(N + NT, 78)
    Lt = np.linalg.cholesky(K[:N, :N])
    logdet = 2.0 * np.log(np.diag(Lt)).sum()
    w = np.linalg.solve(Lt, y[:N])
    l_exact = -0.5 * (w @ w + logdet + N * np.log(2 * np.pi))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dict(X=dev(X[:N]), y=dev(y[:N]), Xt=dev(X[N:]), yt=y[N:], Xh=X[:N], yh=y[:N],
                logdet=logdet, l_exact=l_exact)


def structure(ctx, data, beta_scale, bc, m, T=3, seed=11):
    b = ctx.sbv_blocking(data["X"], beta_scale, bc, T, seed)
    nbr, cnt = ctx.sbv_knn(data["X"], beta_scale, b["ptr"], b["pts"], b["rank"], b["centres"], m)
    return b, nbr.contiguous(), cnt


def loglik(ctx, data, s, y):
    b, nbr, cnt = s
    return float(ctx.sbv_loglik(data["X"], y, b["ptr"], b["pts"], nbr, cnt, THETA, NU2, "fp64")[0])


def kl(ctx, data, s):
    l0 = loglik(ctx, data, s, torch.zeros_like(data["y"]))
    return -l0 - 0.5 * N * np.log(2 * np.pi) - 0.5 * data["logdet"]


VARIANTS = {"CV": (False, N), "BV": (False, N // 10), "SV": (True, N), "SBV": (True, N // 10)}


def test_kl_divergence_of_the_four_variants(ctx, data):
    table = {}
    for m in MS:
        for name, (scaled, bc) in VARIANTS.items():
            table[name, m] = kl(ctx, data, structure(ctx, data, BETA if scaled else np.ones(D), bc, m))
    print({k: round(v, 3) for k, v in table.items()})
    for m in MS:
        assert table["SBV", m] < table["SV", m] < min(table["CV", m], table["BV", m])
        assert 3 * table["SV", m] < min(table["CV", m], table["BV", m])
    for name in VARIANTS:
        assert table[name, 10] > table[name, 30] > table[name, 60] > 0
    # one value against the oracle (same structure bit for bit, FP64 terms)
    s = structure(ctx, data, BETA, N // 10, 30)
    b, nbr, cnt = s
    l0 = sbv.loglik(data["Xh"], np.zeros(N), b["ptr"].cpu().numpy(), b["pts"].cpu().numpy(),
                    nbr.cpu().numpy(), cnt.cpu().numpy(), b["rank"].cpu().numpy(), THETA, NU2)
    want = -l0 - 0.5 * N * np.log(2 * np.pi) - 0.5 * data["logdet"]
    assert abs(table["SBV", 30] - want) <= 1e-9 * N


def test_prediction_error_of_the_four_variants(ctx, data):
    mspe = {}
    for m in MS:
        for name, (scaled, bc) in VARIANTS.items():
            bsc = BETA if scaled else np.ones(D)
            if bc == N:
                mu = ctx.sbv_predict(data["X"], data["y"], data["Xt"], bsc, m, THETA, NU2, "fp64")[0]
            else:
                mu = ctx.sbv_predict_blocked(data["X"], data["y"], data["Xt"], bsc, m, NT // 10, THETA,
                                             NU2, "fp64", 3, 5)[0]
            mspe[name, m] = float(np.mean((mu.cpu().numpy() - data["yt"]) ** 2))
    print({k: round(v, 5) for k, v in mspe.items()})
    for m in MS:
        assert 3 * max(mspe["SV", m], mspe["SBV", m]) < min(mspe["CV", m], mspe["BV", m])
    for name in VARIANTS:
        assert mspe[name, 10] > mspe[name, 30] > mspe[name, 60]


def test_rac_against_kmeans(ctx, data):
    """Relative error |l - l_exact| / |l_exact| of SBV with K-means blocking
    (10 Lloyd iterations) and with RAC (no iteration), five anchor draws each."""
    y = data["y"]
    rows = {}
    for m in MS:
        for T in (0, 10):
            e = [abs(loglik(ctx, data, structure(ctx, data, BETA, N // 10, m, T, 100 + s), y)
                     - data["l_exact"]) / abs(data["l_exact"]) for s in range(5)]
            rows[T, m] = (float(np.mean(e)), float(np.var(e)))
    print(rows)
    for m in MS:
        assert rows[0, m][0] <= 1.2 * rows[10, m][0]          # comparable to K-means
    assert rows[0, 10][0] > rows[0, 30][0] > rows[0, 60][0]
    assert rows[0, 10][1] > rows[0, 60][1]
