"""Pins of oracle.mle: closed-form maximisers and stationarity.

- m = 0 and one point per block: the likelihood is that of independent
  N(0, sigma^2 + tau^2) draws, maximised (tau^2 = 0) at sigma^2 = mean(y^2).
- tau^2 = 0 with the ranges fixed: the scale-family maximiser sigma^2 = Q/n,
  with Q taken from two likelihood evaluations (not from the optimiser).
- All parameters free: the returned point is no worse than the start and its
  central-difference gradient in log theta vanishes to the optimiser's
  tolerance.
"""
import numpy as np

from oracle import mle, sbv
from synth.inputs import uniform_points


def structure(n, d, bc, m, seed):
    X = uniform_points(n, d, seed)
    beta = np.full(d, 0.3)
    b = sbv.blocking(X, beta, bc, 3, seed)
    nbr, cnt = sbv.knn(b["Z"], b["blk"], b["rank"], b["centres"], m)
    return X, b, nbr, cnt


def gp_y(X, theta, nu2, seed):
    idx = np.arange(len(X))
    S = sbv.cov_points(X, idx, idx, theta, nu2)
    return np.linalg.cholesky(S) @ np.random.default_rng(seed).standard_normal(len(X))


def test_independent_blocks_variance_mle():
    X, b, nbr, cnt = structure(120, 2, 120, 0, 4)
    assert np.all(cnt == 0) and len(b["rank"]) == 120
    y = np.random.default_rng(0).standard_normal(120) * 1.7
    f = mle.make_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, b["rank"], 5)
    th, val, _ = mle.mle(f, [1.0, 0.0, 0.3, 0.3], free=[True, False, False, False])
    assert abs(th[0] - np.mean(y * y)) <= 1e-6 * np.mean(y * y)
    s = np.mean(y * y)
    assert abs(val - (-0.5 * 120 * (np.log(2 * np.pi * s) + 1.0))) < 1e-8


def test_scale_family_closed_form():
    theta = np.array([1.3, 0.0, 0.2, 0.5])
    X, b, nbr, cnt = structure(300, 2, 30, 12, 5)
    y = gp_y(X, theta, 1, 6)
    f = mle.make_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, b["rank"], 1)
    want = mle.sigma2_closed_form(f, theta, 300)
    th, _, _ = mle.mle(f, theta, free=[True, False, False, False])
    assert abs(th[0] - want) <= 1e-6 * want, (th[0], want)


def test_all_free_is_stationary_and_improves():
    theta0 = np.array([0.7, 0.05, 0.5, 0.5])
    X, b, nbr, cnt = structure(300, 2, 30, 12, 7)
    y = gp_y(X, np.array([1.2, 0.01, 0.15, 0.4]), 5, 8)
    f = mle.make_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, b["rank"], 5)
    th, val, nev = mle.mle(f, theta0, lower=[1e-3, 1e-6, 1e-3, 1e-3], upper=[1e2, 1e1, 1e1, 1e1])
    assert val >= f(theta0) and abs(val - f(th)) < 1e-9
    u = np.log(th)
    h = 1e-4
    g = np.array([(f(np.exp(u + h * e)) - f(np.exp(u - h * e))) / (2 * h) for e in np.eye(4)])
    inside = (th > 1.001e-6) & (th < 0.999e1)
    assert np.all(np.abs(g[inside]) < 1e-3), g
