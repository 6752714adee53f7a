"""Pins of the FP64 gradient oracle (oracle/grad.py), which writes out the
textbook derivative of the block conditional's Gaussian log-density:

- central differences of the likelihood oracle (oracle.sbv.block_loglik,
  an independent code path: Cholesky factors, no inverses or traces) agree
  with every component, for every nu, on several blocks;
- at tau^2 = 0 the likelihood is a scale family in sigma^2, whose derivative
  has the closed form -bs / (2 sigma^2) + (Q_S - Q_J) / (2 sigma^4) with
  Q = y^T M^{-1} y from linear solves with the correlation matrix;
- the block gradients add up to the derivative of the total likelihood.
"""
import numpy as np
import pytest

from oracle import grad as og
from oracle import sbv
from synth.inputs import uniform_points


def problem(n=300, d=3, bc=30, m=10, seed=2):
    X = uniform_points(n, d, seed)
    y = np.sin(5 * X[:, 0]) + X[:, 1] * X[:, -1] + 0.1 * np.random.default_rng(seed).standard_normal(n)
    b = sbv.blocking(X, np.full(d, 0.3), bc, 3, seed)
    nbr, cnt = sbv.knn(b["Z"], b["blk"], b["rank"], b["centres"], m)
    return X, y, b, nbr, cnt


def fd_block(X, y, J, B, theta, nu2, k, rel=1e-5):
    h = rel * theta[k]
    tp, tm = theta.copy(), theta.copy()
    tp[k] += h
    tm[k] -= h
    return (sbv.block_loglik(X, y, J, B, tp, nu2) - sbv.block_loglik(X, y, J, B, tm, nu2)) / (2 * h)


@pytest.mark.parametrize("nu2", [1, 2, 3, 4, 5, 7, 9])
def test_central_differences(nu2):
    X, y, b, nbr, cnt = problem()
    theta = np.array([1.3, 0.02, 0.25, 0.4, 0.6])
    for blk in [0, 7, 19, 29]:
        J, B = nbr[blk, :cnt[blk]], b["pts"][b["ptr"][blk]:b["ptr"][blk + 1]]
        g = og.block_grad(X, y, J, B, theta, nu2)
        fd = np.array([fd_block(X, y, J, B, theta, nu2, k) for k in range(theta.size)])
        assert np.allclose(g, fd, rtol=1e-5, atol=1e-6 * (1 + np.abs(g).max())), (nu2, blk, g, fd)


def test_sigma2_closed_form_at_zero_nugget():
    X, y, b, nbr, cnt = problem(n=200, d=2, bc=20, m=8, seed=5)
    s2 = 1.7
    # short ranges keep the nugget-free correlation matrices well conditioned
    theta = np.array([s2, 0.0, 0.08, 0.12])
    unit = np.array([1.0, 0.0, 0.08, 0.12])

    def Q(idx):
        M = sbv.cov_points(X, idx, idx, unit, 5)      # the correlation matrix
        return float(y[idx] @ np.linalg.solve(M, y[idx]))

    for blk in [1, 10, 19]:
        J, B = nbr[blk, :cnt[blk]], b["pts"][b["ptr"][blk]:b["ptr"][blk + 1]]
        S = np.concatenate([J, B])
        want = -B.size / (2 * s2) + (Q(S) - (Q(J) if J.size else 0.0)) / (2 * s2 ** 2)
        g = og.block_grad(X, y, J, B, theta, 5)
        assert g[0] == pytest.approx(want, rel=1e-9)


def test_block_gradients_add_up_to_the_total():
    X, y, b, nbr, cnt = problem(n=120, d=2, bc=12, m=6, seed=7)
    theta = np.array([0.9, 0.05, 0.2, 0.35])
    G = og.grad_terms(X, y, b["ptr"], b["pts"], nbr, cnt, theta, 5)
    assert G.shape == (12, 4)

    def total(th):
        return sbv.loglik(X, y, b["ptr"], b["pts"], nbr, cnt, b["rank"], th, 5)

    for k in range(4):
        h = 1e-5 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (total(tp) - total(tm)) / (2 * h)
        assert G[:, k].sum() == pytest.approx(fd, rel=1e-5, abs=1e-6)


def test_h_nu_is_minus_derivative_over_r():
    r = np.linspace(0.05, 6.0, 50)
    for nu2 in (1, 2, 3, 4, 5, 7, 9, 20):
        e = 1e-6
        dM = (sbv.matern(r + e, nu2) - sbv.matern(r - e, nu2)) / (2 * e)
        assert np.allclose(og.h_nu(r, nu2), -dM / r, rtol=1e-7), nu2
    assert og.h_nu(np.array([0.0]), 1)[0] == 0.0
    # the r -> 0 limit 1 / (2 (nu - 1)) of the Bessel form (nu = 2, 4.5)
    for nu2 in (4, 9):
        nu = nu2 / 2
        assert og.h_nu(np.array([1e-7]), nu2)[0] == pytest.approx(0.5 / (nu - 1), rel=1e-6)
        assert og.h_nu(np.array([0.0]), nu2)[0] == 0.5 / (nu - 1)
