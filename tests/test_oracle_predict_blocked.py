"""Pins of the oracle's block prediction (Sec. 5.5) against routes that do
not share its composition: one test point per block is the per-point
prediction (the centre of a one-point block is the point itself), and one
block conditioned on every training point is the exact GP conditional of all
the data, computed here by a dense solve with the joint covariance.
"""
import numpy as np

from oracle import sbv
from synth.inputs import standard_normal, uniform_points

BETA = np.array([0.3, 0.5, 0.7])
THETA = np.array([1.2, 0.02, 0.3, 0.5, 0.7])


def test_one_point_blocks_equal_per_point_prediction():
    X, y = uniform_points(400, 3, 1), standard_normal(400, 2)
    Xt = uniform_points(30, 3, 3)
    m, v, vl, blk, nbr = sbv.predict_blocked(X, y, Xt, BETA, 25, 30, 3, 9, THETA, 5)
    pm, pv, pvl, pn = sbv.predict(X, y, Xt, BETA, 25, THETA, 5)
    assert np.array_equal(np.sort(blk), np.arange(30))
    assert np.array_equal(nbr[blk], pn)
    assert np.array_equal(m, pm) and np.array_equal(v, pv) and np.array_equal(vl, pvl)


def test_one_block_with_all_neighbours_is_the_dense_conditional():
    n = 150
    X, y = uniform_points(n, 3, 4), standard_normal(n, 5)
    Xt = uniform_points(12, 3, 6)
    m, v, vl, blk, nbr = sbv.predict_blocked(X, y, Xt, BETA, n, 1, 0, 1, THETA, 3)
    assert np.all(blk == 0) and np.array_equal(np.sort(nbr[0]), np.arange(n))
    # dense joint covariance of (training, test) and the Gaussian conditional
    idx = np.arange(n)
    K = sbv.cov_points(X, idx, idx, THETA, 3)
    Kt = sbv.cov(np.asarray(X, dtype=np.float64), Xt, THETA, 3)          # n x 12, no nugget
    w = np.linalg.solve(K, Kt)
    mean = w.T @ y
    var = THETA[0] + THETA[1] - np.einsum("ij,ij->j", Kt, w)
    np.testing.assert_allclose(m, mean, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(v, var, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(vl, var - THETA[1], rtol=1e-9, atol=1e-12)
