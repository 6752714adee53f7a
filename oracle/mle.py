"""Maximum-likelihood estimation with the oracle likelihood (test infrastructure only).

The paper fits theta by maximising the SBV log-likelihood with NLopt for a
fixed budget of iterations (Sec. 7: 500), keeping the data resident and
re-evaluating Alg. 5 once per iteration; it does not name the algorithm.
Reading adopted for the oracle: maximise l(exp(u)) over the free components
of u = log theta inside box bounds, with scipy's L-BFGS-B (a library
optimiser serves as a step) and central-difference gradients.  What is pinned
is the optimum, not the path: the scale-family closed form below, and
stationarity at the returned point.

Closed form used as a pin (Eq. 1 with tau^2 = 0): every block covariance is
sigma^2 R with R fixed by the ranges, so
    l(sigma^2) = -1/2 [n log 2 pi + n log sigma^2 + LD + Q / sigma^2],
maximised at sigma^2 = Q / n, and Q follows from two evaluations:
    Q = 2 n log 2 - 4 (l(1) - l(2)).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import minimize

from . import sbv


def make_loglik(X, y, ptr, pts, nbr, cnt, rank, nu2: int):
    """theta -> l(theta) on a fixed structure (Alg. 1 Step 5 over Alg. 5)."""
    def f(theta):
        try:
            return sbv.loglik(X, y, ptr, pts, nbr, cnt, rank, np.asarray(theta, dtype=np.float64), nu2)
        except np.linalg.LinAlgError:
            return -np.inf
    return f


def mle(f, theta0, free=None, lower=None, upper=None, h: float = 1e-5, maxiter: int = 200):
    """Maximise f(theta) over log theta; returns (theta_hat, f(theta_hat), evaluations)."""
    theta0 = np.asarray(theta0, dtype=np.float64)
    p = len(theta0)
    free = np.ones(p, bool) if free is None else np.asarray(free, bool)
    idx = np.flatnonzero(free)
    u0 = np.log(theta0[idx])          # fixed entries (possibly tau^2 = 0) stay as given
    lo = np.full(len(idx), -np.inf) if lower is None else np.log(np.asarray(lower, dtype=np.float64)[idx])
    hi = np.full(len(idx), np.inf) if upper is None else np.log(np.asarray(upper, dtype=np.float64)[idx])
    count = [0]

    def full(v):
        th = theta0.copy()
        th[idx] = np.exp(v)
        return th

    def neg(v):
        count[0] += 1
        val = f(full(v))
        return 1e300 if not np.isfinite(val) else -val

    def grad(v):
        g = np.empty(len(v))
        for j in range(len(v)):
            e = np.zeros(len(v))
            e[j] = h
            g[j] = (neg(v + e) - neg(v - e)) / (2 * h)
        return g

    res = minimize(neg, u0, jac=grad, method="L-BFGS-B", bounds=list(zip(lo, hi)),
                   options=dict(maxiter=maxiter, ftol=1e-13, gtol=1e-7))
    return full(res.x), -res.fun, count[0]


def sigma2_closed_form(f, theta, n: int) -> float:
    """Maximiser of l over sigma^2 alone at tau^2 = 0 (see the module docstring)."""
    t1 = np.array(theta, dtype=np.float64)
    t1[0], t1[1] = 1.0, 0.0
    t2 = t1.copy()
    t2[0] = 2.0
    Q = 2.0 * n * math.log(2.0) - 4.0 * (f(t1) - f(t2))
    return Q / n
