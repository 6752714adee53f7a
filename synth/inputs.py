"""Seeded synthetic inputs for Scaled Block Vecchia workloads.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no scaling, blocking, neighbour search, covariance or
likelihood).  Both the oracle tests and the CUDA path read their inputs from
here, so the two sides always see bit-identical data.

Workloads (each named by what it is, with its sizes):

* ``gp5d``     -- n=4,000 points uniform on [0,1]^5; y is an exact draw of a
  zero-mean Matern-5/2 GP (the draw itself needs the covariance, so this module
  returns the standard-normal vector and the caller multiplies by the Cholesky
  factor of its own covariance).  sigma^2=1, beta=(.05,.1,.2,.5,1), tau^2=1e-4,
  400 blocks, m=60, 500 uniform test points.  Follows the exact-GP-draw design
  of the paper's synthetic study (Sec. 7.1) at d=5.
* ``sine10d``  -- n=1,000,000 points uniform on [0,1]^10, y from the sine-sum
  family below with noise N(0, .05^2); 20,000 blocks, m=120.  The shape of the
  paper's performance workload (Sec. 8: d=10 on [0,1]^10).
* ``sine20d``  -- n=2,000,000 on [0,1]^20, same family at d=20; 40,000 blocks,
  m=200, 64 parameter candidates with ranges log-uniform on [0.05, 2].
* ``sine10d_50m`` -- n=50,000,000 on [0,1]^10 stored as float32 (the 50M-sample
  size of the paper's MetaRVM study, Sec. 7.3); 1,000,000 blocks, m=300,
  1,000,000 test points.

Sine-sum family:  y(x) = sum_j a_j sin(2 pi x_j / b_j) + 0.5 x_1 x_2 + eps,
a_j = 1/j, b = linspace(0.1, 1.0, d), eps ~ N(0, 0.05^2).
"""
from __future__ import annotations

import numpy as np

SINE_NOISE_SD = 0.05


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_points(n: int, d: int, seed: int, dtype=np.float64) -> np.ndarray:
    """n x d row-major points, uniform on [0,1]^d."""
    x = _rng(seed).random((n, d))
    return np.ascontiguousarray(x.astype(dtype))


def sine_ranges(d: int) -> np.ndarray:
    """Range vector b of the sine-sum family: linspace(0.1, 1.0, d)."""
    return np.linspace(0.1, 1.0, d)


def sine_sum_response(x: np.ndarray, seed: int) -> np.ndarray:
    """y = sum_j (1/j) sin(2 pi x_j / b_j) + 0.5 x_1 x_2 + N(0, 0.05^2) noise."""
    n, d = x.shape
    xd = x.astype(np.float64)
    b = sine_ranges(d)
    y = np.zeros(n)
    for j in range(d):
        y += (1.0 / (j + 1)) * np.sin(2.0 * np.pi * xd[:, j] / b[j])
    y += 0.5 * xd[:, 0] * xd[:, 1]
    y += SINE_NOISE_SD * _rng(seed + 7).standard_normal(n)
    return y


def standard_normal(n: int, seed: int) -> np.ndarray:
    return _rng(seed).standard_normal(n)


def loguniform_candidates(B: int, d: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """B x d ranges drawn log-uniformly on [lo, hi]."""
    u = _rng(seed).random((B, d))
    return np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))


def theta_rows(sigma2, tau2, betas) -> np.ndarray:
    """Pack parameter candidates as rows (sigma^2, tau^2, beta_1..beta_d)."""
    betas = np.atleast_2d(np.asarray(betas, dtype=np.float64))
    B = betas.shape[0]
    s = np.broadcast_to(np.asarray(sigma2, dtype=np.float64), (B,))
    t = np.broadcast_to(np.asarray(tau2, dtype=np.float64), (B,))
    return np.ascontiguousarray(np.column_stack([s, t, betas]))


WORKLOADS = {
    "gp5d": dict(n=4000, d=5, bc=400, m=60, ntest=500, m_pred=60, nu2=5,
                 sigma2=1.0, tau2=1e-4, beta=(0.05, 0.1, 0.2, 0.5, 1.0),
                 seed=1000, xdtype="f64", response="gp"),
    "sine10d": dict(n=1_000_000, d=10, bc=20_000, m=120, ntest=0, m_pred=0, nu2=5,
                    sigma2=1.0, tau2=0.0025, beta=None, seed=1001, xdtype="f64",
                    response="sine"),
    "sine20d": dict(n=2_000_000, d=20, bc=40_000, m=200, ntest=0, m_pred=0, nu2=5,
                    sigma2=1.0, tau2=0.0025, beta=None, seed=1002, xdtype="f64",
                    response="sine", B=64),
    "sine10d_50m": dict(n=50_000_000, d=10, bc=1_000_000, m=300, ntest=1_000_000,
                        m_pred=300, nu2=5, sigma2=1.0, tau2=0.0025, beta=None,
                        seed=1004, xdtype="f32", response="sine"),
}


def workload(name: str, n: int | None = None, bc: int | None = None,
             m: int | None = None, ntest: int | None = None, d: int | None = None):
    """Materialise a named workload (optionally shrunk: n, bc, m, ntest, d).

    Returns a dict with X (n x d), y (n, or None for the GP draw), beta_scale,
    theta (B x (2+d) rows), Xtest, z (standard normals for a GP draw) and the
    structural sizes.  The blocking uses beta_scale = the generating ranges.
    """
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = n
    if bc is not None:
        w["bc"] = bc
    if m is not None:
        w["m"] = m
    if ntest is not None:
        w["ntest"] = ntest
    if d is not None:
        w["d"] = d
    n_, d_ = w["n"], w["d"]
    dt = np.float32 if w["xdtype"] == "f32" else np.float64
    X = uniform_points(n_, d_, w["seed"], dt)
    if w["response"] == "gp":
        beta = np.asarray(w["beta"], dtype=np.float64)[:d_]
        y = None
        z = standard_normal(n_, w["seed"] + 1)
    else:
        beta = sine_ranges(d_)
        y = sine_sum_response(X, w["seed"])
        z = None
    if "B" in w:
        bet = loguniform_candidates(w["B"], d_, 0.05, 2.0, w["seed"] + 3)
        theta = theta_rows(w["sigma2"], w["tau2"], bet)
    else:
        theta = theta_rows(w["sigma2"], w["tau2"], beta[None, :])
    Xtest = uniform_points(w["ntest"], d_, w["seed"] + 2, dt) if w["ntest"] else None
    out = dict(w)
    out.update(X=X, y=y, z=z, beta_scale=beta.copy(), theta=theta, Xtest=Xtest)
    return out
