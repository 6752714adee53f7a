"""Gradient of the Block Vecchia log-likelihood with respect to theta, FP64
(test infrastructure only).

The paper evaluates the likelihood and hands gradient information to the
optimiser (Sec. 6) without printing it; this module writes out the
textbook derivative of a Gaussian log-density for the block conditional of
Alg. 5.  Block i's term is the difference of two Gaussian log-densities,

    l_i = log N(y_S; 0, Sigma_SS) - log N(y_J; 0, Sigma_JJ),   S = J u B_i,

and for either system, with x = Sigma^{-1} y,

    d/dtheta_k log N(y; 0, Sigma) = 1/2 x^T (dSigma/dtheta_k) x
                                    - 1/2 tr(Sigma^{-1} dSigma/dtheta_k).

theta = (sigma^2, tau^2, beta_1 .. beta_d) (natural parameters, not logs).
With r = |(x_a - x_b) / beta| (Eq. maternkernel, no sqrt(2 nu)) and
K = sigma^2 M_nu(r) + tau^2 [a is b]:

    dK/dsigma^2 = M_nu(r)
    dK/dtau^2   = [a is b]
    dK/dbeta_t  = sigma^2 M_nu'(r) dr/dbeta_t,  dr/dbeta_t = -u_t^2 / (beta_t r),
                  u_t = (x_at - x_bt) / beta_t,

so dK/dbeta_t = sigma^2 h_nu(r) u_t^2 / beta_t with h_nu(r) = -M_nu'(r) / r:

    nu = 1/2:  h = exp(-r) / r          (pairs at r = 0 contribute 0: u = 0)
    nu = 3/2:  h = exp(-r)
    nu = 5/2:  h = (1 + r) exp(-r) / 3
    nu = 7/2:  h = (3 + 3 r + r^2) exp(-r) / 15

(from M' of the closed forms: -e^-r; -r e^-r; -r (1 + r) e^-r / 3;
-r (3 + 3r + r^2) e^-r / 15), and for any other nu = nu2/2 (nu >= 1)
h = 2^(1-nu)/Gamma(nu) r^(nu-1) K_(nu-1)(r) from the Bessel-function
derivative d/dr [r^nu K_nu(r)] = -r^nu K_(nu-1)(r).  Dense inverses and traces, one block at a time;
pinned by central differences of oracle.sbv.block_loglik, by the closed form
of dl/dsigma^2 at tau^2 = 0, and by additivity over blocks.
"""
from __future__ import annotations

import numpy as np
from scipy import special

from . import sbv


def h_nu(r: np.ndarray, nu2: int) -> np.ndarray:
    """-M_nu'(r) / r for nu = nu2 / 2 (0 where r = 0 for nu = 1/2).

    Other 2 <= nu2 <= 40: from d/dr [r^nu K_nu(r)] = -r^nu K_(nu-1)(r),
    -M'(r)/r = 2^(1-nu)/Gamma(nu) r^(nu-1) K_(nu-1)(r) (scipy's K), with its
    r -> 0 limit 1/(2 (nu - 1)) for nu > 1 and 0 at r = 0 for nu = 1 (where
    it multiplies u_t^2 = 0)."""
    e = np.exp(-r)
    if nu2 == 1:
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(r > 0, e / np.where(r > 0, r, 1.0), 0.0)
    if nu2 == 3:
        return e
    if nu2 == 5:
        return (1.0 + r) * e / 3.0
    if nu2 == 7:
        return (3.0 + 3.0 * r + r * r) * e / 15.0
    if 2 <= nu2 <= 40:
        nu = nu2 / 2.0
        r = np.asarray(r, dtype=np.float64)
        out = np.full_like(r, 0.5 / (nu - 1.0) if nu > 1.0 else 0.0)
        pos = r > 0
        rp = r[pos]
        out[pos] = 2.0 ** (1.0 - nu) / special.gamma(nu) * rp ** (nu - 1.0) * special.kv(abs(nu - 1.0), rp)
        return out
    raise ValueError("nu2 must be an integer in [1, 40]")


def cov_derivatives(X, idx, theta, nu2: int) -> list[np.ndarray]:
    """dSigma/dtheta_k for k = sigma^2, tau^2, beta_1..beta_d over the points idx."""
    theta = np.asarray(theta, dtype=np.float64)
    s2, beta = theta[0], theta[2:]
    U = np.asarray(X, dtype=np.float64)[idx] / beta[None, :]
    diff = U[:, None, :] - U[None, :, :]                 # u_t for every pair
    r = np.sqrt(np.sum(diff * diff, axis=2))
    same = (np.asarray(idx)[:, None] == np.asarray(idx)[None, :]).astype(np.float64)
    out = [sbv.matern(r, nu2), same]
    h = h_nu(r, nu2)
    for t in range(beta.size):
        out.append(s2 * h * diff[:, :, t] ** 2 / beta[t])
    return out


def gaussian_loglik_grad(S: np.ndarray, y: np.ndarray, dS: list[np.ndarray]) -> np.ndarray:
    """d/dtheta_k log N(y; 0, S) = 1/2 x^T dS_k x - 1/2 tr(S^{-1} dS_k), x = S^{-1} y."""
    Si = np.linalg.inv(S)
    x = Si @ y
    return np.array([0.5 * x @ D @ x - 0.5 * np.sum(Si * D) for D in dS])   # S^{-1}, D symmetric


def block_grad(X, y, J, Bpts, theta, nu2: int) -> np.ndarray:
    """d l_i / d theta for one block: joint system minus the J system."""
    J = np.asarray(J, dtype=np.int64)
    Bpts = np.asarray(Bpts, dtype=np.int64)
    idx = np.concatenate([J, Bpts])
    g = gaussian_loglik_grad(sbv.cov_points(X, idx, idx, theta, nu2), y[idx],
                             cov_derivatives(X, idx, theta, nu2))
    if J.size:
        g = g - gaussian_loglik_grad(sbv.cov_points(X, J, J, theta, nu2), y[J],
                                     cov_derivatives(X, J, theta, nu2))
    return g


def grad_terms(X, y, ptr, pts, nbr, cnt, theta, nu2: int, blocks=None) -> np.ndarray:
    """Per-block gradients (len(blocks) x (2 + d)), default all blocks."""
    bc = len(ptr) - 1
    blocks = np.arange(bc) if blocks is None else np.asarray(blocks)
    d = np.asarray(theta).size - 2
    out = np.empty((blocks.size, 2 + d))
    for i, b in enumerate(blocks):
        out[i] = block_grad(X, y, nbr[b, :cnt[b]], pts[ptr[b]:ptr[b + 1]], theta, nu2)
    return out
