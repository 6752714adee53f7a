"""Conditional simulation at the test points (Sec. 5.5) -- oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 5.5: the predictive mean mu_j and variance sigma_j (the diagonal of
Sigma^new) of every test point define N(mu_j, sigma_j); 1000 samples are drawn
from it, their sample mean and sample variance are computed, and the 95 %
interval is the sample mean -/+ z_{alpha/2} times the sample standard
deviation, alpha = 0.05.

The draws need random numbers that the GPU can reproduce one by one, so both
sides implement the same counter-based generator from its published
definition: Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC 2011, Sec. 4 and Table 2), then the
Box-Muller transform (Box & Muller, Ann. Math. Stat. 29, 1958).  Draw k of
test point j (counted from index_base) comes from the output block of
counter (k // 4, index_base + j, 0, 0) under
key (seed, 0): words 2p, 2p + 1 (p = (k % 4) // 2) give u1, u2 in (0, 1) and
z = sqrt(-2 ln u1) cos(2 pi u2) for even k, sqrt(-2 ln u1) sin(2 pi u2) for odd k.

Pins (tests/test_oracle_simulate.py): the block function equals numpy's
independent Philox implementation word for word; the normals pass a
Kolmogorov-Smirnov test against the normal law; standardised sample means are
N(0, 1) over many test points; the interval covers fresh draws at 95 % within
binomial bounds; z_{0.975} equals scipy's normal quantile.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15   # golden ratio
W1 = 0xBB67AE8584CAA73B   # sqrt(3) - 1
MASK = (1 << 64) - 1
Z975 = 1.959963984540054  # 0.975 quantile of the standard normal


def philox4x64(counter, key, rounds: int = 10) -> list[int]:
    """One Philox4x64 block: four 64-bit words from a 4-word counter and a
    2-word key.  Each round multiplies words 0 and 2 by M0, M1 into 128-bit
    products (hi, lo), outputs (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), and
    the key advances by the Weyl constants (W0, W1) between rounds."""
    c = [int(v) & MASK for v in counter]
    k0, k1 = int(key[0]) & MASK, int(key[1]) & MASK
    for _ in range(rounds):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> 64, p0 & MASK
        hi1, lo1 = p1 >> 64, p1 & MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return c


def unit_open(w: int) -> float:
    """A 64-bit word to a double in (0, 1): the top 52 bits, centred (exact in
    FP64, so neither 0 nor 1 can occur)."""
    return ((w >> 12) + 0.5) * 2.0 ** -52


def std_normals(j: int, ndraws: int, seed: int) -> np.ndarray:
    """The ndraws standard normal draws of test point j."""
    z = np.empty(ndraws)
    for b in range((ndraws + 3) // 4):
        w = philox4x64((b, j, 0, 0), (seed, 0))
        for p in range(2):
            u1, u2 = unit_open(w[2 * p]), unit_open(w[2 * p + 1])
            r = np.sqrt(-2.0 * np.log(u1))
            for q, v in ((0, r * np.cos(2.0 * np.pi * u2)), (1, r * np.sin(2.0 * np.pi * u2))):
                k = 4 * b + 2 * p + q
                if k < ndraws:
                    z[k] = v
    return z


def simulate(mean, var, ndraws: int, seed: int, rows=None, index_base: int = 0):
    """Sec. 5.5 for the test points `rows` (default: all): returns the draws
    (len(rows) x ndraws), sample means, sample variances (divisor ndraws - 1)
    and the interval ends."""
    mean = np.asarray(mean, dtype=np.float64)
    var = np.asarray(var, dtype=np.float64)
    rows = np.arange(mean.size) if rows is None else np.asarray(rows)
    draws = np.empty((rows.size, ndraws))
    for i, j in enumerate(rows):
        draws[i] = mean[j] + np.sqrt(var[j]) * std_normals(index_base + int(j), ndraws, seed)
    mu = draws.mean(axis=1)
    s2 = ((draws - mu[:, None]) ** 2).sum(axis=1) / (ndraws - 1)
    h = Z975 * np.sqrt(s2)
    return draws, mu, s2, mu - h, mu + h
