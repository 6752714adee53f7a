"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

None of these re-types an oracle formula: each compares the oracle with an
independent route (a different factorisation, a closed form, a library special
function, brute force written another way, a published test vector).
"""
import math
from pathlib import Path

import numpy as np
import pytest
from scipy.special import gamma, kv

from oracle import prng, sbv
from synth.inputs import uniform_points, standard_normal

GOLDEN = Path(__file__).parent / "golden"


def dense_loglik(X, y, theta, nu2):
    """Eq. (1) by LU (slogdet + solve), a different route than Cholesky."""
    n = len(y)
    idx = np.arange(n)
    S = sbv.cov_points(X, idx, idx, theta, nu2)
    sign, logdet = np.linalg.slogdet(S)
    assert sign > 0
    return -0.5 * n * math.log(2 * math.pi) - 0.5 * logdet - 0.5 * y @ np.linalg.solve(S, y)


def small_problem(n=60, d=3, seed=5, tau2=1e-2):
    X = uniform_points(n, d, seed)
    y = standard_normal(n, seed + 1)
    theta = np.array([1.3, tau2] + [0.3 + 0.2 * t for t in range(d)])
    return X, y, theta


# ---------------------------------------------------------------- generator
def test_splitmix64_published_vector():
    want = [int(l) for l in (GOLDEN / "splitmix64_seed1234567.txt").read_text().split("\n")
            if l and not l.startswith("#")]
    r = prng.SplitMix64(1234567)
    assert [r.next() for _ in range(5)] == want


def test_lemire_power_of_two_is_top_bits():
    # for s = 2^k no draw is rejected ((2^64 - s) mod s = 0) and the result is the top k bits
    for k in (1, 5, 17, 40):
        a, b = prng.SplitMix64(99), prng.SplitMix64(99)
        for _ in range(50):
            assert a.below(1 << k) == b.next() >> (64 - k)


def test_lemire_rejection_threshold():
    # s = 3: (2^64 - 3) mod 3 = 1, so only a low word of 0 is rejected.
    class Fixed(prng.SplitMix64):
        def __init__(self, seq):
            self.seq = list(seq)

        def next(self):
            return self.seq.pop(0)
    # x = 0 -> low word 0 < t = 1 -> rejected, next x = 2^63 -> 3 * 2^63 = 2^64 + 2^63 -> high word 1
    r = Fixed([0, 1 << 63])
    assert r.below(3) == 1 and r.seq == []
    # brute force: every x with a non-rejected low word maps to x*s >> 64
    s = 7
    t = ((1 << 64) - s) % s
    for x in [1, 12345, (1 << 64) - 1, 3 << 61]:
        r = Fixed([x])
        if (x * s) & ((1 << 64) - 1) >= t:
            assert r.below(s) == (x * s) >> 64


def test_fisher_yates_is_bijection_and_prefix_consistent():
    a = prng.full_shuffle(1000, prng.SplitMix64(3))
    assert sorted(a) == list(range(1000))
    p = prng.partial_shuffle_prefix(1000, 37, prng.SplitMix64(3))
    assert p == a[:37]


# ---------------------------------------------------------------- kernel
@pytest.mark.parametrize("nu2", [1, 3, 5, 7])
def test_matern_closed_form_equals_bessel(nu2):
    nu = nu2 / 2
    r = np.linspace(1e-3, 12.0, 400)
    bessel = 2 ** (1 - nu) / gamma(nu) * r ** nu * kv(nu, r)
    np.testing.assert_allclose(sbv.matern(r, nu2), bessel, rtol=1e-12, atol=1e-300)
    assert sbv.matern(np.array([0.0]), nu2)[0] == 1.0


def test_cov_scaled_distance_against_loop():
    X = uniform_points(5, 4, 11)
    th = np.array([2.0, 0.1, 0.5, 1.0, 2.0, 4.0])
    K = sbv.cov_points(X, np.arange(5), np.arange(5), th, 3)
    for a in range(5):
        for b in range(5):
            r = math.sqrt(sum(((X[a, t] - X[b, t]) / th[2 + t]) ** 2 for t in range(4)))
            want = 2.0 * (1 + r) * math.exp(-r) + (0.1 if a == b else 0.0)
            assert abs(K[a, b] - want) < 1e-14


# ---------------------------------------------------------------- likelihood
def blocks_of(labels):
    labels = np.asarray(labels)
    k = labels.max() + 1
    counts = np.bincount(labels, minlength=k)
    ptr = np.concatenate([[0], np.cumsum(counts)])
    pts = np.argsort(labels, kind="stable")
    return ptr, pts


def exact_neighbours(n_blocks, ptr, pts, rank):
    """NN sets = every point of every earlier block (m >= n - 1)."""
    m = int(ptr[-1])
    nbr = np.full((n_blocks, m), -1)
    cnt = np.zeros(n_blocks, dtype=np.int64)
    for b in range(n_blocks):
        J = np.concatenate([pts[ptr[c]:ptr[c + 1]] for c in range(n_blocks) if rank[c] < rank[b]]
                           + [np.zeros(0, dtype=np.int64)])
        nbr[b, :J.size] = np.sort(J)
        cnt[b] = J.size
    return nbr, cnt


def test_one_block_is_exact_gp():
    X, y, th = small_problem()
    n = len(y)
    ptr, pts = np.array([0, n]), np.arange(n)
    nbr, cnt = np.full((1, 1), -1), np.array([0])
    got = sbv.loglik(X, y, ptr, pts, nbr, cnt, np.array([0]), th, 5)
    assert abs(got - dense_loglik(X, y, th, 5)) < 1e-9


@pytest.mark.parametrize("nu2", [1, 5, 7])
def test_full_conditioning_is_exact_gp(nu2):
    # chain rule: with every earlier point as neighbour the product is exact (Sec. 4.2)
    X, y, th = small_problem(n=48, d=2, seed=8)
    labels = np.arange(48) % 6
    ptr, pts = blocks_of(labels)
    rank = np.array([3, 0, 5, 1, 4, 2])
    nbr, cnt = exact_neighbours(6, ptr, pts, rank)
    got = sbv.loglik(X, y, ptr, pts, nbr, cnt, rank, th, nu2)
    assert abs(got - dense_loglik(X, y, th, nu2)) < 1e-9


def test_singleton_blocks_without_neighbours():
    X, y, th = small_problem(n=30)
    ptr, pts = np.arange(31), np.arange(30)
    nbr, cnt = np.full((30, 1), -1), np.zeros(30, dtype=np.int64)
    got = sbv.loglik(X, y, ptr, pts, nbr, cnt, np.arange(30), th, 5)
    v = th[0] + th[1]
    want = sum(-0.5 * (math.log(2 * math.pi * v) + yi * yi / v) for yi in y)
    assert abs(got - want) < 1e-11


def joint_term(X, y, J, B, th, nu2):
    """Joint Cholesky of [J; B] with y bordered: a second formulation of Alg. 5."""
    P = np.concatenate([J, B])
    S = sbv.cov_points(X, P, P, th, nu2)
    M = np.zeros((P.size + 1, P.size + 1))
    M[:-1, :-1] = S
    M[-1, :-1] = y[P]
    M[:-1, -1] = y[P]
    M[-1, -1] = y[P] @ np.linalg.solve(S, y[P]) + 1.0  # any value keeping M positive definite
    L = np.linalg.cholesky(M)
    m = J.size
    w = L[-1, :-1]
    return -0.5 * (B.size * math.log(2 * math.pi) + 2 * np.sum(np.log(np.diag(L)[m:-1]))
                   + np.sum(w[m:] ** 2))


def test_alg5_matches_joint_factorisation():
    X, y, th = small_problem(n=80, d=3, seed=21, tau2=1e-3)
    rng = np.random.default_rng(0)
    for _ in range(10):
        perm = rng.permutation(80)
        J, B = perm[:25], perm[25:33]
        a = sbv.block_loglik(X, y, J, B, th, 5)
        b = joint_term(X, y, J, B, th, 5)
        assert abs(a - b) < 1e-9 * max(1, abs(a))


def test_block_term_permutation_invariance():
    X, y, th = small_problem(n=60, d=3, seed=4)
    J, B = np.arange(0, 30), np.arange(30, 38)
    ref = sbv.block_loglik(X, y, J, B, th, 5)
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = sbv.block_loglik(X, y, rng.permutation(J), rng.permutation(B), th, 5)
        assert abs(a - ref) < 1e-12 * max(1.0, abs(ref))


def test_kl_nonnegative_and_monotone_in_m():
    # D_KL = l_exact(theta; 0) - l_approx(theta; 0) >= 0, non-increasing for nested NN sets
    X, _, th = small_problem(n=120, d=2, seed=9, tau2=1e-3)
    y0 = np.zeros(120)
    exact = dense_loglik(X, y0, th, 5)
    blk = sbv.blocking(X, np.array([0.3, 0.5]), 24, 3, 2)
    prev = None
    for m in (0, 5, 10, 20, 40):
        nbr, cnt = sbv.knn(blk["Z"], blk["blk"], blk["rank"], blk["centres"], m)
        nb = np.zeros((len(cnt), max(m, 1)), dtype=np.int64) - 1
        nb[:, :m] = nbr
        ll = sbv.loglik(X, y0, blk["ptr"], blk["pts"], nb, cnt, blk["rank"], th, 5)
        kl = exact - ll
        assert kl >= -1e-9
        if prev is not None:
            assert kl <= prev + 1e-9
        prev = kl


# ---------------------------------------------------------------- blocking and kNN
def test_blocking_invariants():
    X = uniform_points(500, 3, 17)
    beta = np.array([0.2, 0.5, 1.0])
    for T in (0, 4):
        b = sbv.blocking(X, beta, 40, T, 123)
        Z = X / beta
        k = b["bc_eff"]
        assert sorted(b["rank"]) == list(range(k))
        assert b["ptr"][-1] == 500 and np.all(np.diff(b["ptr"]) > 0)
        for j in range(k):
            mem = b["pts"][b["ptr"][j]:b["ptr"][j + 1]]
            assert np.all(b["blk"][mem] == j) and np.all(np.diff(mem) > 0)
            s = np.zeros(3)
            for i in mem:  # plain sequential mean
                s = s + Z[i]
            assert np.array_equal(s / mem.size, b["centres"][j])
    # T = 0 is RAC: every point sits with its nearest anchor (the anchors are data points)
    b0 = sbv.blocking(X, beta, 40, 0, 123)
    anchors = prng.partial_shuffle_prefix(500, 40, prng.SplitMix64(123))
    Za = Z[np.asarray(anchors)]
    for i in range(0, 500, 7):
        D = [sum((Z[i, t] - Za[j, t]) ** 2 for t in range(3)) for j in range(40)]
        jbest = int(np.argmin(D))
        # compacted ids preserve order; anchors keep their own (non-empty) block
        assert b0["blk"][i] == jbest


def test_converged_kmeans_assigns_each_point_to_nearest_centre():
    X = uniform_points(400, 2, 3)
    beta = np.array([1.0, 0.5])
    b = sbv.blocking(X, beta, 20, 100, 5)
    Z = X / beta
    for i in range(400):
        D = [sum((Z[i, t] - b["centres"][j, t]) ** 2 for t in range(2)) for j in range(b["bc_eff"])]
        assert b["blk"][i] == int(np.argmin(D))


def brute_knn(Z, c, cand, m):
    """Pure-Python loop, distances summed left to right, sorted by (D, index)."""
    keys = []
    for k in cand:
        D = 0.0
        for t in range(Z.shape[1]):
            df = float(Z[k, t]) - float(c[t])
            D = D + df * df
        keys.append((D, int(k)))
    keys.sort()
    return [k for _, k in keys[:m]]


def test_knn_matches_brute_force_with_ties():
    # integer-valued coordinates force many equal distances: ties go to the smaller index
    rng = np.random.default_rng(7)
    X = rng.integers(0, 4, size=(200, 2)).astype(np.float64)
    b = sbv.blocking(X, np.array([1.0, 1.0]), 30, 2, 11)
    nbr, cnt = sbv.knn(b["Z"], b["blk"], b["rank"], b["centres"], 12)
    prank = b["rank"][b["blk"]]
    for j in range(b["bc_eff"]):
        cand = [k for k in range(200) if prank[k] < b["rank"][j]]
        want = brute_knn(b["Z"], b["centres"][j], cand, 12)
        assert list(nbr[j, :cnt[j]]) == want
        assert cnt[j] == min(12, len(cand))


# ---------------------------------------------------------------- prediction
def test_prediction_with_all_neighbours_is_exact_conditional():
    X, y, th = small_problem(n=50, d=2, seed=13, tau2=1e-2)
    Xt = uniform_points(6, 2, 14)
    mean, var, var_lat, _ = sbv.predict(X, y, Xt, np.array([1.0, 1.0]), 50, th, 5)
    idx = np.arange(50)
    S = sbv.cov_points(X, idx, idx, th, 5)
    for j in range(6):
        k = sbv.cov(X, Xt[j:j + 1], th, 5)[:, 0]
        mu = k @ np.linalg.solve(S, y)
        v = th[0] + th[1] - k @ np.linalg.solve(S, k)
        assert abs(mean[j] - mu) < 1e-9
        assert abs(var[j] - v) < 1e-9
        assert abs(var_lat[j] - (v - th[1])) < 1e-12


def test_prediction_interpolates_without_nugget():
    X, y, th = small_problem(n=40, d=2, seed=15, tau2=0.0)
    th[1] = 0.0
    Xt = X[[3, 17]].copy()
    mean, var, _, _ = sbv.predict(X, y, Xt, np.array([1.0, 1.0]), 10, th, 5)
    assert np.allclose(mean, y[[3, 17]], atol=1e-6)
    assert np.all(np.abs(var) < 1e-6)


def test_matern_bessel_form_general_nu():
    """Eq. maternkernel through the Bessel function K_nu (any nu = nu2/2):
    equal to the closed forms at the half-integers, to a direct quadrature of
    the defining integral K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt at
    integer nu, 1 at r = 0 and decreasing in r."""
    from scipy import integrate
    r = np.array([1e-6, 0.05, 0.3, 1.0, 2.5, 7.0])
    for nu2 in (1, 3, 5, 7):
        assert np.allclose(sbv.matern_bessel(r, nu2 / 2), sbv.matern(r, nu2), rtol=1e-12, atol=0)
    for nu2 in (2, 4):
        nu = nu2 / 2
        for x in r[1:]:
            # beyond t_max the integrand is below exp(-800 + nu t_max) ~ 0
            t_max = math.acosh(800.0 / x)
            K, _ = integrate.quad(lambda t: math.exp(-x * math.cosh(t)) * math.cosh(nu * t), 0, t_max,
                                  epsabs=0, epsrel=1e-13, limit=400)
            want = 2 ** (1 - nu) / math.gamma(nu) * x ** nu * K
            assert sbv.matern(np.array([x]), nu2)[0] == pytest.approx(want, rel=1e-10)
    for nu2 in (2, 4, 9, 20):
        m = sbv.matern(np.concatenate([[0.0], r]), nu2)
        assert m[0] == 1.0 and np.all(np.diff(m) < 0) and m[1] == pytest.approx(1.0, abs=1e-9)
    with pytest.raises(ValueError):
        sbv.matern(r, 41)
