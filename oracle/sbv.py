"""Scaled Block Vecchia, step by step in FP64 (test infrastructure only).

Every function follows one passage of arxiv 2504.12004 and is written for a
reader checking it against the paper, not for speed.  Readings taken where the
paper is silent or garbled are stated at the function that uses them.

Distances used for decisions (cluster assignment, neighbour ranking) are fixed
bit for bit: D(a, c) = sum over t = 0..d-1, left to right, of (a_t - c_t)^2,
every difference, product and sum rounded on its own (numpy elementwise
operations never fuse a multiply into an add), ties broken by the smaller
index.  Means are sums in increasing point index followed by one division.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special
from scipy.linalg import solve_triangular

from .prng import SplitMix64, full_shuffle, partial_shuffle_prefix

LOG2PI = math.log(2.0 * math.pi)


# --------------------------------------------------------------------------
# Scaling (Alg. 2, dimension scaling X_j := X^org_j / beta_j)
# --------------------------------------------------------------------------
def scale(X: np.ndarray, beta_scale) -> np.ndarray:
    """z_ij = x_ij / beta_j in FP64 (float32 inputs are widened exactly first)."""
    return np.asarray(X, dtype=np.float64) / np.asarray(beta_scale, dtype=np.float64)[None, :]


def sq_dist_rows(Z: np.ndarray, c: np.ndarray) -> np.ndarray:
    """D(z_k, c) for every row k, dimensions summed left to right."""
    diff = Z[:, 0] - c[0]
    D = diff * diff
    for t in range(1, Z.shape[1]):
        diff = Z[:, t] - c[t]
        D = D + diff * diff
    return D


# --------------------------------------------------------------------------
# Random Anchor Clustering + Lloyd iterations (Alg. 3; K-means of Sec. 5.2)
# --------------------------------------------------------------------------
def assign(Z: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Alg. 3 assignment: block of each point = argmin_j ||z - c_j||^2, ties to the smaller j."""
    n = Z.shape[0]
    best = np.full(n, np.inf)
    arg = np.zeros(n, dtype=np.int64)
    for j in range(C.shape[0]):
        D = sq_dist_rows(Z, C[j])
        better = D < best
        best = np.where(better, D, best)
        arg = np.where(better, j, arg)
    return arg


def centroids(Z: np.ndarray, blk: np.ndarray, k: int, prev: np.ndarray | None = None) -> np.ndarray:
    """Mean of each block's members (Alg. 4 centre update).

    Members are summed one at a time in increasing point index, then divided by
    the count.  A block with no members keeps its previous centre.
    """
    n, d = Z.shape
    order = np.argsort(blk, kind="stable")          # by block, then point index
    counts = np.bincount(blk, minlength=k)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    acc = np.zeros((k, d))
    for s in range(int(counts.max()) if n else 0):
        has = counts > s
        idx = order[starts[has] + s]
        acc[has] = acc[has] + Z[idx]
    C = np.empty((k, d))
    nz = counts > 0
    C[nz] = acc[nz] / counts[nz][:, None]
    if prev is not None:
        C[~nz] = prev[~nz]
    else:
        C[~nz] = np.nan
    return C


def slabs(X, beta_scale, P: int):
    """Alg. 2: slab of each point along d_max = argmax_j 1/beta_j.

    The slab index is int(x_dmax * P) on the unscaled coordinate (FP64
    product, then floor), clamped to [0, P-1] for points outside [0, 1);
    ties in 1/beta go to the first dimension.
    """
    beta = np.asarray(beta_scale, dtype=np.float64)
    dmax = int(np.argmax(1.0 / beta))
    x = np.asarray(X, dtype=np.float64)[:, dmax]
    q = np.floor(x * float(P))
    return np.clip(q, 0, P - 1).astype(np.int64), dmax


def slab_quota(counts, bc: int) -> np.ndarray:
    """Anchors per slab (Alg. 3 chooses k_p per partition; the paper does not
    say how many).  Reading: one anchor for every non-empty slab, the other
    bc - (#non-empty) shared in proportion to the slab sizes by the largest
    remainder method (exact integers; ties to the lower slab), and never more
    anchors than points in a slab."""
    counts = [int(c) for c in counts]
    n = sum(counts)
    k = [1 if c > 0 else 0 for c in counts]
    R = max(bc - sum(k), 0)
    base = [R * c // n for c in counts]
    rem = [R * c % n for c in counts]
    extra = R - sum(base)
    order = sorted(range(len(counts)), key=lambda q: (-rem[q], q))
    for q in range(len(counts)):
        k[q] += base[q]
    for q in order[:extra]:
        k[q] += 1
    return np.array([min(kq, c) for kq, c in zip(k, counts)], dtype=np.int64)


def assign_within(Z: np.ndarray, C: np.ndarray, pslab: np.ndarray, cslab: np.ndarray) -> np.ndarray:
    """Alg. 3 assignment inside each slab: argmin over the slab's own centres."""
    blk = np.zeros(Z.shape[0], dtype=np.int64)
    for q in np.unique(pslab):
        pi = np.flatnonzero(pslab == q)
        ci = np.flatnonzero(cslab == q)
        blk[pi] = ci[assign(Z[pi], C[ci])]
    return blk


def blocking(X, beta_scale, bc: int, kmeans_iters: int, seed: int, partitions: int = 1):
    """Scale, pick random anchors (RAC), run up to T Lloyd iterations, order blocks.

    With partitions = P > 1 the points are first split into P slabs along the
    most relevant dimension (Alg. 2) and RAC (and the Lloyd iterations) run in
    every slab on its own points and anchors (Alg. 3, per worker); P = 1 is
    the single-partition case.

    Readings: the anchors of slab q are the first k_q entries of a
    Fisher-Yates shuffle of that slab's points (listed in increasing index),
    slabs taken in increasing q, all draws from one SplitMix64(seed) stream;
    the k_q follow slab_quota.  Centres are numbered slab by slab.  T = 0 is
    RAC exactly as in Alg. 3; iteration stops early when no assignment
    changes; empty blocks are dropped keeping the relative order of the
    others; the random block order of Alg. 1 Step 2 is a full Fisher-Yates
    shuffle drawn from the same stream after the anchors; block perm[r]
    receives rank r.

    Returns dict(blk, ptr, pts, rank, centres, bc_eff, Z).
    """
    Z = scale(X, beta_scale)
    n = Z.shape[0]
    if partitions > 1:
        pslab, _ = slabs(X, beta_scale, partitions)
    else:
        pslab = np.zeros(n, dtype=np.int64)
    P = max(int(partitions), 1)
    kq = slab_quota(np.bincount(pslab, minlength=P), bc)
    rng = SplitMix64(seed)
    anchors, cslab = [], []
    for q in range(P):
        if kq[q] == 0:
            continue
        members = np.flatnonzero(pslab == q)
        pos = partial_shuffle_prefix(members.size, int(kq[q]), rng)
        anchors.extend(members[np.asarray(pos, dtype=np.int64)])
        cslab.extend([q] * int(kq[q]))
    K = len(anchors)
    cslab = np.asarray(cslab, dtype=np.int64)
    C = Z[np.asarray(anchors, dtype=np.int64)].copy()
    blk = assign_within(Z, C, pslab, cslab)
    for _ in range(kmeans_iters):
        C = centroids(Z, blk, K, prev=C)
        new = assign_within(Z, C, pslab, cslab)
        if np.array_equal(new, blk):
            break
        blk = new
    bc = K
    used = np.unique(blk)
    remap = np.full(bc, -1, dtype=np.int64)
    remap[used] = np.arange(used.size)
    blk = remap[blk]
    bc_eff = int(used.size)
    centres = centroids(Z, blk, bc_eff)
    perm = full_shuffle(bc_eff, rng)
    rank = np.empty(bc_eff, dtype=np.int64)
    rank[np.asarray(perm, dtype=np.int64)] = np.arange(bc_eff)
    counts = np.bincount(blk, minlength=bc_eff)
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    pts = np.argsort(blk, kind="stable").astype(np.int64)
    return dict(blk=blk, ptr=ptr, pts=pts, rank=rank, centres=centres, bc_eff=bc_eff, Z=Z)


# --------------------------------------------------------------------------
# Earlier-ordered m nearest neighbours (Alg. 4 Step 3; Eq. mmsearchingBV)
# --------------------------------------------------------------------------
def knn_block(Z, centre, cand: np.ndarray, m: int) -> np.ndarray:
    """The min(m, |cand|) candidates nearest to centre, ascending by (D, index)."""
    if cand.size == 0 or m == 0:
        return np.zeros(0, dtype=np.int64)
    D = sq_dist_rows(Z[cand], centre)
    o = np.lexsort((cand, D))
    return cand[o[:m]]


def knn(Z, blk, rank, centres, m: int, blocks=None):
    """NN set of each block: points of strictly earlier-ranked blocks nearest to its centre.

    Readings: the query is the block centre (Alg. 4 searches each block's
    neighbours from one query point per block); a neighbour's block may not
    come later in the order, taken here as strictly earlier so that a block
    never conditions on itself; with fewer than m earlier points all of them
    are taken.  The lambda filter of Alg. 4 changes
    only which points are examined, not the answer, so it is not applied here.

    Returns (nbr (k x m, -1 padded), cnt (k)) for the requested blocks (default all).
    """
    bc = centres.shape[0]
    blocks = np.arange(bc) if blocks is None else np.asarray(blocks)
    prank = np.asarray(rank)[np.asarray(blk)]
    nbr = np.full((blocks.size, m), -1, dtype=np.int64)
    cnt = np.zeros(blocks.size, dtype=np.int64)
    for i, b in enumerate(blocks):
        cand = np.nonzero(prank < rank[b])[0]
        J = knn_block(Z, centres[b], cand, m)
        nbr[i, :J.size] = J
        cnt[i] = J.size
    return nbr, cnt


# --------------------------------------------------------------------------
# Scaled Matern kernel (Eq. scale, Eq. maternkernel)
# --------------------------------------------------------------------------
def matern(r: np.ndarray, nu2: int) -> np.ndarray:
    """2^(1-nu)/Gamma(nu) r^nu K_nu(r) for nu = nu2/2: closed forms for
    nu2 in {1, 3, 5, 7}, the Bessel-function definition (scipy's K_nu) for any
    other 2 <= nu2 <= 40, with M(0) = 1.

    Reading: the argument is the scaled distance r itself, with no sqrt(2 nu)
    factor, exactly as Eq. maternkernel is printed.
    """
    e = np.exp(-r)
    if nu2 == 1:
        return e
    if nu2 == 3:
        return (1.0 + r) * e
    if nu2 == 5:
        return (1.0 + r + r * r / 3.0) * e
    if nu2 == 7:
        return (1.0 + r + 2.0 * r * r / 5.0 + r ** 3 / 15.0) * e
    if 2 <= nu2 <= 40:
        return matern_bessel(r, nu2 / 2.0)
    raise ValueError("nu2 must be an integer in [1, 40]")


def matern_bessel(r, nu: float) -> np.ndarray:
    """Eq. maternkernel written out with the Bessel function K_nu (scipy), M(0) = 1."""
    r = np.asarray(r, dtype=np.float64)
    out = np.ones_like(r)
    pos = r > 0
    rp = r[pos]
    out[pos] = 2.0 ** (1.0 - nu) / special.gamma(nu) * rp ** nu * special.kv(nu, rp)
    return out


def cov(Xa: np.ndarray, Xb: np.ndarray, theta, nu2: int, same: np.ndarray | None = None) -> np.ndarray:
    """K_theta(a, b) = sigma^2 M_nu(r) + tau^2 [a is b], r^2 = sum_t ((x_at - x_bt)/beta_t)^2.

    theta = (sigma^2, tau^2, beta_1..beta_d).  Reading: the nugget sigma_0^2 =
    tau^2 enters only where a and b are the same data point (``same`` marks
    those pairs), not for every pair as the printed equation would suggest.
    """
    theta = np.asarray(theta, dtype=np.float64)
    s2, t2, beta = theta[0], theta[1], theta[2:]
    A = np.asarray(Xa, dtype=np.float64) / beta[None, :]
    B = np.asarray(Xb, dtype=np.float64) / beta[None, :]
    diff = A[:, None, :] - B[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    K = s2 * matern(r, nu2)
    if same is not None:
        K = K + t2 * same
    return K


def cov_points(X, ia: np.ndarray, ib: np.ndarray, theta, nu2: int) -> np.ndarray:
    """Covariance between the data points with indices ia and ib (nugget on equal indices)."""
    same = (np.asarray(ia)[:, None] == np.asarray(ib)[None, :]).astype(np.float64)
    return cov(X[ia], X[ib], theta, nu2, same)


# --------------------------------------------------------------------------
# Batched Block Vecchia log-likelihood (Alg. 5) and total (Alg. 1 Step 5)
# --------------------------------------------------------------------------
def block_loglik(X, y, J: np.ndarray, Bpts: np.ndarray, theta, nu2: int) -> float:
    """log p(y_B | y_J) for one block, by the steps of Alg. 5.

    Readings: the Schur step uses Sigma^lk (Alg. 5 prints Sigma^con, whose
    dimensions cannot match Sigma^cor); the -bs/2 log(2 pi) constant of
    Eq. (1) is kept so that one block with no neighbours reproduces Eq. (1).
    """
    J = np.asarray(J, dtype=np.int64)
    Bpts = np.asarray(Bpts, dtype=np.int64)
    bs = Bpts.size
    S_lk = cov_points(X, Bpts, Bpts, theta, nu2)
    yB = y[Bpts]
    if J.size:
        S_con = cov_points(X, J, J, theta, nu2)
        S_cross = cov_points(X, J, Bpts, theta, nu2)
        L = np.linalg.cholesky(S_con)                              # POTRF
        S_cross_p = solve_triangular(L, S_cross, lower=True)       # TRSM
        yJ_p = solve_triangular(L, y[J], lower=True)               # TRSV
        S_cor = S_cross_p.T @ S_cross_p                            # GEMM
        mu_cor = S_cross_p.T @ yJ_p                                # GEMV
        S_new = S_lk - S_cor                                       # Schur complement
        mu_new = mu_cor
    else:
        S_new = S_lk
        mu_new = np.zeros(bs)
    Lp = np.linalg.cholesky(S_new)                                 # POTRF
    v = solve_triangular(Lp, yB - mu_new, lower=True)              # TRSV
    u = float(v @ v)                                               # dot
    dd = 2.0 * float(np.sum(np.log(np.diag(Lp))))                  # log-det
    return -0.5 * (u + dd) - 0.5 * bs * LOG2PI


def loglik_terms(X, y, ptr, pts, nbr, cnt, theta, nu2: int, blocks=None) -> np.ndarray:
    """Per-block terms l_i for the requested blocks (default all)."""
    bc = len(ptr) - 1
    blocks = np.arange(bc) if blocks is None else np.asarray(blocks)
    out = np.empty(blocks.size)
    for i, b in enumerate(blocks):
        Bpts = pts[ptr[b]:ptr[b + 1]]
        J = nbr[b, :cnt[b]]
        out[i] = block_loglik(X, y, J, Bpts, theta, nu2)
    return out


def loglik(X, y, ptr, pts, nbr, cnt, rank, theta, nu2: int) -> float:
    """l = sum of the block terms, added in block-rank order (Alg. 1 Step 5)."""
    terms = loglik_terms(X, y, ptr, pts, nbr, cnt, theta, nu2)
    total = 0.0
    for b in np.argsort(rank):
        total += terms[b]
    return total


# --------------------------------------------------------------------------
# Prediction (Sec. 4.2 block-Vecchia prediction; Sec. 5.5)
# --------------------------------------------------------------------------
def predict(X, y, Xtest, beta_scale, m_pred: int, theta, nu2: int, rows=None):
    """Predictive mean and variances at test points, one test point per block.

    Each test point conditions on its m_pred nearest training points in the
    scaled space (ranked by (D, index) like the estimation neighbours).  The
    mean is Sigma'^cross^T y'_J and the variance the diagonal of Sigma^new,
    following Alg. 5 Step 1 with the test point as the block.  Reading of the
    garbled Sec. 5.5 sentence: var is the observation-scale variance
    (sigma^2 + tau^2 - ...) and var_latent = var - tau^2; the 1000-draw
    conditional simulation from these is oracle/simulate.py.
    Returns (mean, var, var_latent, nbr) for the requested test rows.
    """
    Z = scale(X, beta_scale)
    Zt = scale(Xtest, beta_scale)
    theta = np.asarray(theta, dtype=np.float64)
    s2, t2 = theta[0], theta[1]
    rows = np.arange(Zt.shape[0]) if rows is None else np.asarray(rows)
    mean = np.empty(rows.size)
    var = np.empty(rows.size)
    nbr = np.full((rows.size, m_pred), -1, dtype=np.int64)
    allidx = np.arange(Z.shape[0])
    Xd = np.asarray(X, dtype=np.float64)
    for i, j in enumerate(rows):
        J = knn_block(Z, Zt[j], allidx, m_pred)
        nbr[i, :J.size] = J
        mean[i], var[i] = predict_given(Xd, y, Xtest[j:j + 1], J, theta, nu2)
    return mean, var, var - t2, nbr


def predict_blocked(X, y, Xtest, beta_scale, m_pred: int, bc_test: int, kmeans_iters: int,
                    seed: int, theta, nu2: int, blocks=None):
    """Block prediction (Sec. 5.5: prediction follows the estimation
    pipeline): the test points are blocked like the training points
    (`blocking`, one partition), each test block's conditioning set J is the
    m_pred training points nearest to its centre (all training points are
    candidates, ranked by (D, index)), and each test point of the block gets
    the exact Gaussian conditional given y_J (`predict_given`).
    Returns (mean, var, var_latent, test_block, nbr (blocks x m_pred)) for the
    requested test blocks (default all; mean/var NaN for the others)."""
    tb = blocking(Xtest, beta_scale, bc_test, kmeans_iters, seed)
    Z = scale(X, beta_scale)
    theta = np.asarray(theta, dtype=np.float64)
    Xd = np.asarray(X, dtype=np.float64)
    nt = np.asarray(Xtest).shape[0]
    mean = np.full(nt, np.nan)
    var = np.full(nt, np.nan)
    K = tb["bc_eff"]
    nbr = np.full((K, m_pred), -1, dtype=np.int64)
    allidx = np.arange(Z.shape[0])
    for b in (range(K) if blocks is None else blocks):
        J = knn_block(Z, tb["centres"][b], allidx, m_pred)
        nbr[b, :J.size] = J
        for q in tb["pts"][tb["ptr"][b]:tb["ptr"][b + 1]]:
            mean[q], var[q] = predict_given(Xd, y, Xtest[q:q + 1], J, theta, nu2)
    return mean, var, var - theta[1], tb["blk"], nbr


def predict_given(Xd, y, xt, J, theta, nu2: int):
    """Mean and observation-scale variance at one test point xt (1 x d) given
    its neighbour set J (the conditional of Alg. 5 Step 1 with xt as block)."""
    theta = np.asarray(theta, dtype=np.float64)
    s2, t2 = theta[0], theta[1]
    xt = np.asarray(xt, dtype=np.float64)
    S_con = cov_points(Xd, J, J, theta, nu2)
    S_cross = cov(Xd[J], xt, theta, nu2)                         # distinct points: no nugget
    L = np.linalg.cholesky(S_con)
    S_cross_p = solve_triangular(L, S_cross, lower=True)
    yJ_p = solve_triangular(L, y[J], lower=True)
    return float(S_cross_p[:, 0] @ yJ_p), s2 + t2 - float(S_cross_p[:, 0] @ S_cross_p[:, 0])
