"""Pins of the partitioned blocking (Alg. 2 slabs, then Alg. 3 RAC per slab).

- Slab index int(x_dmax * P) on hand-picked coordinates, d_max = argmax 1/beta.
- Anchor quota: a hand-worked largest-remainder example and its invariants.
- All points in one slab: identical to the single-partition blocking.
- Every block lies in one slab; with T = 0 every point sits in the block of
  the nearest anchor of its own slab (brute force); with converged Lloyd
  iterations, of the nearest final centre of its own slab.
"""
import numpy as np

from oracle import sbv
from synth.inputs import uniform_points


def test_slab_index_and_dmax():
    X = np.array([[0.3, 0.0], [0.3, 0.2499999], [0.3, 0.25], [0.3, 0.5], [0.3, 0.999],
                  [0.3, 1.0], [0.3, -0.1], [0.3, 1.7]])
    q, dmax = sbv.slabs(X, np.array([0.9, 0.2]), 4)      # 1/beta largest for dimension 1
    assert dmax == 1
    assert list(q) == [0, 0, 1, 2, 3, 3, 0, 3]
    _, dmax2 = sbv.slabs(X, np.array([0.5, 0.5]), 4)     # tie: the first dimension
    assert dmax2 == 0


def test_slab_quota():
    assert list(sbv.slab_quota([5, 3, 2], 5)) == [2, 2, 1]
    assert list(sbv.slab_quota([10], 7)) == [7]
    assert list(sbv.slab_quota([0, 4, 0, 6], 2)) == [0, 1, 0, 1]
    # R = 497 after one each: bases 0, 495, 1; remainders 497, 20, 487 -> the
    # extra anchor goes to slab 0, which holds one point, so it is dropped
    assert list(sbv.slab_quota([1, 1000, 3], 500)) == [1, 496, 2]
    rng = np.random.default_rng(0)
    for _ in range(50):
        c = rng.integers(0, 300, size=rng.integers(1, 20))
        if c.sum() == 0:
            continue
        bc = int(rng.integers(int((c > 0).sum()), c.sum() + 1))
        k = sbv.slab_quota(c, bc)
        assert np.all(k <= c) and np.all((k > 0) == (c > 0))
        assert k.sum() <= bc


def test_single_populated_slab_equals_flat():
    X = uniform_points(500, 3, 31)
    X[:, 2] *= 0.2                         # d_max = 2; every point in slab 0 of P = 4
    beta = np.array([0.5, 0.7, 0.1])
    a = sbv.blocking(X, beta, 40, 3, 9, partitions=4)
    b = sbv.blocking(X, beta, 40, 3, 9)
    for key in ("blk", "ptr", "pts", "rank", "centres"):
        assert np.array_equal(a[key], b[key]), key


def test_blocks_stay_in_slabs_and_points_take_nearest_anchor():
    X = uniform_points(1200, 4, 33)
    beta = np.array([0.2, 0.4, 0.6, 0.8])
    P = 5
    pslab, _ = sbv.slabs(X, beta, P)
    out = sbv.blocking(X, beta, 60, 0, 5, partitions=P)
    blk, Z = out["blk"], out["Z"]
    for b in range(out["bc_eff"]):
        assert np.unique(pslab[blk == b]).size == 1
    # T = 0: recover the anchors (each centre's members include its anchor, the
    # block's single point nearest ... ) by re-running the draws
    kq = sbv.slab_quota(np.bincount(pslab, minlength=P), 60)
    rng = sbv.SplitMix64(5)
    anchors = []
    for q in range(P):
        mem = np.flatnonzero(pslab == q)
        anchors += list(mem[sbv.partial_shuffle_prefix(mem.size, int(kq[q]), rng)])
    A = Z[np.array(anchors)]
    aslab = pslab[np.array(anchors)]
    for i in range(0, 1200, 7):
        cand = np.flatnonzero(aslab == pslab[i])
        D = ((Z[i] - A[cand]) ** 2).sum(1)
        j = cand[np.argmin(D)]
        # the block holding anchor j is the block of point i
        assert blk[i] == blk[anchors[j]]


def test_converged_lloyd_is_nearest_centre_within_slab():
    X = uniform_points(800, 3, 35)
    beta = np.array([0.3, 0.5, 0.9])
    P = 3
    pslab, _ = sbv.slabs(X, beta, P)
    out = sbv.blocking(X, beta, 30, 200, 6, partitions=P)
    blk, Z, C = out["blk"], out["Z"], out["centres"]
    cslab = np.array([pslab[blk == b][0] for b in range(out["bc_eff"])])
    for i in range(800):
        cand = np.flatnonzero(cslab == pslab[i])
        D = ((Z[i] - C[cand]) ** 2).sum(1)
        assert blk[i] == cand[np.argmin(D)]
