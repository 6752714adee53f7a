"""Sharding one evaluation over ranks (Alg. 1 Step 5), host logic on CPU.

- The block ranges are contiguous, cover [0, bc) in order and balance the
  per-rank cost sum_i (N_i^3/3 + N_i^2): each boundary is off its target by at
  most half a block, so no rank exceeds total/world by more than one block.
- Two gloo ranks evaluate their ranges with the oracle and exchange the
  per-theta partial sums: every rank returns the same total, equal bit for bit
  to the rank-ordered sum of the range sums and to the oracle's total within
  rounding.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import sbv
from paper_2504_12004_gb300 import shard
from synth.inputs import uniform_points

THETA = np.array([[1.1, 0.02, 0.15, 0.4], [0.8, 0.05, 0.3, 0.2]])


def problem():
    X = uniform_points(500, 2, 3)
    y = np.sin(6 * X[:, 0]) + X[:, 1] ** 2 + 0.1 * np.random.default_rng(4).standard_normal(500)
    b = sbv.blocking(X, np.array([0.3, 0.3]), 50, 3, 5)
    nbr, cnt = sbv.knn(b["Z"], b["blk"], b["rank"], b["centres"], 12)
    return X, y, b["ptr"], b["pts"], nbr, cnt


def range_sums(P, lo, hi):
    X, y, ptr, pts, nbr, cnt = P
    if hi <= lo:
        return np.zeros(len(THETA))
    blocks = np.arange(lo, hi)
    return np.array([sbv.loglik_terms(X, y, ptr, pts, nbr, cnt, th, 5, blocks=blocks).sum()
                     for th in THETA])


def test_ranges_cover_in_order_and_balance():
    rng = np.random.default_rng(1)
    sz = rng.integers(1, 100, 1000)
    ptr = np.concatenate([[0], np.cumsum(sz)])
    cnt = rng.integers(0, 120, 1000)
    cost = shard.block_cost(ptr, cnt)
    N = sz + cnt
    assert np.allclose(cost, N ** 3 / 3.0 + N ** 2)
    for world in (1, 2, 3, 8, 64):
        R = shard.balanced_ranges(ptr, cnt, world)
        assert len(R) == world and R[0][0] == 0 and R[-1][1] == 1000
        assert all(R[r][1] == R[r + 1][0] and R[r][0] <= R[r][1] for r in range(world - 1))
        per = np.array([cost[a:b].sum() for a, b in R])
        assert per.max() <= cost.sum() / world + cost.max() + 1e-9
    assert shard.balanced_ranges(ptr, cnt, 1) == [(0, 1000)]


def test_more_ranks_than_blocks_leaves_empty_ranges():
    ptr = np.array([0, 3, 5, 9])
    cnt = np.array([0, 3, 4])
    R = shard.balanced_ranges(ptr, cnt, 5)
    assert R[0][0] == 0 and R[-1][1] == 3
    # at least world - bc ranges are empty; here block 2 alone is 73 % of the
    # cost, so ranks share blocks 0 and 1 before it and more ranges stay empty
    assert sum(b - a for a, b in R) == 3 and sum(1 for a, b in R if a == b) >= 2
    assert R == [(0, 2), (2, 2), (2, 2), (2, 3), (3, 3)]
    with pytest.raises(ValueError):
        shard.balanced_ranges(ptr, cnt, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = problem()
        tot = shard.sharded_loglik(lambda lo, hi: range_sums(P, lo, hi), P[2], P[5], len(THETA),
                                   rank, world)
        np.save(os.path.join(out, f"rank{rank}.npy"), tot)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_in_rank_order(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    assert np.array_equal(got[0], got[1])            # every rank holds the same total
    P = problem()
    R = shard.balanced_ranges(P[2], P[5], world)
    want = shard.combine_rank_order([range_sums(P, lo, hi) for lo, hi in R])
    assert np.array_equal(got[0], want)              # rank-ordered sum, bit for bit
    full = range_sums(P, 0, len(P[5]))
    assert np.allclose(got[0], full, rtol=1e-12, atol=0)
