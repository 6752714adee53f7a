"""One likelihood evaluation sharded over ranks (Alg. 1 Step 5).

Given a fixed structure (blocks, their order and neighbour sets) the block
terms are independent and read only X and y.  A rank evaluates a contiguous
range [lo, hi) of blocks by passing the sliced structure to sbv_loglik
(ptr[lo:hi+1], nbr[lo:hi], cnt[lo:hi]; ptr holds absolute offsets into pts,
so pts is shared as is).  The one exchange is a sum of B doubles per
evaluation: every rank's per-theta partial sums are gathered and added on the
host in rank order, so the total is bit-identical for a given world size and
does not depend on timing.  The ranges split the blocks so that each rank's
share of sum_i (N_i^3 / 3 + N_i^2), N_i = m_i + bs_i, is as even as contiguous
ranges allow.

This module holds host logic only; the evaluation of a range runs in
libsbv.so (loglik_range).
"""
from __future__ import annotations

import numpy as np
import torch


def block_cost(ptr: np.ndarray, cnt: np.ndarray) -> np.ndarray:
    """Algorithmic flops of each block's bordered Cholesky, N^3/3 + N^2."""
    N = np.diff(np.asarray(ptr, dtype=np.int64)).astype(np.float64) + np.asarray(cnt, dtype=np.float64)
    return N ** 3 / 3.0 + N ** 2


def balanced_ranges(ptr, cnt, world: int) -> list[tuple[int, int]]:
    """Contiguous block ranges, one per rank, covering [0, bc) in order.

    The boundary between ranks r - 1 and r is the block boundary whose running
    cost is nearest to r / world of the total, so every boundary is off its
    target by at most half a block's cost.  Ranges are empty (lo == hi) when
    there are fewer blocks than ranks.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = block_cost(ptr, cnt)
    bc = cost.size
    run = np.concatenate([[0.0], np.cumsum(cost)])   # run[c] = cost of blocks [0, c)
    total = float(run[-1])
    cuts = [0]
    for r in range(1, world):
        t = total * r / world
        c = int(np.searchsorted(run, t, side="left"))   # run[c] >= t
        if c > 0 and (c > bc or t - run[c - 1] <= run[c] - t):
            c -= 1
        cuts.append(min(max(c, cuts[-1]), bc))
    cuts.append(bc)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def loglik_range(ctx, X, y, ptr, pts, nbr, cnt, theta, lo: int, hi: int, **kw) -> torch.Tensor:
    """Per-theta sums of the block terms of blocks [lo, hi), on the device."""
    d = X.shape[1]
    B = np.asarray(theta, dtype=np.float64).reshape(-1, 2 + d).shape[0]
    if hi <= lo:
        return torch.zeros(B, dtype=torch.float64, device=X.device)
    return ctx.sbv_loglik(X, y, ptr[lo:hi + 1], pts, nbr[lo:hi], cnt[lo:hi], theta, **kw)


def combine_rank_order(parts) -> np.ndarray:
    """Sum of the ranks' per-theta partial sums, added in rank order."""
    parts = [np.asarray(p, dtype=np.float64) for p in parts]
    tot = np.zeros_like(parts[0])
    for p in parts:
        tot = tot + p
    return tot


def sharded_loglik(eval_range, ptr, cnt, B: int, rank: int, world: int, group=None) -> np.ndarray:
    """Total log-likelihood (B values) of one evaluation split over `world` ranks.

    eval_range(lo, hi) returns this rank's B per-theta sums of blocks [lo, hi)
    (loglik_range on a GPU).  With world > 1 the partial sums are exchanged by
    one all_gather on `group` (gloo: host tensors; nccl: device tensors) and
    every rank returns the same rank-ordered total.
    """
    lo, hi = balanced_ranges(ptr, cnt, world)[rank]
    part = torch.as_tensor(np.asarray(eval_range(lo, hi), dtype=np.float64).reshape(B))
    if world == 1:
        return part.numpy().copy()
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        part = part.cuda()
    got = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(got, part, group=group)
    return combine_rank_order([g.cpu().numpy() for g in got])
