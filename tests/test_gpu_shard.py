"""A rank's share of an evaluation on the GPU: the sliced structure of a
contiguous block range gives the same block terms, bit for bit, as the full
call (same kernel per item, same launch plan when the same nmax is passed),
and the rank-ordered sum of the range totals equals the full total within
rounding (the sums group the blocks differently).  One GPU evaluates the
ranges in turn; no collective is involved.
"""
import numpy as np
import pytest
import torch

from paper_2504_12004_gb300 import shard
from synth.inputs import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("world", [2, 3, 7])
def test_ranges_reproduce_block_terms(ctx, precision, world):
    w = workload("sine10d", n=20000, bc=400, m=60)
    X = torch.from_numpy(w["X"]).cuda()
    y = torch.from_numpy(w["y"]).cuda()
    b = ctx.sbv_blocking(X, w["beta_scale"], w["bc"], 3, 11)
    nbr, cnt = ctx.sbv_knn(X, w["beta_scale"], b["ptr"], b["pts"], b["rank"], b["centres"], w["m"])
    nbr = nbr.contiguous()
    nmax = ctx.max_block_size(b["ptr"], cnt)
    th0 = np.asarray(w["theta"], dtype=np.float64).reshape(-1, X.shape[1] + 2)[0]
    th1 = th0.copy()
    th1[0] *= 1.3
    th1[2:] *= 0.8
    th = np.stack([th0, th1])          # two parameter rows
    bc = cnt.numel()
    bt = torch.empty(2, bc, dtype=torch.float64, device="cuda")
    ll = ctx.sbv_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, th, 5, precision=precision,
                        block_terms=bt, nmax=nmax).cpu().numpy()
    bt = bt.cpu().numpy()
    R = shard.balanced_ranges(b["ptr"].cpu().numpy(), cnt.cpu().numpy(), world)
    parts = []
    for lo, hi in R:
        if hi > lo:
            bt_r = torch.empty(2, hi - lo, dtype=torch.float64, device="cuda")
            part = shard.loglik_range(ctx, X, y, b["ptr"], b["pts"], nbr, cnt, th, lo, hi,
                                      precision=precision, block_terms=bt_r, nmax=nmax)
            assert np.array_equal(bt_r.cpu().numpy(), bt[:, lo:hi])
        else:
            part = shard.loglik_range(ctx, X, y, b["ptr"], b["pts"], nbr, cnt, th, lo, hi)
        parts.append(part.cpu().numpy())
    tot = shard.combine_rank_order(parts)
    assert np.allclose(tot, ll, rtol=1e-12, atol=0)
    # the one-rank path returns the rank's own sums
    one = shard.sharded_loglik(lambda lo, hi: shard.loglik_range(
        ctx, X, y, b["ptr"], b["pts"], nbr, cnt, th, lo, hi, precision=precision,
        nmax=nmax).cpu().numpy(), b["ptr"].cpu().numpy(), cnt.cpu().numpy(), 2, 0, 1)
    assert np.array_equal(one, ll)
