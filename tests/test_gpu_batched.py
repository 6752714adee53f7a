"""Batched likelihood over many parameter candidates with large blocks.

The workload: 2,000,000 points on [0,1]^20 (sine-sum response), 40,000
K-means blocks, m = 200 earlier neighbours (N = m_i + bs_i up to ~320, past
the shared memory of one CTA, so the mixed kernel keeps its triangle in a
per-CTA global slice), and 64 log-uniform range candidates evaluated in one
graph-captured launch.  At full size the oracle checks sampled items: the
nearest-centre property of sampled points, exact neighbour sets of sampled
blocks, and block terms of sampled (candidate, block) pairs; the totals of
the mixed path are checked against the FP64 path.
"""
import time

import numpy as np
import pytest
import torch

from oracle import sbv
from synth.inputs import loguniform_candidates, theta_rows, workload

pytestmark = pytest.mark.gpu

TOLS = {"fp64": 1e-9, "mixed": 1e-6, "mixed_bf16": 1e-6}   # |dl| / n


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


def structure(ctx, w, T=3, seed=11):
    X = torch.from_numpy(w["X"]).cuda()
    b = ctx.sbv_blocking(X, w["beta_scale"], w["bc"], T, seed)
    nbr, cnt = ctx.sbv_knn(X, w["beta_scale"], b["ptr"], b["pts"], b["rank"], b["centres"], w["m"])
    return X, torch.from_numpy(w["y"]).cuda(), b, nbr.contiguous(), cnt


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
def test_blocks_past_shared_memory_match_oracle(ctx, precision):
    # 40 blocks of ~100 points with 200 neighbours: N up to ~300 at d = 20
    w = workload("sine20d", n=4000, bc=40, m=200)
    X, y, b, nbr, cnt = structure(ctx, w)
    nmax = ctx.max_block_size(b["ptr"], cnt)
    assert nmax > 280
    th = w["theta"][:3]
    bt = torch.empty(3, cnt.numel(), dtype=torch.float64, device="cuda")
    ll = ctx.sbv_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, th, nu2=5, precision=precision,
                        block_terms=bt).cpu().numpy()
    ptr, pts = b["ptr"].cpu().numpy(), b["pts"].cpu().numpy()
    nb, cn = nbr.cpu().numpy(), cnt.cpu().numpy()
    for r in range(3):
        want = sbv.loglik_terms(w["X"], w["y"], ptr, pts, nb, cn, th[r], 5)
        assert abs(ll[r] - want.sum()) / 4000 <= TOLS[precision], (precision, r, ll[r], want.sum())


def test_full_size_batched_candidates(ctx):
    from paper_2504_12004_gb300._lib import Context  # noqa: F401
    w = workload("sine20d")
    n, d, B = w["n"], w["d"], w["B"]
    t0 = time.time()
    X, y, b, nbr, cnt = structure(ctx, w)
    torch.cuda.synchronize()
    t_pre = time.time() - t0
    bc = cnt.numel()
    sizes = np.diff(b["ptr"].cpu().numpy())
    nmax = ctx.max_block_size(b["ptr"], cnt)
    print(f"preprocessing {t_pre:.1f} s; {bc} blocks, sizes {sizes.min()}..{sizes.max()} "
          f"(median {np.median(sizes):.0f}); largest N = {nmax}")
    rng = np.random.default_rng(5)
    # blocking: every point in exactly one block, and each sampled block's
    # centre is the mean of its members (FP64 sum in increasing point index,
    # one division), bit for bit
    Z = sbv.scale(w["X"], w["beta_scale"])
    C = b["centres"].cpu().numpy()
    blk = b["blk"].cpu().numpy()
    ptr_h, pts_h = b["ptr"].cpu().numpy(), b["pts"].cpu().numpy()
    assert ptr_h[-1] == n and np.array_equal(np.sort(pts_h), np.arange(n))
    for bi in rng.choice(bc, 20, replace=False):
        mem = np.sort(pts_h[ptr_h[bi]:ptr_h[bi + 1]])
        assert np.all(blk[mem] == bi)
        mean = np.cumsum(Z[mem], axis=0)[-1] / len(mem)
        assert np.array_equal(C[bi], mean)
    # kNN: exact neighbour sets of sampled blocks
    rank = b["rank"].cpu().numpy()
    nb, cn = nbr.cpu().numpy(), cnt.cpu().numpy()
    sample = rng.choice(bc, 6, replace=False)
    want_nbr, want_cnt = sbv.knn(Z, blk, rank, C, w["m"], blocks=sample)
    for k, blk_i in enumerate(sample):
        assert cn[blk_i] == want_cnt[k]
        assert np.array_equal(nb[blk_i, :cn[blk_i]], want_nbr[k, :want_cnt[k]])
    # 64 candidates in one captured launch (mixed), against FP64 on two rows
    th = w["theta"]
    assert th.shape == (B, 2 + d)
    g = ctx.sbv_loglik_graph_create(X, y, b["ptr"], b["pts"], nbr, cnt, B=B, nu2=5,
                                    precision="mixed", nmax=nmax)
    try:
        ll = g.launch(th).clone()
        torch.cuda.synchronize()
        t1 = time.time()
        ll2 = g.launch(th).clone()
        torch.cuda.synchronize()
        t_launch = time.time() - t1
    finally:
        g.close()
    ctx.sbv_sync_status()
    assert torch.equal(ll, ll2)
    ll = ll.cpu().numpy()
    ref = ctx.sbv_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, th[:2], nu2=5, precision="fp64",
                         nmax=nmax).cpu().numpy()
    err = np.abs(ll[:2] - ref) / n
    print(f"64 candidates: {t_launch:.2f} s per launch; |dl|/n vs FP64 {err}")
    assert np.all(err <= TOLS["mixed"])
    # sampled block terms of one candidate against the oracle
    bt = torch.empty(1, bc, dtype=torch.float64, device="cuda")
    ctx.sbv_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, th[7:8], nu2=5, precision="mixed",
                   block_terms=bt, nmax=nmax)
    bt = bt.cpu().numpy()[0]
    ptr, pts = b["ptr"].cpu().numpy(), b["pts"].cpu().numpy()
    want = sbv.loglik_terms(w["X"], w["y"], ptr, pts, nb, cn, th[7], 5, blocks=sample)
    # per block the mixed bar scales with the block's size (|dl|/n <= 1e-6 per point)
    assert np.all(np.abs(bt[sample] - want) <= 1e-6 * sizes[sample] + 1e-9), (bt[sample], want)
