"""Distributed preprocessing and evaluation (Alg. 1-4) on gloo ranks on the
CPU: slab routing with an all-to-all, blocking of each rank's slab, the
replayed block order, the filtered neighbour search with the block exchange
and the rank-ordered sum.  The per-rank arithmetic comes from the oracle
(injected as the backend; the product module never imports it), so this
checks the host logic and the exchanges: gathered over the ranks, blocks,
order, centres and neighbour sets must equal the oracle's single-process
partitioned blocking and search with P = world, exactly.  The replay of the
random choices (sbv_rac_plan, host code of libsbv.so) is checked against the
oracle's generator directly.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import prng, sbv
from synth.inputs import standard_normal, uniform_points

N, D, BC, M, T, SEED = 2400, 3, 48, 16, 3, 77
BETA = np.array([0.5, 0.2, 0.9])       # d_max = dimension 1
THETA = np.array([1.0, 0.02, 0.3, 0.15, 0.6])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2504_12004_gb300 import build
    build.build()


class OracleBackend:
    """The oracle's arithmetic behind the backend interface of the
    distributed module."""

    def slabs(self, X, beta, P):
        return sbv.slabs(X, beta, P)[0]

    def blocking_anchored(self, X, beta, anchors, T):
        Z = sbv.scale(X, beta)
        K = len(anchors)
        C = Z[np.asarray(anchors)].copy()
        blk = sbv.assign(Z, C)
        for _ in range(T):
            C = sbv.centroids(Z, blk, K, prev=C)
            new = sbv.assign(Z, C)
            if np.array_equal(new, blk):
                break
            blk = new
        used = np.unique(blk)
        remap = np.full(K, -1, dtype=np.int64)
        remap[used] = np.arange(used.size)
        blk = remap[blk]
        centres = sbv.centroids(Z, blk, used.size)
        counts = np.bincount(blk, minlength=used.size)
        ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        return dict(ptr=ptr, pts=np.argsort(blk, kind="stable"), centres=centres)

    def knn(self, X, beta, ptr, pts, rank, centres, m):
        Z = sbv.scale(X, beta)
        blk = np.empty(Z.shape[0], dtype=np.int64)
        for b in range(len(ptr) - 1):
            blk[pts[ptr[b]:ptr[b + 1]]] = b
        return sbv.knn(Z, blk, rank, centres, m)

    def loglik_terms(self, X, y, ptr, pts, nbr, cnt, theta, nu2, precision):
        return sbv.loglik_terms(X, y, ptr, pts, nbr, cnt, theta, nu2)[None, :]


def data():
    X = uniform_points(N, D, 5)
    y = np.sin(4 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.1 * standard_normal(N, 6)
    return X, y


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out, layout, alpha):
    import torch.distributed as dist
    from paper_2504_12004_gb300 import distributed as dd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, y = data()
        gid = np.arange(N)
        # the points each worker loads (Step 0): interleaved, or all on rank 0
        mine = gid % world == rank if layout == "interleaved" else (gid >= 0) == (rank == 0)
        be = OracleBackend()
        lb = dd.distributed_blocking(be, X[mine], y[mine], gid[mine], BETA, BC, T, SEED)
        lp = dd.distributed_knn(be, lb, BETA, M, alpha=alpha)
        tot, terms = dd.distributed_loglik(be, lp, THETA)
        members = [lb.gid[lb.pts[lb.ptr[i]:lb.ptr[i + 1]]] for i in range(lb.block_id.size)]
        np.savez(os.path.join(out, f"rank{rank}.npz"), block_id=lb.block_id, rank=lb.rank,
                 centres=lb.centres, nbr=lp.nbr_gid, cnt=lp.cnt, tot=tot, terms=terms[0],
                 rounds=lp.rounds, sizes=np.array([m.size for m in members]),
                 members=np.concatenate(members) if members else np.zeros(0, np.int64))
    finally:
        dist.destroy_process_group()


def run_world(tmp_path, world, layout, alpha=100.0):
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), layout, alpha), nprocs=world,
             join=True)
    return [dict(np.load(tmp_path / f"rank{r}.npz")) for r in range(world)]


def check_against_single_process(got, world):
    X, y = data()
    ref = sbv.blocking(X, BETA, BC, T, SEED, partitions=world)
    Z = ref["Z"]
    nbr, cnt = sbv.knn(Z, ref["blk"], ref["rank"], ref["centres"], M)
    terms = sbv.loglik_terms(X, y, ref["ptr"], ref["pts"], nbr, cnt, THETA, 5)
    bid = np.concatenate([g["block_id"] for g in got])
    assert np.array_equal(bid, np.arange(ref["bc_eff"]))     # every block once, slab by slab
    assert np.array_equal(np.concatenate([g["rank"] for g in got]), ref["rank"])
    assert np.array_equal(np.concatenate([g["centres"] for g in got]), ref["centres"])
    members = np.concatenate([g["members"] for g in got])
    assert np.array_equal(members, ref["pts"])
    assert np.array_equal(np.concatenate([g["sizes"] for g in got]), np.diff(ref["ptr"]))
    assert np.array_equal(np.concatenate([g["cnt"] for g in got]), cnt)
    assert np.array_equal(np.concatenate([g["nbr"] for g in got]), nbr)
    assert np.array_equal(np.concatenate([g["terms"] for g in got]), terms)
    # every rank holds the same rank-ordered total, equal to the plain sum
    for g in got[1:]:
        assert np.array_equal(g["tot"], got[0]["tot"])
    assert got[0]["tot"][0] == pytest.approx(terms.sum(), rel=1e-13)


@pytest.mark.parametrize("world,layout", [(2, "interleaved"), (3, "interleaved"), (2, "rank0")])
def test_distributed_pipeline_equals_single_process(tmp_path, world, layout):
    got = run_world(tmp_path, world, layout)
    check_against_single_process(got, world)
    # the paper's alpha = 100 holds enough candidates in one exchange
    assert all(int(g["rounds"]) == 1 for g in got), [int(g["rounds"]) for g in got]


def test_small_lambda_grows_until_exact(tmp_path):
    """alpha = 0.5 starts with a lambda whose ball holds fewer than m points:
    lambda doubles until every block's m-th neighbour lies inside it, and the
    answer is the exact one."""
    got = run_world(tmp_path, 2, "interleaved", alpha=0.5)
    assert all(int(g["rounds"]) >= 2 for g in got)
    check_against_single_process(got, 2)


def test_rac_plan_replays_the_oracle_generator():
    from paper_2504_12004_gb300._lib import rac_plan
    counts = np.array([700, 0, 1300, 401])
    bc = 37
    quota, pos, rank = rac_plan(1234, counts, bc, 35)
    kq = sbv.slab_quota(counts, bc)
    assert np.array_equal(quota, kq)
    rng = prng.SplitMix64(1234)
    want = []
    for q in range(counts.size):
        if kq[q]:
            want.extend(prng.partial_shuffle_prefix(int(counts[q]), int(kq[q]), rng))
    assert np.array_equal(pos, np.array(want))
    perm = prng.full_shuffle(35, rng)
    r = np.empty(35, dtype=np.int64)
    r[np.asarray(perm)] = np.arange(35)
    assert np.array_equal(rank, r)
    with pytest.raises(Exception):
        rac_plan(1, counts, 2)          # fewer blocks than slabs
