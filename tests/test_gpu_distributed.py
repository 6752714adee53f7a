"""The distributed pipeline (Alg. 1-4) with the GPU backend: two gloo ranks,
both on this GPU (their kernels never wait on each other; the exchanges are
host collectives).  Gathered over the ranks, blocks, order, centres,
neighbour sets and block terms must equal the single-process GPU path
(sbv_blocking_partitioned with P = 2, sbv_knn, sbv_loglik) bit for bit.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from synth.inputs import standard_normal, uniform_points

pytestmark = pytest.mark.gpu

N, D, BC, M, T, SEED = 40_000, 5, 800, 30, 3, 9
BETA = np.array([0.3, 0.6, 0.15, 0.9, 0.5])
THETA = np.array([1.0, 0.01, 0.3, 0.6, 0.15, 0.9, 0.5])


def data():
    X = uniform_points(N, D, 21)
    y = np.sin(6 * X[:, 2]) + X[:, 0] * X[:, 1] + 0.05 * standard_normal(N, 22)
    return X, y


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2504_12004_gb300 import Context
    from paper_2504_12004_gb300 import distributed as dd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, y = data()
        gid = np.arange(N)
        mine = gid % world == rank
        be = dd.GpuBackend(Context(0))
        lb = dd.distributed_blocking(be, X[mine], y[mine], gid[mine], BETA, BC, T, SEED)
        lp = dd.distributed_knn(be, lb, BETA, M)
        tot, terms = dd.distributed_loglik(be, lp, THETA, precision="fp64")
        members = [lb.gid[lb.pts[lb.ptr[i]:lb.ptr[i + 1]]] for i in range(lb.block_id.size)]
        np.savez(os.path.join(out, f"rank{rank}.npz"), block_id=lb.block_id, rank=lb.rank,
                 centres=lb.centres, nbr=lp.nbr_gid, cnt=lp.cnt, tot=tot, terms=terms[0],
                 rounds=lp.rounds, sizes=np.array([m.size for m in members]),
                 members=np.concatenate(members), received=lp.received)
    finally:
        dist.destroy_process_group()


def test_two_ranks_equal_single_process(tmp_path):
    from paper_2504_12004_gb300 import build, Context
    build.build()
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [dict(np.load(tmp_path / f"rank{r}.npz")) for r in range(world)]
    ctx = Context(0)
    X, y = data()
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    b = ctx.sbv_blocking(Xd, BETA, BC, T, SEED, partitions=world)
    nbr, cnt = ctx.sbv_knn(Xd, BETA, b["ptr"], b["pts"], b["rank"], b["centres"], M)
    terms = torch.empty(1, b["bc_eff"], dtype=torch.float64, device="cuda")
    ll = ctx.sbv_loglik(Xd, yd, b["ptr"], b["pts"], nbr.contiguous(), cnt, THETA, nu2=5,
                        precision="fp64", block_terms=terms)
    assert np.array_equal(np.concatenate([g["block_id"] for g in got]), np.arange(b["bc_eff"]))
    assert np.array_equal(np.concatenate([g["rank"] for g in got]), b["rank"].cpu().numpy())
    assert np.array_equal(np.concatenate([g["centres"] for g in got]), b["centres"].cpu().numpy())
    assert np.array_equal(np.concatenate([g["members"] for g in got]), b["pts"].cpu().numpy())
    assert np.array_equal(np.concatenate([g["cnt"] for g in got]), cnt.cpu().numpy())
    assert np.array_equal(np.concatenate([g["nbr"] for g in got]), nbr.cpu().numpy())
    assert np.array_equal(np.concatenate([g["terms"] for g in got]), terms[0].cpu().numpy())
    assert np.array_equal(got[0]["tot"], got[1]["tot"])
    assert got[0]["tot"][0] == pytest.approx(float(ll[0]), rel=1e-13)
    # the neighbour search needed points of the other rank's slab
    assert all(int(g["received"]) > 0 for g in got)
    print("rounds", [int(g["rounds"]) for g in got], "received", [int(g["received"]) for g in got])
