"""Distributed SBV preprocessing and evaluation over ranks (Alg. 1-4).

One rank per GPU.  The steps and their exchanges:

* Alg. 2 -- every rank routes its points to slab q = int(x_dmax * P) (the
  slab kernel, `sbv_slabs`) and one all-to-all delivers to rank q the points
  of slab q (global id, y and coordinates travel together).
* Alg. 3 -- every rank blocks its own slab (RAC from its anchors, then Lloyd
  iterations, `sbv_blocking_anchored`) with no communication.  The random
  choices depend only on the seed and the slab sizes, so after one all-gather
  of the sizes every rank replays them (`sbv_rac_plan`): anchors per slab, and,
  after an all-gather of the non-empty block counts, the random block order
  (Alg. 1 Step 2).  The result equals `sbv_blocking_partitioned` with
  P = world on all points, block for block and bit for bit.
* Alg. 4 -- every block i gets a threshold lambda_i from Eq.
  distancethreshold with its own candidate count (the points of earlier
  blocks) in place of n; the centres with radii, ranks and thresholds are
  all-gathered; each rank sends to rank q every block j that can hold a point
  within lambda_i of some later-ordered block i of rank q,
  ||c_i - c_j|| <= lambda_i + r_j (r_j the largest distance of block j's
  points to c_j); the receiving rank runs the neighbour search on its own
  points plus those blocks.  A block's answer is accepted when its m-th
  neighbour lies within lambda_i (then every nearer earlier-ordered point is
  among the candidates) or when it has all the earlier-ordered points there
  are; otherwise its lambda_i doubles and the exchange repeats.  The neighbour
  sets therefore equal the single-GPU search.
* Alg. 1 Steps 4-5 -- every rank evaluates the block terms of its own blocks
  on its local problem (own points plus received ones) and the per-theta sums
  are combined in rank order.

The exchanges run on host tensors for the gloo backend and on device tensors
for nccl.  The per-rank compute goes through a backend object: `GpuBackend`
(libsbv.so on this rank's GPU) in the product; tests may pass another with the
same methods.  This module holds host logic only: routing, bookkeeping and
the lambda schedule.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch
import torch.distributed as dist

from ._lib import rac_plan


# --------------------------------------------------------------------------
# exchanges
# --------------------------------------------------------------------------
def _coll_device(group) -> torch.device:
    return torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")


def alltoall_rows(parts: list[np.ndarray], group=None) -> list[np.ndarray]:
    """parts[q] (rows x w float64, same w everywhere) goes to rank q; returns
    the row blocks received from every rank, in rank order."""
    world = dist.get_world_size(group)
    dev = _coll_device(group)
    w = parts[0].shape[1]
    counts = torch.tensor([p.shape[0] for p in parts], dtype=torch.int64, device=dev)
    recv_counts = torch.empty(world, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv_counts, counts, group=group)
    rc = recv_counts.cpu().tolist()
    send = torch.from_numpy(np.ascontiguousarray(np.concatenate(parts, axis=0))).to(dev).reshape(-1)
    recv = torch.empty(sum(rc) * w, dtype=torch.float64, device=dev)
    dist.all_to_all_single(recv, send, [c * w for c in rc], [p.shape[0] * w for p in parts],
                           group=group)
    out = recv.cpu().numpy().reshape(-1, w)
    offs = np.concatenate([[0], np.cumsum(rc)])
    return [out[offs[q]:offs[q + 1]] for q in range(world)]


def allgather_rows(a: np.ndarray, group=None) -> list[np.ndarray]:
    """Every rank's row block (rows x w float64), in rank order."""
    world = dist.get_world_size(group)
    dev = _coll_device(group)
    n = torch.tensor([a.shape[0]], dtype=torch.int64, device=dev)
    ns = [torch.empty(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    ns = [int(t.item()) for t in ns]
    w = a.shape[1]
    mx = max(ns)
    buf = torch.zeros(mx * w, dtype=torch.float64, device=dev)
    if a.size:
        buf[:a.size] = torch.from_numpy(np.ascontiguousarray(a)).to(dev).reshape(-1)
    outs = [torch.empty(mx * w, dtype=torch.float64, device=dev) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return [o.cpu().numpy()[:k * w].reshape(k, w) for o, k in zip(outs, ns)]


def allreduce_max(v: float, group=None) -> float:
    t = torch.tensor([float(v)], dtype=torch.float64, device=_coll_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


# --------------------------------------------------------------------------
# per-rank compute on this rank's GPU
# --------------------------------------------------------------------------
class GpuBackend:
    """libsbv.so on one GPU: every step's arithmetic runs in its kernels;
    arrays cross this interface as host numpy arrays."""

    def __init__(self, ctx, dtype=torch.float64):
        self.ctx = ctx
        self.dtype = dtype

    def _dev(self, X):
        return torch.from_numpy(np.ascontiguousarray(X)).to(self.dtype).cuda()

    def slabs(self, X, beta_scale, P):
        return self.ctx.sbv_slabs(self._dev(X), beta_scale, P).cpu().numpy()

    def blocking_anchored(self, X, beta_scale, anchors, kmeans_iters):
        b = self.ctx.sbv_blocking_anchored(self._dev(X), beta_scale, anchors, kmeans_iters)
        return dict(ptr=b["ptr"].cpu().numpy(), pts=b["pts"].cpu().numpy(),
                    centres=b["centres"].cpu().numpy())

    def knn(self, X, beta_scale, ptr, pts, rank, centres, m):
        nbr, cnt = self.ctx.sbv_knn(
            self._dev(X), beta_scale, torch.from_numpy(ptr).cuda(),
            torch.from_numpy(pts.astype(np.int32)).cuda(),
            torch.from_numpy(rank.astype(np.int32)).cuda(), torch.from_numpy(centres).cuda(), m)
        return nbr.cpu().numpy(), cnt.cpu().numpy()

    def loglik_terms(self, X, y, ptr, pts, nbr, cnt, theta, nu2, precision):
        bc = cnt.size
        B = np.asarray(theta, dtype=np.float64).reshape(-1, 2 + X.shape[1]).shape[0]
        terms = torch.empty(B, bc, dtype=torch.float64, device="cuda")
        if bc:
            self.ctx.sbv_loglik(self._dev(X), torch.from_numpy(y).cuda(), torch.from_numpy(ptr).cuda(),
                                torch.from_numpy(pts.astype(np.int32)).cuda(),
                                torch.from_numpy(nbr.astype(np.int32)).cuda(),
                                torch.from_numpy(cnt.astype(np.int32)).cuda(), theta, nu2=nu2,
                                precision=precision, block_terms=terms)
        return terms.cpu().numpy()


# --------------------------------------------------------------------------
# Alg. 2 + 3 + Alg. 1 Step 2
# --------------------------------------------------------------------------
@dataclass
class LocalBlocks:
    gid: np.ndarray        # global ids of this rank's points, ascending
    X: np.ndarray          # their coordinates (n_local x d)
    y: np.ndarray          # their observations
    ptr: np.ndarray        # CSR over local points: block i = pts[ptr[i]:ptr[i+1]]
    pts: np.ndarray        # local point indices grouped by block, ascending inside a block
    centres: np.ndarray    # block centres (scaled space)
    block_id: np.ndarray   # global block number (slab by slab, as the single-GPU blocking)
    rank: np.ndarray       # global block order
    sizes_all: np.ndarray  # block sizes of every block, by global block number
    rank_all: np.ndarray   # block order of every block, by global block number


def _pack(gid, X, y):
    return np.column_stack([gid.astype(np.float64), y.astype(np.float64), X.astype(np.float64)])


def distributed_blocking(backend, X, y, gid, beta_scale, bc: int, kmeans_iters: int, seed: int,
                         group=None) -> LocalBlocks:
    """Alg. 2 routing, Alg. 3 on this rank's slab, the replayed block order."""
    world, me = dist.get_world_size(group), dist.get_rank(group)
    X = np.asarray(X)
    d = X.shape[1]
    slab = backend.slabs(X, beta_scale, world) if X.shape[0] else np.zeros(0, dtype=np.int32)
    rows = _pack(np.asarray(gid), X, np.asarray(y))
    got = np.concatenate(alltoall_rows([rows[slab == q] for q in range(world)], group), axis=0)
    got = got[np.argsort(got[:, 0], kind="stable")]
    lgid = got[:, 0].astype(np.int64)
    ly = got[:, 1].copy()
    lX = got[:, 2:].astype(X.dtype)
    counts = np.array([int(r[0, 0]) for r in allgather_rows(np.array([[lgid.size]], np.float64), group)])
    quota, pos, _ = rac_plan(seed, counts, bc)
    off = np.concatenate([[0], np.cumsum(quota)])
    if quota[me] > 0:
        b = backend.blocking_anchored(lX, beta_scale, pos[off[me]:off[me + 1]], kmeans_iters)
        ptr, pts, centres = b["ptr"], b["pts"].astype(np.int64), b["centres"]
    else:
        ptr, pts, centres = np.zeros(1, np.int64), np.zeros(0, np.int64), np.zeros((0, d))
    k = centres.shape[0]
    sizes = np.diff(ptr).astype(np.float64)[:, None]
    sizes_all = np.concatenate(allgather_rows(sizes, group), axis=0)[:, 0].astype(np.int64)
    ks = [int(r[0, 0]) for r in allgather_rows(np.array([[k]], np.float64), group)]
    first = sum(ks[:me])
    _, _, rank_all = rac_plan(seed, counts, bc, sum(ks))
    bid = np.arange(first, first + k, dtype=np.int64)
    return LocalBlocks(gid=lgid, X=lX, y=ly, ptr=ptr.astype(np.int64), pts=pts, centres=centres,
                       block_id=bid, rank=rank_all[bid].astype(np.int64), sizes_all=sizes_all,
                       rank_all=rank_all.astype(np.int64))


# --------------------------------------------------------------------------
# Alg. 4 (filtered neighbour search with the block exchange)
# --------------------------------------------------------------------------
def lambda_threshold(n: int, m: int, d: int, volume: float, alpha: float = 100.0) -> float:
    """Eq. distancethreshold read as the radius of a ball expected to hold
    alpha m of n candidate points spread over `volume` (the scaled data's
    bounding box):
    lambda = (alpha m zeta volume / n)^(1/d), zeta = Gamma(d/2 + 1) / pi^(d/2)
    (one over the unit ball's volume)."""
    zeta = math.gamma(d / 2 + 1) / math.pi ** (d / 2)
    return (alpha * m * zeta * max(volume, 1e-300) / max(n, 1)) ** (1.0 / d)


@dataclass
class LocalProblem:
    """This rank's blocks on its own points plus the received ones."""
    gid: np.ndarray        # global ids of the union's points, ascending
    X: np.ndarray
    y: np.ndarray
    ptr: np.ndarray        # this rank's blocks over union indices
    pts: np.ndarray
    nbr: np.ndarray        # union indices (-1 padded), m columns
    cnt: np.ndarray
    nbr_gid: np.ndarray    # the same neighbours as global ids
    rounds: int            # exchange rounds until every block was accepted
    received: int          # points received in the last round


def distributed_knn(backend, lb: LocalBlocks, beta_scale, m: int, alpha: float = 100.0,
                    group=None) -> LocalProblem:
    world, me = dist.get_world_size(group), dist.get_rank(group)
    beta = np.asarray(beta_scale, dtype=np.float64)
    d = lb.X.shape[1]
    k = lb.centres.shape[0]
    Z = lb.X.astype(np.float64) / beta
    # radius of every local block (largest distance of a member to its centre)
    rad = np.zeros(k)
    for i in range(k):
        mem = lb.pts[lb.ptr[i]:lb.ptr[i + 1]]
        if mem.size:
            rad[i] = math.sqrt(float(((Z[mem] - lb.centres[i]) ** 2).sum(axis=1).max()))
    # earlier-ordered points of every block (all of them when fewer than m)
    order = np.argsort(lb.rank_all, kind="stable")
    before = np.zeros(lb.rank_all.size, dtype=np.int64)
    before[order] = np.concatenate([[0], np.cumsum(lb.sizes_all[order])[:-1]])
    # Step 1: lambda of every local block from the scaled data's extent and its
    # number of earlier-ordered points (the candidates of Eq. mmsearchingBV)
    lo = Z.min(axis=0) if Z.shape[0] else np.full(d, np.inf)
    hi = Z.max(axis=0) if Z.shape[0] else np.full(d, -np.inf)
    lo = -np.array([allreduce_max(-v, group) for v in lo])
    hi = np.array([allreduce_max(v, group) for v in hi])
    vol = float(np.prod(np.maximum(hi - lo, 1e-12)))
    diam = float(np.sqrt(((hi - lo) ** 2).sum()))
    lam = np.array([lambda_threshold(max(int(before[b]), 1), m, d, vol, alpha)
                    for b in lb.block_id])
    rounds = 0
    while True:
        rounds += 1
        meta = np.column_stack([lb.rank.astype(np.float64), rad, lam, lb.centres]) if k else \
            np.zeros((0, 3 + d))
        allmeta = allgather_rows(meta, group)
        # Step 2: coarse candidates -- every block that may hold a point within
        # lambda_i of a later-ordered block i of the receiving rank
        parts = []
        for q in range(world):
            if q == me or k == 0 or allmeta[q].shape[0] == 0:
                parts.append(np.zeros((0, 3 + d)))
                continue
            rq, lq, cq = allmeta[q][:, 0], allmeta[q][:, 2], allmeta[q][:, 3:]
            send = np.zeros(k, dtype=bool)
            for j in range(k):
                later = rq > lb.rank[j]
                if not later.any():
                    continue
                dc = np.sqrt(((cq[later] - lb.centres[j]) ** 2).sum(axis=1))
                send[j] = bool((dc <= (lq[later] + rad[j]) * (1 + 1e-9)).any())
            sel = np.flatnonzero(send)
            idx = [lb.pts[lb.ptr[j]:lb.ptr[j + 1]] for j in sel]
            blk = [np.full(a.size, lb.block_id[j], dtype=np.float64) for a, j in zip(idx, sel)]
            idx = np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)
            blk = np.concatenate(blk) if blk else np.zeros(0)
            parts.append(np.column_stack([blk, _pack(lb.gid[idx], lb.X[idx], lb.y[idx])]))
        got = np.concatenate(alltoall_rows(parts, group), axis=0)
        # Step 3: the union of own and received points, ascending by global id
        ugid = np.concatenate([lb.gid, got[:, 1].astype(np.int64)])
        uX = np.concatenate([lb.X, got[:, 3:].astype(lb.X.dtype)], axis=0)
        uy = np.concatenate([lb.y, got[:, 2]])
        ublk = np.concatenate([lb.block_id[np.repeat(np.arange(k), np.diff(lb.ptr))][np.argsort(lb.pts)]
                               if k else np.zeros(0, np.int64), got[:, 0].astype(np.int64)])
        srt = np.argsort(ugid, kind="stable")
        ugid, uX, uy, ublk = ugid[srt], uX[srt], uy[srt], ublk[srt]
        bids = np.unique(ublk)
        local = np.searchsorted(bids, lb.block_id)
        ub = np.searchsorted(bids, ublk)
        cnts = np.bincount(ub, minlength=bids.size)
        uptr = np.concatenate([[0], np.cumsum(cnts)]).astype(np.int64)
        upts = np.argsort(ub, kind="stable").astype(np.int64)
        # the union's blocks keep their global relative order, renumbered 0..nb-1
        urank = np.empty(bids.size, dtype=np.int64)
        urank[np.argsort(lb.rank_all[bids], kind="stable")] = np.arange(bids.size)
        ucent = np.zeros((bids.size, d))
        if k:
            ucent[local] = lb.centres
        for q in range(world):
            if q == me or allmeta[q].shape[0] == 0:
                continue
            first = int(sum(a.shape[0] for a in allmeta[:q]))
            qb = np.arange(first, first + allmeta[q].shape[0])
            hit = np.isin(qb, bids)
            ucent[np.searchsorted(bids, qb[hit])] = allmeta[q][hit, 3:]
        nbr, cnt = backend.knn(uX, beta, uptr, upts, urank, ucent, m) if bids.size else \
            (np.zeros((0, m), np.int32), np.zeros(0, np.int32))
        nbr, cnt = nbr[local], cnt[local]
        # acceptance: all earlier points found, or the m-th neighbour within
        # lambda_i (then every nearer earlier point is a candidate); a failing
        # block doubles its lambda for the next round
        uZ = uX.astype(np.float64) / beta
        fail = np.zeros(k, dtype=bool)
        for i in range(k):
            nb = int(before[lb.block_id[i]])
            if cnt[i] != min(m, nb):
                fail[i] = True
            elif nb > m and m > 0:
                dm = math.sqrt(float(((uZ[nbr[i, m - 1]] - lb.centres[i]) ** 2).sum()))
                fail[i] = dm > lam[i] * (1 - 1e-9)
        lam[fail] *= 2.0
        if allreduce_max(float(fail.any()), group) == 0.0:
            break
        if rounds > 64 + int(math.log2(max(diam, 1.0) + 1.0)):
            raise RuntimeError("distributed_knn: lambda schedule did not converge")
    lptr = np.concatenate([[0], np.cumsum([cnts[j] for j in local])]).astype(np.int64)
    lpts = np.concatenate([upts[uptr[j]:uptr[j + 1]] for j in local]) if k else np.zeros(0, np.int64)
    ngid = np.where(nbr >= 0, ugid[np.maximum(nbr, 0)], -1)
    return LocalProblem(gid=ugid, X=uX, y=uy, ptr=lptr, pts=lpts, nbr=nbr, cnt=cnt, nbr_gid=ngid,
                        rounds=rounds, received=int(got.shape[0]))


def distributed_loglik(backend, lp: LocalProblem, theta, nu2: int = 5, precision="fp64",
                       group=None):
    """Alg. 1 Steps 4-5: this rank's block terms, and the per-theta total
    with the ranks' partial sums added in rank order (bit-identical on every
    rank)."""
    terms = backend.loglik_terms(lp.X, lp.y, lp.ptr, lp.pts, lp.nbr, lp.cnt, theta, nu2, precision)
    part = terms.sum(axis=1) if terms.size else np.zeros(terms.shape[0])
    parts = allgather_rows(part[None, :], group)
    tot = np.zeros_like(part)
    for p in parts:
        tot = tot + p[0]
    return tot, terms
