"""sbv_loglik_fp64_noalloc, the allocation-free variant, against sbv_loglik.

The entry point serves callers that may not allocate device memory while they
run (memory owned by another allocator, or loops that cannot afford
cudaMalloc's synchronisation); its scratch is a fixed device array inside
libsbv.so.  Two calls in a row, with different parameter rows, must give the
FP64 path's results.  This file is collected last so that a failure here
leaves every other test already run; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9  # |dl| / n, the FP64 bar of the parity tests


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_matches_loglik_on_two_calls():
    from paper_2504_12004_gb300 import build, Context, _lib
    from synth.inputs import workload

    build.build()
    lib = _lib.load()
    ctx = Context(0)
    w = workload("sine10d", n=20000, bc=400, m=60)
    X = torch.from_numpy(w["X"]).cuda()
    y = torch.from_numpy(w["y"]).cuda()
    b = ctx.sbv_blocking(X, w["beta_scale"], w["bc"], 3, 11)
    nbr, cnt = ctx.sbv_knn(X, w["beta_scale"], b["ptr"], b["pts"], b["rank"], b["centres"], w["m"])
    nbr = nbr.contiguous()
    n, d = X.shape
    bc, m = cnt.numel(), nbr.shape[1]
    th1 = np.repeat(w["theta"], 2, axis=0)
    th1[1, 0] *= 1.3
    th2 = th1.copy()
    th2[:, 1] *= 2.0
    th2[:, 2:] *= 0.8
    refs = [ctx.sbv_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, th, nu2=5, precision="fp64")
            for th in (th1, th2)]
    torch.cuda.synchronize()

    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for th in (th1, th2):  # two calls in a row on the same fixed scratch
        th = np.ascontiguousarray(th, dtype=np.float64)
        ll = torch.empty(th.shape[0], dtype=torch.float64, device="cuda")
        rc = lib.sbv_loglik_fp64_noalloc(
            _p(X), 0, _p(y), n, d, _p(b["ptr"]), _p(b["pts"]), _p(nbr), _p(cnt), bc, m, 0,
            th.ctypes.data_as(C.c_void_p), th.shape[0], 5, _p(ll), None, None, stream)
        assert rc == 0
        outs.append(ll)
    torch.cuda.synchronize()
    for ref, out in zip(refs, outs):
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - r)) / n <= TOL_FP64, (o, r)


def _structure(ctx, n, bc, m, seed):
    from synth.inputs import workload
    w = workload("sine10d", n=n, bc=bc, m=m)
    X = torch.from_numpy(w["X"]).cuda()
    y = torch.from_numpy(w["y"]).cuda()
    b = ctx.sbv_blocking(X, w["beta_scale"], w["bc"], 3, seed)
    nbr, cnt = ctx.sbv_knn(X, w["beta_scale"], b["ptr"], b["pts"], b["rank"], b["centres"], w["m"])
    return w, X, y, b, nbr.contiguous(), cnt


def _noalloc(lib, X, y, b, nbr, cnt, th, nu2):
    th = np.ascontiguousarray(th, dtype=np.float64)
    ll = torch.empty(th.shape[0], dtype=torch.float64, device="cuda")
    n, d = X.shape
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.sbv_loglik_fp64_noalloc(
        _p(X), 0, _p(y), n, d, _p(b["ptr"]), _p(b["pts"]), _p(nbr), _p(cnt), cnt.numel(),
        nbr.shape[1], 0, th.ctypes.data_as(C.c_void_p), th.shape[0], nu2, _p(ll), None, None,
        stream)
    return rc, ll


def test_noalloc_general_smoothness():
    # nu = 2 (nu2 = 4) goes through the Bessel form of the FP64 kernel, as in sbv_loglik
    from paper_2504_12004_gb300 import build, Context, _lib

    build.build()
    lib = _lib.load()
    ctx = Context(0)
    w, X, y, b, nbr, cnt = _structure(ctx, 8000, 160, 30, 5)
    th = w["theta"]
    ref = ctx.sbv_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, th, nu2=4, precision="fp64")
    rc, ll = _noalloc(lib, X, y, b, nbr, cnt, th, 4)
    torch.cuda.synchronize()
    assert rc == 0
    assert np.max(np.abs(ll.cpu().numpy() - ref.cpu().numpy())) / X.shape[0] <= TOL_FP64


def test_loglik_after_noalloc_with_larger_blocks():
    # a small no-alloc call must leave sbv_loglik's FP64 kernel able to take
    # blocks that need more shared memory later in the same process
    from paper_2504_12004_gb300 import build, Context, _lib

    build.build()
    lib = _lib.load()
    ctx = Context(0)
    w1, X1, y1, b1, nbr1, cnt1 = _structure(ctx, 4000, 400, 8, 3)
    # sbv_loglik first (its one-time set-up of the kernel), then the small
    # no-alloc call, then sbv_loglik with blocks of ~170 points
    ctx.sbv_loglik(X1, y1, b1["ptr"], b1["pts"], nbr1, cnt1, w1["theta"], nu2=5, precision="fp64")
    rc, _ = _noalloc(lib, X1, y1, b1, nbr1, cnt1, w1["theta"], 5)
    torch.cuda.synchronize()
    assert rc == 0
    w2, X2, y2, b2, nbr2, cnt2 = _structure(ctx, 20000, 400, 120, 4)
    got = ctx.sbv_loglik(X2, y2, b2["ptr"], b2["pts"], nbr2, cnt2, w2["theta"], nu2=5,
                         precision="fp64")
    rc, ll = _noalloc(lib, X2, y2, b2, nbr2, cnt2, w2["theta"], 5)
    torch.cuda.synchronize()
    assert rc == 0
    ctx.sbv_sync_status()
    g, o = got.cpu().numpy(), ll.cpu().numpy()
    assert np.all(np.isfinite(g))
    assert np.max(np.abs(g - o)) / X2.shape[0] <= TOL_FP64


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2504_12004_gb300 import build, _lib

    build.build()
    lib = _lib.load()
    torch.cuda.init()
    one = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    pts = torch.arange(4, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    too_many = np.tile(np.array([1.0, 0.1, 1.0]), (65, 1))  # 65 > SBV_NOALLOC_MAX_THETA rows
    rc = lib.sbv_loglik_fp64_noalloc(_p(one), 0, _p(one), 4, 1, _p(ptr), _p(pts), None, _p(cnt),
                                     1, 0, 4, too_many.ctypes.data_as(C.c_void_p), 65, 5, _p(one),
                                     None, None, None)
    assert rc == 6  # SBV_EUNSUPPORTED, before any work
