"""Graph-captured evaluation and the launch-shape autotuner, through the C ABI.

A captured evaluation replayed with new parameter rows must give exactly what
sbv_loglik gives with the same launch shape (the block terms and their fixed
order sum are deterministic); after autotuning, sbv_loglik must still meet the
parity bar of its precision.
"""
import numpy as np
import pytest
import torch

from synth.inputs import workload

pytestmark = pytest.mark.gpu

TOLS = {"fp64": 1e-9, "mixed": 1e-6, "mixed_bf16": 1e-6}  # |dl| / n


@pytest.fixture(scope="module")
def setup():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    ctx = Context(0)
    w = workload("sine10d", n=20000, bc=400, m=60)
    X = torch.from_numpy(w["X"]).cuda()
    y = torch.from_numpy(w["y"]).cuda()
    b = ctx.sbv_blocking(X, w["beta_scale"], w["bc"], 3, 11)
    nbr, cnt = ctx.sbv_knn(X, w["beta_scale"], b["ptr"], b["pts"], b["rank"], b["centres"], w["m"])
    nbr = nbr.contiguous()
    th1 = np.repeat(w["theta"], 3, axis=0)
    th1[1, 0] *= 1.3
    th1[2, 2:] *= 1.2
    th2 = th1.copy()
    th2[:, 1] *= 2.0
    th2[:, 2:] *= 0.8
    return dict(ctx=ctx, X=X, y=y, b=b, nbr=nbr, cnt=cnt, th=(th1, th2), n=w["X"].shape[0])


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
def test_graph_replay_equals_loglik(setup, precision):
    s = setup
    ctx, b = s["ctx"], s["b"]
    refs = [ctx.sbv_loglik(s["X"], s["y"], b["ptr"], b["pts"], s["nbr"], s["cnt"], th, nu2=5,
                           precision=precision).clone() for th in s["th"]]
    g = ctx.sbv_loglik_graph_create(s["X"], s["y"], b["ptr"], b["pts"], s["nbr"], s["cnt"],
                                    B=s["th"][0].shape[0], nu2=5, precision=precision)
    try:
        outs = []
        for rep in range(2):  # each set twice, alternating: the staging must not mix rows up
            for th in s["th"]:
                outs.append(g.launch(th).clone())
        torch.cuda.synchronize()
        ctx.sbv_sync_status()
    finally:
        g.close()
    for k, out in enumerate(outs):
        ref = refs[k % 2]
        assert torch.equal(out, ref), (precision, k, (out - ref).abs().max().item())


def test_graph_general_smoothness_fp64(setup):
    # the captured FP64 kernel takes any nu = nu2/2 (Eq. maternkernel through
    # K_nu) exactly as sbv_loglik does; the mixed precisions keep the closed forms
    from paper_2504_12004_gb300 import SBVError
    s = setup
    ctx, b = s["ctx"], s["b"]
    th = s["th"][0]
    ref = ctx.sbv_loglik(s["X"], s["y"], b["ptr"], b["pts"], s["nbr"], s["cnt"], th, nu2=4,
                         precision="fp64").clone()
    g = ctx.sbv_loglik_graph_create(s["X"], s["y"], b["ptr"], b["pts"], s["nbr"], s["cnt"],
                                    B=th.shape[0], nu2=4, precision="fp64")
    try:
        out = g.launch(th).clone()
        torch.cuda.synchronize()
    finally:
        g.close()
    assert torch.equal(out, ref)
    with pytest.raises(SBVError):
        ctx.sbv_loglik_graph_create(s["X"], s["y"], b["ptr"], b["pts"], s["nbr"], s["cnt"],
                                    B=th.shape[0], nu2=4, precision="mixed")


def test_graph_rejects_bad_rows(setup):
    from paper_2504_12004_gb300 import SBVError
    s = setup
    b = s["b"]
    g = s["ctx"].sbv_loglik_graph_create(s["X"], s["y"], b["ptr"], b["pts"], s["nbr"], s["cnt"],
                                         B=3, nu2=5, precision="mixed")
    try:
        bad = s["th"][0].copy()
        bad[1, 0] = -1.0
        with pytest.raises(SBVError):
            g.launch(bad)
        good = g.launch(s["th"][0])
        torch.cuda.synchronize()
        assert torch.isfinite(good).all()
    finally:
        g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_parity(setup, precision):
    s = setup
    ctx, b = s["ctx"], s["b"]
    th = s["th"][0]
    args = (s["X"], s["y"], b["ptr"], b["pts"], s["nbr"], s["cnt"])
    before = ctx.sbv_loglik(*args, th, nu2=5, precision="fp64").clone()
    threads, per_sm = ctx.sbv_autotune(*args, th, nu2=5, precision=precision)
    assert threads in (256, 512) and 1 <= per_sm <= 4
    after = ctx.sbv_loglik(*args, th, nu2=5, precision=precision)
    torch.cuda.synchronize()
    err = ((after - before).abs() / s["n"]).max().item()
    assert err <= TOLS[precision], err
