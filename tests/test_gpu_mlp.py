"""Surrogate network kernels (tcgen05 BF16 layers) against the FP64 oracle.

The oracle's emulate mode rounds to BF16 exactly where the kernels do, so
the remaining difference is FP32 accumulation order and the odd BF16 rounding
that flips on an FP32-vs-FP64 difference: gradients agree to ~1e-5 relative
(bar 1e-3).  Against plain FP64 (no rounding) the BF16 operands cost about the
BF16 unit, 2^-8 (bar 3e-2).
"""
import numpy as np
import pytest
import torch

from oracle import mlp as om
from oracle.prng import SplitMix64, full_shuffle

pytestmark = pytest.mark.gpu

TOL_EMU = 1e-3     # relative Frobenius error per tensor vs the BF16-emulating oracle
TOL_FP64 = 3e-2    # vs the unrounded FP64 oracle


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def data(K, in_dim, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((K, in_dim)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.3 * X[:, 1] ** 2 - 0.5 * X[:, 2 % in_dim] * X[:, 3 % in_dim]
         + 0.1 * rng.standard_normal(K)).astype(np.float32)
    return X, t


def test_init_matches_oracle_bit_exact(ctx):
    from paper_2504_12004_gb300 import Mlp
    net = Mlp(ctx, 12, seed=99)
    want = om.pack(om.init_params(12, 99)).astype(np.float32)
    assert np.array_equal(net.get_params(), want)


@pytest.mark.parametrize("K,in_dim", [(300, 12), (128, 5), (20000, 12)])
def test_gradients_match_oracle(ctx, K, in_dim):
    from paper_2504_12004_gb300 import Mlp
    net = Mlp(ctx, in_dim, seed=7)
    X, t = data(K, in_dim, K)
    g, loss = net.grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    P = om.unpack(net.get_params().astype(np.float64), in_dim)
    L_emu, G_emu = om.mse_loss_grads(P, X.astype(np.float64), t.astype(np.float64), emulate=True)
    L_64, G_64 = om.mse_loss_grads(P, X.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - L_emu) <= 1e-5 * L_emu
    Gg = om.unpack(g, in_dim)
    for k in om.ORDER:
        assert rel(Gg[k], G_emu[k]) <= TOL_EMU, (k, rel(Gg[k], G_emu[k]))
        assert rel(Gg[k], G_64[k]) <= TOL_FP64, (k, rel(Gg[k], G_64[k]))


def test_adam_step_matches_oracle(ctx):
    from paper_2504_12004_gb300 import Mlp
    net = Mlp(ctx, 12, seed=3)
    X, t = data(500, 12, 1)
    p0 = net.get_params().astype(np.float64)
    g, _ = net.grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    net.adam(1e-3)
    p1 = net.get_params().astype(np.float64)
    P = om.unpack(p0, 12)
    S = om.adam_init(P)
    om.adam_step(P, om.unpack(g.cpu().numpy().astype(np.float64), 12), S, 1e-3)
    want = om.pack(P)
    assert np.all(np.abs(p1 - want) <= 2e-7 * np.abs(want) + 1e-9)
    # the refreshed BF16 copies are used by the next pass: the gradient moves
    g2, _ = net.grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    L_emu, G_emu = om.mse_loss_grads(om.unpack(p1, 12), X.astype(np.float64), t.astype(np.float64),
                                     emulate=True)
    assert rel(g2.cpu().numpy(), om.pack(G_emu)) <= TOL_EMU


def test_predict_and_input_gradient(ctx):
    from paper_2504_12004_gb300 import Mlp
    net = Mlp(ctx, 12, seed=5)
    X, _ = data(333, 12, 2)
    s, dx = net.predict(torch.from_numpy(X).cuda(), want_grad=True)
    P = om.unpack(net.get_params().astype(np.float64), 12)
    s_e, dx_e = om.predict(P, X.astype(np.float64), emulate=True)
    # s sums 256 FP32 products; an FP32-vs-FP64 difference can flip one BF16
    # rounding of H2 (a 2^-8 change of one operand), ~3e-5 of s measured
    assert rel(s.cpu().numpy(), s_e) <= 1e-4
    assert rel(dx.cpu().numpy(), dx_e) <= TOL_EMU
    s_only = net.predict(torch.from_numpy(X).cuda())
    assert torch.equal(s_only, s)


def test_training_tracks_oracle(ctx):
    from paper_2504_12004_gb300 import Mlp
    K, in_dim, steps, batch, lr, seed = 2048, 12, 60, 256, 2e-3, 11
    X, t = data(K, in_dim, 4)
    net = Mlp(ctx, in_dim, seed=21)
    L0 = float(np.mean((net.predict(torch.from_numpy(X).cuda()).cpu().numpy() - t) ** 2))
    net.train(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), steps, batch, lr, seed)
    L_gpu = float(np.mean((net.predict(torch.from_numpy(X).cuda()).cpu().numpy() - t) ** 2))
    # the oracle takes the same mini-batches from the same SplitMix64 stream
    P = om.init_params(in_dim, 21)
    S = om.adam_init(P)
    rng = SplitMix64(seed)
    perm, pos = None, K
    X64, t64 = X.astype(np.float64), t.astype(np.float64)
    for _ in range(steps):
        if pos >= K:
            perm, pos = np.array(full_shuffle(K, rng)), 0
        b = perm[pos:pos + batch]
        pos += len(b)
        _, G = om.mse_loss_grads(P, X64[b], t64[b])
        om.adam_step(P, G, S, lr)
    L_or = float(np.mean((om.forward(P, X64)["s"] - t64) ** 2))
    assert L_gpu < 0.5 * L0 and L_or < 0.5 * L0
    assert abs(L_gpu - L_or) <= 0.1 * L_or, (L0, L_gpu, L_or)


def test_invalid_arguments(ctx):
    from paper_2504_12004_gb300 import Mlp, SBVError
    with pytest.raises(SBVError):
        Mlp(ctx, 0)
    with pytest.raises(SBVError):
        Mlp(ctx, 17)
    net = Mlp(ctx, 4)
    with pytest.raises(SBVError):
        net.adam(1e-3)      # no gradient yet
    with pytest.raises(SBVError):
        net.set_params(np.zeros(3, dtype=np.float32))
