"""Pins of oracle.mlp against mathematics that does not come from the oracle itself.

- GELU: Phi(1) from the standard normal table, the identity
  GELU(z) - GELU(-z) = z, and torch's own GELU (a separate implementation).
- Backward: central finite differences of the FP64 loss, and torch.autograd
  on a float64 torch network built from the same parameters.
- BF16 rounding: round-to-nearest-even cases worked out by hand, and torch's
  float32 -> bfloat16 conversion.
- Adam: with a constant gradient the bias-corrected moments are exactly g and
  g^2, so every step moves p by -lr g / (|g| + eps).
- Initialisation: the SplitMix64 draws reproduce the stream pinned in
  tests/golden, and every value lies in (-1/sqrt(fan_in), 1/sqrt(fan_in)).
"""
import math

import numpy as np
import pytest
import torch

from oracle import mlp
from oracle.prng import SplitMix64


def small_problem(seed=3, K=9, in_dim=12):
    P = mlp.init_params(in_dim, seed)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((K, in_dim))
    t = rng.standard_normal(K)
    return P, X, t


def test_gelu_values_and_identity():
    assert mlp.gelu(np.array(0.0)) == 0.0
    # Phi(1) = 0.841344746068543 (standard normal table)
    assert abs(mlp.gelu(np.array(1.0)) - 0.841344746068543) < 1e-15
    z = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-14)
    assert np.allclose(mlp.gelu(z), torch.nn.functional.gelu(torch.tensor(z)).numpy(), atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_prime(z), fd, atol=1e-9)


def test_backward_matches_finite_differences():
    P, X, t = small_problem()
    L, G = mlp.mse_loss_grads(P, X, t)
    rng = np.random.default_rng(0)
    h = 1e-6
    for name in mlp.ORDER:
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name].reshape(-1)[idx] += h
            Pm[name].reshape(-1)[idx] -= h
            fd = (mlp.mse_loss_grads(Pp, X, t)[0] - mlp.mse_loss_grads(Pm, X, t)[0]) / (2 * h)
            an = np.asarray(G[name]).reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (name, idx, fd, an)
    # input gradient of s
    s, dX = mlp.predict(P, X)
    for j in range(X.shape[1]):
        Xp, Xm = X.copy(), X.copy()
        Xp[:, j] += h
        Xm[:, j] -= h
        fd = (mlp.forward(P, Xp)["s"] - mlp.forward(P, Xm)["s"]) / (2 * h)
        assert np.allclose(dX[:, j], fd, atol=1e-8)


def test_backward_matches_torch_autograd():
    P, X, t = small_problem(seed=5, K=17)
    L, G = mlp.mse_loss_grads(P, X, t)
    T = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in P.items()}
    x = torch.tensor(X)
    h = torch.nn.functional.gelu(x @ T["W1"].T + T["b1"])
    h = torch.nn.functional.gelu(h @ T["W2"].T + T["b2"])
    h = torch.nn.functional.gelu(h @ T["W3"].T + T["b3"])
    s = h @ T["w4"] + T["b4"]
    loss = ((s - torch.tensor(t)) ** 2).mean()
    loss.backward()
    assert abs(loss.item() - L) < 1e-13 * max(1, abs(L))
    for k in mlp.ORDER:
        assert np.allclose(T[k].grad.numpy(), G[k], rtol=1e-10, atol=1e-14), k


def test_bf16_rounding():
    one = 1.0
    assert mlp.bf16(one + 2.0 ** -8) == 1.0                      # tie -> even mantissa 0
    assert mlp.bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6      # tie -> even mantissa 2
    assert mlp.bf16(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7  # above the tie
    assert mlp.bf16(-(one + 2.0 ** -8 + 2.0 ** -20)) == -(one + 2.0 ** -7)
    x = np.random.default_rng(1).standard_normal(10000) * 10.0 ** np.random.default_rng(2).uniform(-5, 5, 10000)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_emulated_precision_is_close_to_fp64():
    # BF16 operands change the gradients by about the BF16 unit (2^-8 relative)
    P, X, t = small_problem(seed=7, K=64)
    _, G = mlp.mse_loss_grads(P, X, t)
    _, Ge = mlp.mse_loss_grads(P, X, t, emulate=True)
    for k in mlp.ORDER:
        rel = np.linalg.norm(np.ravel(G[k] - Ge[k])) / np.linalg.norm(np.ravel(G[k]))
        assert 0.0 < rel < 3e-2 or k in ("w4", "b4"), (k, rel)


def test_adam_constant_gradient_closed_form():
    P = {"W1": np.array([[0.5, -0.25]]), "b1": np.array([0.0]), "W2": np.zeros((1, 1)),
         "b2": np.zeros(1), "W3": np.zeros((1, 1)), "b3": np.zeros(1), "w4": np.zeros(1),
         "b4": np.zeros(())}
    g = {"W1": np.array([[2.0, -1e-3]]), "b1": np.array([0.3]), "W2": np.full((1, 1), 5.0),
         "b2": np.full(1, -7.0), "W3": np.full((1, 1), 1e-6), "b3": np.full(1, 1.0),
         "w4": np.full(1, -2.0), "b4": np.full((), 4.0)}
    P0 = {k: v.copy() for k, v in P.items()}
    S = mlp.adam_init(P)
    lr, eps, steps = 1e-2, 1e-8, 25
    for _ in range(steps):
        mlp.adam_step(P, g, S, lr, eps=eps)
    for k in mlp.ORDER:
        want = P0[k] - steps * lr * g[k] / (np.abs(g[k]) + eps)
        assert np.allclose(P[k], want, rtol=0, atol=1e-12), k


def test_init_stream_and_bounds():
    P = mlp.init_params(12, 99)
    rng = SplitMix64(99)
    u = (rng.next() >> 11) * 2.0 ** -53
    assert P["W1"][0, 0] == float(np.float32((2 * u - 1) / math.sqrt(12)))
    for k in mlp.ORDER:
        a = 1.0 / math.sqrt(mlp.fan_in(k, 12))
        assert np.all(np.abs(P[k]) < a * (1 + 1e-7)), k
        assert P[k].shape == mlp.shapes(12)[k]
    v = mlp.pack(P)
    assert v.size == 256 * 12 + 256 + 2 * (256 * 256 + 256) + 256 + 1
    Q = mlp.unpack(v, 12)
    assert all(np.array_equal(P[k], Q[k]) for k in mlp.ORDER)
    assert np.array_equal(mlp.pack(mlp.init_params(12, 99)), v)   # deterministic
