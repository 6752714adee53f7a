"""FP64 reference of the likelihood surrogate network (test infrastructure only).

The paper has no learned component.  The surrogate s(u) approximates the
standardised SBV log-likelihood as a function of u = standardised log theta,
so that an optimiser can ask it for candidate parameters; the exact
likelihood (Alg. 5 summed as in Alg. 1 Step 5) judges every candidate.

Network (fixed by the method's design, not by the paper):
    in_dim -> 256 -> 256 -> 256 -> 1, GELU after each hidden layer,
    GELU(z) = z * Phi(z) with Phi the standard normal CDF (erf form).
Loss: L = (1/K) sum_k (s(x_k) - t_k)^2 over the K rows of a batch.
Optimiser: Adam (Kingma & Ba, ICLR 2015, Algorithm 1) with bias correction.

Precision model of the GPU kernels, reproduced here when emulate=True:
the two 256x256 layers take BF16 operands (weights, activations, and in the
backward pass the pre-activation gradients) with products summed exactly
(FP64 here, FP32 on the GPU); everything else -- the input layer, biases,
GELU and its derivative, the output layer, the bias and input-layer weight
gradients, Adam -- is unrounded.  With emulate=False every step is plain
FP64.  BF16 rounding is round-to-nearest-even applied to the FP32 value,
i.e. the value is rounded to FP32 first and then to 8 significant bits.

Parameters are a dict of FP64 arrays: W1 (256, in), b1 (256), W2, W3
(256, 256), b2, b3 (256), w4 (256), b4 (scalar array of shape ()).
Weights are stored [out][in]; a layer computes z = h W^T + b.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .prng import SplitMix64

WIDTH = 256
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")


# --------------------------------------------------------------------------
# rounding and activation
# --------------------------------------------------------------------------
def bf16(x):
    """Round to FP32 (nearest-even), then to BF16 (nearest-even on the 16 dropped bits)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    """z * Phi(z), Phi(z) = (1 + erf(z / sqrt 2)) / 2."""
    return z * 0.5 * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z), phi the standard normal density."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
def shapes(in_dim: int) -> dict:
    return {"W1": (WIDTH, in_dim), "b1": (WIDTH,), "W2": (WIDTH, WIDTH), "b2": (WIDTH,),
            "W3": (WIDTH, WIDTH), "b3": (WIDTH,), "w4": (WIDTH,), "b4": ()}


def fan_in(name: str, in_dim: int) -> int:
    return {"W1": in_dim, "b1": in_dim, "W2": WIDTH, "b2": WIDTH, "W3": WIDTH, "b3": WIDTH,
            "w4": WIDTH, "b4": WIDTH}[name]


def init_params(in_dim: int, seed: int) -> dict:
    """Uniform(-a, a), a = 1/sqrt(fan_in), from one SplitMix64 stream.

    Tensors are drawn in the order W1 b1 W2 b2 W3 b3 w4 b4, each row-major;
    one draw u = (next() >> 11) * 2^-53 gives the value (2u - 1) a, stored as
    the nearest FP32 (the master precision of the GPU copy).
    """
    rng = SplitMix64(seed)
    P = {}
    for name in ORDER:
        shp = shapes(in_dim)[name]
        a = 1.0 / math.sqrt(fan_in(name, in_dim))
        cnt = int(np.prod(shp)) if shp else 1
        vals = np.empty(cnt)
        for i in range(cnt):
            u = (rng.next() >> 11) * (2.0 ** -53)
            vals[i] = (2.0 * u - 1.0) * a
        P[name] = vals.astype(np.float32).astype(np.float64).reshape(shp)
    return P


def pack(P: dict) -> np.ndarray:
    return np.concatenate([np.asarray(P[k], dtype=np.float64).ravel() for k in ORDER])


def unpack(v: np.ndarray, in_dim: int) -> dict:
    P, o = {}, 0
    for name in ORDER:
        shp = shapes(in_dim)[name]
        cnt = int(np.prod(shp)) if shp else 1
        P[name] = np.asarray(v[o:o + cnt], dtype=np.float64).reshape(shp)
        o += cnt
    return P


# --------------------------------------------------------------------------
# forward / backward
# --------------------------------------------------------------------------
def forward(P: dict, X, emulate: bool = False) -> dict:
    """Forward pass over the rows of X; returns every intermediate and s."""
    r = bf16 if emulate else (lambda a: a)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ P["W1"].T + P["b1"]
    H1 = gelu(Z1)
    Z2 = r(H1) @ r(P["W2"]).T + P["b2"]
    H2 = gelu(Z2)
    Z3 = r(H2) @ r(P["W3"]).T + P["b3"]
    H3 = gelu(Z3)
    s = H3 @ P["w4"] + P["b4"]
    return dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Z3=Z3, H3=H3, s=s)


def backward(P: dict, c: dict, ds, emulate: bool = False) -> tuple[dict, np.ndarray]:
    """Gradients of sum_k ds_k s_k with respect to every parameter and to X."""
    r = bf16 if emulate else (lambda a: a)
    ds = np.asarray(ds, dtype=np.float64)
    G = {}
    G["w4"] = c["H3"].T @ ds
    G["b4"] = np.asarray(ds.sum())
    dZ3 = np.outer(ds, P["w4"]) * gelu_prime(c["Z3"])
    G["W3"] = r(dZ3).T @ r(c["H2"])
    G["b3"] = dZ3.sum(0)
    dZ2 = (r(dZ3) @ r(P["W3"])) * gelu_prime(c["Z2"])
    G["W2"] = r(dZ2).T @ r(c["H1"])
    G["b2"] = dZ2.sum(0)
    dZ1 = (r(dZ2) @ r(P["W2"])) * gelu_prime(c["Z1"])
    G["W1"] = dZ1.T @ c["X"]
    G["b1"] = dZ1.sum(0)
    dX = dZ1 @ P["W1"]
    return G, dX


def mse_loss_grads(P: dict, X, t, emulate: bool = False):
    """L = mean_k (s_k - t_k)^2 and its gradients (ds_k = 2 (s_k - t_k) / K)."""
    c = forward(P, X, emulate)
    t = np.asarray(t, dtype=np.float64)
    K = len(t)
    res = c["s"] - t
    L = float(res @ res) / K
    G, _ = backward(P, c, 2.0 * res / K, emulate)
    return L, G


def predict(P: dict, X, emulate: bool = False):
    """s(x) and ds/dx for every row."""
    c = forward(P, X, emulate)
    _, dX = backward(P, c, np.ones(len(c["s"])), emulate)
    return c["s"], dX


# --------------------------------------------------------------------------
# Adam
# --------------------------------------------------------------------------
def adam_init(P: dict) -> dict:
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in P.items()},
            "v": {k: np.zeros_like(v) for k, v in P.items()}}


def adam_step(P: dict, G: dict, S: dict, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place: moments, bias correction, p -= lr m_hat / (sqrt(v_hat) + eps)."""
    S["t"] += 1
    t = S["t"]
    for k in ORDER:
        m = beta1 * S["m"][k] + (1.0 - beta1) * G[k]
        v = beta2 * S["v"][k] + (1.0 - beta2) * G[k] * G[k]
        S["m"][k], S["v"][k] = m, v
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        P[k] = P[k] - lr * mhat / (np.sqrt(vhat) + eps)
