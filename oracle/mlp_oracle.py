"""Reference of the apparent-viscosity surrogate network (test infrastructure).

The network and its training are a build component (the paper has no
surrogate): a multilayer perceptron 3 -> 128 -> 128 -> 128 -> 128 -> 1 with
GELU activations (erf form) and an MSE loss, trained by Adam (Kingma & Ba).
Layers 2-4 (128 x 128) run on tensor cores on the GPU with BF16 operands and
FP32 accumulation; the input and output layers and all element-wise work are
FP32.  This module computes the same quantities with numpy:

  precision="bf16": the GPU's rounding points reproduced (weights of layers
                    2-4 and the inputs of those GEMMs rounded to BF16 with
                    round-to-nearest-even, everything else float64)
  precision="fp64": no rounding, for finite-difference pins.

Only the tests may import this module.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

WIDTH = 128
N_IN = 3


def bf16(a):
    """Round float values to bfloat16 (round to nearest, ties to even)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(f), f, out).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int, width: int = WIDTH) -> dict:
    """He-style uniform initialisation, seeded (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    p = {}
    dims = [(width, N_IN), (width, width), (width, width), (width, width), (1, width)]
    for k, (o, i) in enumerate(dims):
        lim = math.sqrt(6.0 / i)
        p[f"W{k}"] = rng.uniform(-lim, lim, size=(o, i))
        p[f"b{k}"] = np.zeros(o)
    return p


def forward(p: dict, X, precision="bf16"):
    """Returns y [B] and the cache for backward."""
    rnd = bf16 if precision == "bf16" else (lambda a: np.asarray(a, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z = [None] * 5
    a = [None] * 5
    z[0] = X @ p["W0"].T + p["b0"]
    h = gelu(z[0])
    for k in (1, 2, 3):
        a[k - 1] = rnd(h)                       # GEMM input of layer k
        z[k] = a[k - 1] @ rnd(p[f"W{k}"]).T + p[f"b{k}"]
        h = gelu(z[k])
    a[3] = h                                    # output layer input (FP32)
    y = h @ p["W4"][0] + p["b4"][0]
    return y, {"X": X, "z": z, "a": a, "precision": precision}


def loss(y, t):
    return float(np.mean((np.asarray(y) - np.asarray(t)) ** 2))


def backward(p: dict, cache: dict, y, t) -> dict:
    """Gradients of the mean squared error with respect to every parameter,
    with the same rounding points as the forward (GEMM operands of layers 2-4
    in BF16 when precision == "bf16")."""
    rnd = bf16 if cache["precision"] == "bf16" else (lambda a: np.asarray(a, dtype=np.float64))
    z, a, X = cache["z"], cache["a"], cache["X"]
    B = len(y)
    g = {}
    dy = 2.0 * (np.asarray(y) - np.asarray(t)) / B
    g["W4"] = (dy @ a[3])[None, :]
    g["b4"] = np.array([dy.sum()])
    dz = (dy[:, None] * p["W4"][0][None, :]) * gelu_prime(z[3])
    for k in (3, 2, 1):
        dzr = rnd(dz)
        g[f"W{k}"] = dzr.T @ a[k - 1]
        g[f"b{k}"] = dz.sum(axis=0)
        dh = dzr @ rnd(p[f"W{k}"])
        dz = dh * gelu_prime(z[k - 1])
    g["W0"] = dz.T @ X
    g["b0"] = dz.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, state: dict, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8) -> None:
    """One Adam update in place (Kingma & Ba, bias-corrected moments)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
