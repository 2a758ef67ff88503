"""Pins of the surrogate-network oracle (oracle/mlp_oracle.py) and the Sobol
sampler: finite-difference gradients, Adam's first step, GELU identities,
BF16 rounding, net properties of the Sobol points."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2002_03120_gb300.sobol import sobol


def test_gelu_identities():
    assert M.gelu(np.array(0.0)) == 0.0
    assert M.gelu(np.array(10.0)) == pytest.approx(10.0, rel=1e-12)
    assert M.gelu_prime(np.array(0.0)) == pytest.approx(0.5)
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    assert np.allclose(M.gelu_prime(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), atol=1e-8)


def test_bf16_rounding():
    assert M.bf16(np.array([1.0]))[0] == 1.0
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert M.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert M.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    x = np.random.default_rng(0).normal(size=1000)
    assert np.max(np.abs(M.bf16(x) - x) / np.abs(x)) <= 2 ** -8


def test_fp64_gradients_match_finite_differences():
    p = M.init_params(3, width=16)
    rng = np.random.default_rng(1)
    X = rng.uniform(size=(7, 3))
    t = rng.normal(size=7)
    y, cache = M.forward(p, X, "fp64")
    g = M.backward(p, cache, y, t)
    h = 1e-6
    for k in ("W0", "b0", "W1", "b2", "W3", "W4", "b4"):
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(M.forward(p, X, "fp64")[0], t)
            flat[idx] = old - h
            lm = M.loss(M.forward(p, X, "fp64")[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-4, abs=1e-9), (k, idx)


def test_bf16_path_close_to_fp64():
    p = M.init_params(4)
    X = np.random.default_rng(2).uniform(size=(256, 3))
    y64, _ = M.forward(p, X, "fp64")
    y16, _ = M.forward(p, X, "bf16")
    assert np.linalg.norm(y16 - y64) / np.linalg.norm(y64) < 2e-2


def test_adam_first_step_is_signed_lr():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    st = {}
    M.adam_step(p, g, st, lr=1e-3)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> lr * g / (|g| + eps)
    assert np.allclose(p["w"], [1.0 - 1e-3, -2.0 + 1e-3, 0.5 - 1e-3 * 1e-3 / (1e-3 + 1e-8)])


def test_training_reduces_loss():
    p = M.init_params(5, width=32)
    rng = np.random.default_rng(6)
    X = rng.uniform(size=(256, 3))
    t = np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2]
    st = {}
    l0 = M.loss(M.forward(p, X, "fp64")[0], t)
    for _ in range(300):
        y, c = M.forward(p, X, "fp64")
        M.adam_step(p, M.backward(p, c, y, t), st, lr=3e-3)
    assert M.loss(M.forward(p, X, "fp64")[0], t) < 0.1 * l0


def test_sobol_is_a_0m2_net_in_dims_1_2():
    # the first 2^m points of dims 1-2 put exactly one point in every
    # elementary dyadic box of area 2^-m
    m = 6
    P = sobol(1 << m, 2)
    for a in range(m + 1):
        b = m - a
        ix = np.floor(P[:, 0] * (1 << a)).astype(int)
        iy = np.floor(P[:, 1] * (1 << b)).astype(int)
        counts = np.zeros((1 << a, 1 << b), dtype=int)
        np.add.at(counts, (ix, iy), 1)
        assert np.all(counts == 1), (a, b)


def test_sobol_one_dimensional_stratification_all_dims():
    P = sobol(1024, 3)
    for d in range(3):
        for k in range(1, 11):
            n = 1 << k
            counts = np.bincount(np.floor(P[:n, d] * n).astype(int), minlength=n)
            assert np.all(counts == 1)
    assert np.all(P >= 0) and np.all(P < 1)
    assert np.allclose(P.mean(axis=0), 0.5, atol=2e-3)
