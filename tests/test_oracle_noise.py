"""Pins of the counter-based noise and the random force (Section 2.1,
Eqs. FijT and reldWij; Section 3.3 symmetric dW_ij per pair).

The paper draws dW with MT19937-64; the build draws it from Philox4x32-10
(Salmon et al., SC'11).  Philox is pinned here by its statistics and its
bijectivity; the random force by the fluctuation-dissipation identity
Cov(impulse) = 2 kBT dt [ga (1 + ee/3) + (2 gb/3) ee], which holds only with
sigma = 2 sqrt(kBT gamma), the traceless-symmetric part of dW and the trace part
weighted as printed."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def test_philox_known_answer_vectors():
    # the published Random123 known-answer vectors (tests/golden/): a wrong
    # round constant, Weyl increment, output permutation or round count
    # changes every one of them, while the statistical checks below would
    # still pass for any other bijective mixing
    from _gpu_common import philox_kat
    ctr, key, want = philox_kat()
    for c, k, w in zip(ctr, key, want):
        assert oracle.philox(c.tolist(), k.tolist()) == [int(v) for v in w]


def test_philox_uniform_bits():
    outs = []
    for c in range(4000):
        outs += oracle.philox([c, 7, 11, 0], [0x1234, 0xABCD])
    u = np.array(outs, dtype=np.uint64)
    # every bit is balanced
    bits = ((u[:, None] >> np.arange(32, dtype=np.uint64)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.02)
    # bytes uniform (chi-square)
    b = (u & 0xFF).astype(np.int64)
    hist = np.bincount(b, minlength=256)
    chi2, pval = stats.chisquare(hist)
    assert pval > 1e-4


def test_philox_avalanche():
    base = oracle.philox([5, 6, 7, 8], [9, 10])
    flips = []
    for bit in range(32):
        o = oracle.philox([5 ^ (1 << bit), 6, 7, 8], [9, 10])
        flips.append(sum(bin(a ^ b).count("1") for a, b in zip(base, o)))
    assert 40 < np.mean(flips) < 88  # about half of 128 bits flip


def test_philox_is_injective_on_a_sample():
    seen = set()
    for c in range(20000):
        seen.add(tuple(oracle.philox([c, 0, 0, 0], [1, 2])))
    assert len(seen) == 20000


def test_pair_normals_symmetric_and_step_keyed():
    z1 = oracle.pair_normals(1, 0, 17, 903, 5)
    z2 = oracle.pair_normals(1, 0, 903, 17, 5)
    assert np.array_equal(z1, z2)
    assert not np.array_equal(z1, oracle.pair_normals(1, 0, 17, 903, 6))
    assert not np.array_equal(z1, oracle.pair_normals(1, 1, 17, 903, 5))
    assert not np.array_equal(z1, oracle.pair_normals(2, 0, 17, 903, 5))


def test_pair_normals_are_standard_normal():
    z = np.concatenate([oracle.pair_normals(3, 0, i, i + 1000, 0) for i in range(20000)])
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 0.05
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_random_impulse_satisfies_fdt():
    kBT, dt = 1.7, 0.01
    ga, gb = 0.8, 1.9
    sa, sb = 2 * math.sqrt(kBT * ga), 2 * math.sqrt(kBT * gb)
    e = np.array([0.3, -0.5, 0.8])
    e /= np.linalg.norm(e)
    n = 60000
    imp = np.empty((n, 3))
    for k in range(n):
        z = oracle.pair_normals(11, 0, k, k + n, 3)
        # impulse over dt: F~ dt = (sigma Z . e) sqrt(dt)
        imp[k] = oracle.noise_vector(z, sa, sb, e) * math.sqrt(dt)
    cov = np.cov(imp.T)
    ee = np.outer(e, e)
    target = 2 * kBT * dt * (ga * (np.eye(3) + ee / 3) + 2 * gb / 3 * ee)
    err = np.abs(cov - target).max() / np.abs(target).max()
    assert err < 0.03, (cov, target)


def test_noise_vector_parts():
    e = np.array([0.0, 0.0, 1.0])
    # pure trace: S = I -> deviatoric part 0, trace part sb * e
    z = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    assert np.allclose(oracle.noise_vector(z, 2.0, 5.0, e), [0, 0, 5.0])
    # pure off-diagonal xz: S_xz = z4/sqrt2 -> (sa * S_xz, 0, 0)
    z = np.array([0.0, 0.0, 0.0, 0.0, math.sqrt(2.0), 0.0])
    assert np.allclose(oracle.noise_vector(z, 2.0, 5.0, e), [2.0, 0, 0])
