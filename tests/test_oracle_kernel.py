"""Pins of the oracle's kernel, density, equation of state and filter
(Section 2.1: Eqs. kernel, F, compdens, prtcpres; Section 3.3 normalisation and
pressure smoothing) against closed forms and invariants."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2002_03120_gb300 import cases


@pytest.mark.parametrize("h", [1.0, 3.9e-3, 2.7])
def test_lucy_kernel_integrates_to_one(h):
    # A normalised smoothing kernel has unit volume integral (Eq. kernel).
    val, err = integrate.quad(lambda r: 4 * math.pi * r * r * oracle.W(r, h), 0.0, h,
                              epsabs=0, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("q", [0.05, 0.2, 0.5, 0.77, 0.95])
def test_F_is_minus_dW_over_r(q):
    # Eq. defF: F(r) = -W'(r)/r; checked by a central difference of W.
    h = 1.3
    r = q * h
    eps = 1e-6 * h
    dW = (oracle.W(r + eps, h) - oracle.W(r - eps, h)) / (2 * eps)
    assert oracle.Fk(r, h) == pytest.approx(-dW / r, rel=1e-7)


def test_kernel_vanishes_at_support():
    h = 2.0
    assert oracle.W(h, h) == 0.0 and oracle.Fk(h, h) == 0.0
    assert oracle.W(h * (1 - 1e-9), h) < 1e-20
    assert oracle.W(0.0, h) == pytest.approx(105.0 / (16.0 * math.pi * h ** 3), rel=1e-15)


def _perfect_lattice(n=(8, 8, 8), **over):
    c = cases.poiseuille_si(nx=n[0], ny=n[1], nz=n[2], jitter=0.0, g_amp=0.0, **over)
    return c


def test_perfect_lattice_has_reference_density():
    # Normalisation of the kernel coefficient: a perfect lattice must give
    # rho = rho0 exactly, hence p = p0 - beta = 0.
    c = _perfect_lattice()
    s = oracle.OracleSim(c)
    s.neighbors()
    s.density()
    st = s.state()
    dx = c["params"]["dx"]
    assert np.allclose(st["d"] * dx ** 3, 1.0, rtol=1e-12, atol=0)
    assert np.max(np.abs(st["p"])) < 1e-9 * c["params"]["p0"]


def test_lattice_neighbour_count():
    # 250 lattice neighbours strictly inside 3.9 dx (counted by brute force on
    # integer offsets, independent of the oracle).
    k = np.arange(-4, 5)
    I, J, K = np.meshgrid(k, k, k, indexing="ij")
    r2 = I ** 2 + J ** 2 + K ** 2
    expected = int(np.sum((r2 > 0) & (r2 < 3.9 ** 2)))
    assert expected == 250
    c = _perfect_lattice()
    s = oracle.OracleSim(c)
    s.neighbors()
    assert len(s.pairs()) * 2 == expected * s.n


def test_density_is_translation_invariant():
    c = cases.poiseuille_si(nx=8, ny=8, nz=8)
    s = oracle.OracleSim(c)
    s.neighbors(); s.density()
    d0 = s.state()["d"]
    c2 = dict(c)
    L = np.asarray(c["params"]["box"])
    c2["x"] = np.mod(c["x"] + np.array([0.37, 0.11, 0.73]) * L, L)
    s2 = oracle.OracleSim(c2)
    s2.neighbors(); s2.density()
    assert np.allclose(s2.state()["d"], d0, rtol=1e-12)


def test_eos_sound_speed():
    # dp/drho at rho0 equals c^2 = alpha p0 / rho0 (the EOS's compressibility).
    rho0, p0, alpha, beta = 1000.0, 14285.714, 7.0, 14285.714
    h = 1e-3
    dp = (oracle.eos(rho0 + h, rho0, p0, alpha, beta) - oracle.eos(rho0 - h, rho0, p0, alpha, beta)) / (2 * h)
    assert dp == pytest.approx(alpha * p0 / rho0, rel=1e-8)
    assert oracle.eos(rho0, rho0, p0, alpha, beta) == pytest.approx(p0 - beta, abs=1e-9)
    # alpha = 1 makes the law affine
    assert oracle.eos(2 * rho0, rho0, p0, 1.0, beta) == pytest.approx(2 * p0 - beta, rel=1e-14)


def test_filter_keeps_constant_pressure():
    # With p0 = 0 every particle has p = -beta; the Shepard average of a
    # constant field is that constant.
    c = cases.poiseuille_si(nx=8, ny=8, nz=8, pressure_filter=1)
    c["params"]["p0"] = 0.0
    c["params"]["beta_p"] = 3.5
    s = oracle.OracleSim(c)
    s.neighbors(); s.density(); s.filter()
    assert np.allclose(s.state()["p"], -3.5, rtol=1e-13)


def test_filter_is_a_convex_average():
    c = cases.poiseuille_si(nx=8, ny=8, nz=8, pressure_filter=1)
    s = oracle.OracleSim(c)
    s.neighbors(); s.density()
    p_raw = s.state()["p"].copy()
    s.filter()
    p_f = s.state()["p"]
    assert p_f.min() >= p_raw.min() - 1e-9 and p_f.max() <= p_raw.max() + 1e-9
    assert np.std(p_f) < np.std(p_raw)


def test_clamp_negative_pressure():
    c = cases.poiseuille_si(nx=8, ny=8, nz=8, clamp_negative_p=1)
    s = oracle.OracleSim(c)
    s.neighbors(); s.density()
    assert s.state()["p"].min() >= 0.0
