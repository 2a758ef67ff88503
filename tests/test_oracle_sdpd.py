"""Pins of the oracle's SDPD pair forces (Section 2.1: Eqs. FijC, FijD, FijR,
FijT) and time integration (Section 2.6) against invariants and closed forms."""
import math

import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import cases


def _pair_case(xi, xj, vi, vj, wi, wj, **over):
    p = cases.base_params(dx=1.0, rho0=1.0, eta=2.0, kBT=0.5, dt=1e-3, **over)
    p.update(box=[50.0] * 3, periodic=[0, 0, 0], origin=[0.0] * 3)
    for k, v in over.items():
        p[k] = v
    return dict(params=p, x=np.array([xi, xj], float), v=np.array([vi, vj], float),
                w=np.array([wi, wj], float), type=np.array([0, 0], np.int32),
                radius=np.array([0.5, 0.5]), mass=np.array([1.0, 1.0]))


def test_pair_forces_are_exactly_antisymmetric():
    c = _pair_case([20.0, 20.3, 19.9], [21.7, 19.4, 20.8], [0.3, -0.2, 0.1], [-0.4, 0.5, 0.2],
                   [0.1, 0.2, -0.3], [0.05, -0.1, 0.4])
    s = oracle.OracleSim(c)
    s.step = 7
    s.evaluate(1)
    F = s.component("sdpd")
    assert np.any(F != 0)
    assert np.array_equal(F[0], -F[1])


def test_rigid_rotation_is_force_free():
    # SDPD+a (angular-momentum form): a rigid-body rotation v = W x r with
    # spins w = W produces no dissipative + rotational force (Eqs. FijD, FijR).
    Om = np.array([0.3, -0.7, 0.45])
    xi = np.array([20.0, 20.3, 19.9])
    xj = np.array([21.7, 19.4, 20.8])
    c = _pair_case(xi, xj, np.cross(Om, xi), np.cross(Om, xj), Om, Om, coeff_c=0.0, coeff_t=0.0)
    s = oracle.OracleSim(c)
    s.evaluate(1)
    F = s.component("sdpd")
    scale = 2.0 * np.linalg.norm(np.cross(Om, xi - xj))  # size of F^D alone
    assert np.abs(F).max() < 1e-13 * max(scale, 1.0)
    # without the rotational part the same motion is dissipated
    c2 = _pair_case(xi, xj, np.cross(Om, xi), np.cross(Om, xj), Om, Om, coeff_c=0.0, coeff_t=0.0,
                    coeff_r=0.0)
    s2 = oracle.OracleSim(c2)
    s2.evaluate(1)
    assert np.abs(s2.component("sdpd")).max() > 1e-3


def test_uniform_translation_is_force_free():
    c = _pair_case([20.0, 20.3, 19.9], [21.7, 19.4, 20.8], [0.3, -0.2, 0.1], [0.3, -0.2, 0.1],
                   [0, 0, 0], [0, 0, 0], coeff_c=0.0, coeff_t=0.0)
    s = oracle.OracleSim(c)
    s.evaluate(1)
    assert np.abs(s.component("sdpd")).max() == 0.0


def test_fluid_momentum_is_conserved():
    c = cases.poiseuille_si(nx=10, ny=10, nz=10, g_amp=0.0)
    rng = np.random.default_rng(2)
    c["v"] = rng.normal(0, 1e-3, size=c["v"].shape)
    c["w"] = rng.normal(0, 1.0, size=c["w"].shape)
    c["params"]["kBT"] = 4.1e-15  # make the noise visible
    s = oracle.OracleSim(c)
    s.evaluate(1)
    F = s.state()["F"]
    assert np.abs(F.sum(axis=0)).max() < 1e-13 * np.abs(F).sum()


def test_dissipative_power_is_negative():
    c = cases.poiseuille_si(nx=10, ny=10, nz=10, g_amp=0.0, coeff_c=0.0, coeff_t=0.0, coeff_r=0.0)
    rng = np.random.default_rng(3)
    c["v"] = rng.normal(0, 1e-3, size=c["v"].shape)
    s = oracle.OracleSim(c)
    s.evaluate(1)
    F = s.state()["F"]
    assert np.sum(F * c["v"]) < 0


def test_probe_reads_viscosity_of_exact_profile():
    # Eq. poiseuave: a particle field carrying exactly the steady profile of
    # Eq. poiseuanasol in each half reads back the viscosity (up to the
    # O(dx^2/D^2) error of sampling the parabola at lattice sites).
    c = cases.poiseuille_meso(nx=8, ny=40, nz=8, jitter=0.0)
    p = c["params"]
    mu, a, rho = p["eta"], p["body_amp"], p["rho0"]
    L = p["box"][1]
    D = 0.5 * L
    y = c["x"][:, 1]
    z = np.where(y < D, y, y - D)
    prof = rho * a / (2 * mu) * (z * D - z * z)
    c["v"][:, 0] = np.where(y < D, prof, -prof)
    s = oracle.OracleSim(c)
    prof_b, mu_app = s.profile(20)
    dx = p["dx"]
    # discrete mean of the parabola over n = D/dx sites at (k+1/2) dx
    nsite = int(round(D / dx))
    zz = (np.arange(nsite) + 0.5) * dx
    V = np.mean(rho * a / (2 * mu) * (zz * D - zz * zz))
    assert mu_app == pytest.approx(rho * a * D * D / (12 * V), rel=1e-10)
    assert mu_app == pytest.approx(mu, rel=2 * (dx / D) ** 2)


@pytest.mark.parametrize("slip", [0.0, 0.37])
def test_fit_reads_viscosity_of_exact_profile_whatever_the_slip(slip):
    # Reading B6: a parabola fitted per half is exact on a field that carries
    # the steady profile of Eq. poiseuanasol, with or without a slip
    # velocity at the ends of the halves (where the mean-velocity read-out of
    # Eq. poiseuave is biased), so the curvature gives mu to rounding.
    c = cases.poiseuille_meso(nx=8, ny=48, nz=8, jitter=0.0)
    p = c["params"]
    mu, a, rho = p["eta"], p["body_amp"], p["rho0"]
    D = 0.5 * p["box"][1]
    y = c["x"][:, 1]
    z = np.where(y < D, y, y - D)
    prof = rho * a / (2 * mu) * (z * D - z * z) + slip
    c["v"][:, 0] = np.where(y < D, prof, -prof)
    s = oracle.OracleSim(c)
    assert s.viscosity_fit(24) == pytest.approx(mu, rel=1e-9)
    _, mu_app = s.profile(24)
    if slip:
        assert abs(mu_app / mu - 1) > 0.01


def test_diagnostics_are_the_plain_sums():
    # closed forms: a uniform drift U of every mobile particle has momentum
    # M U, kinetic energy M U^2 / 2 and no kinetic temperature; adding
    # +-w along x on alternate particles of equal mass gives temperature
    # m w^2 / 3; a perfect lattice has number density 1/dx^3 everywhere
    # (the kernel normalisation), walls excepted
    c = cases.poiseuille_meso(nx=8, ny=8, nz=8, jitter=0.0)
    n = len(c["x"])
    U = np.array([0.3, -0.2, 0.1])
    c["v"] = np.tile(U, (n, 1))
    s = oracle.OracleSim(c)
    s.neighbors()
    s.density()
    d = s.diagnostics()
    M = c["mass"].sum()
    assert np.allclose(d[0:3], M * U, rtol=1e-12)
    assert d[3] == pytest.approx(0.5 * M * U @ U, rel=1e-12)
    assert abs(d[4]) < 1e-12 * M * (U @ U)
    assert d[5] == pytest.approx(np.linalg.norm(U), rel=1e-12)
    dx = c["params"]["dx"]
    assert d[6] == pytest.approx(1 / dx ** 3, rel=1e-12) and d[7] == pytest.approx(1 / dx ** 3, rel=1e-12)
    assert d[8] == 0
    w = 0.05
    c["v"][:, 0] += np.where(np.arange(n) % 2 == 0, w, -w)
    c["x"][3, 1] = np.nan
    s2 = oracle.OracleSim(c)
    d2 = s2.diagnostics()
    assert d2[4] == pytest.approx(c["mass"][0] * w * w / 3, rel=1e-9)
    assert d2[8] == 1


def _transient_profile(y, t, a, nu, L, kmax=401):
    # start-up of the reverse-Poiseuille flow (square-wave forcing +a on
    # [0, L/2), -a on [L/2, L)): Fourier series of the diffusion equation.
    u = np.zeros_like(y)
    for k in range(1, kmax, 2):
        kap = 2 * math.pi * k / L
        u += 4 * a / (math.pi * k) * np.sin(kap * y) * (1 - math.exp(-nu * kap * kap * t)) / (nu * kap * kap)
    return u


@pytest.mark.slow
def test_reverse_poiseuille_transient_gives_input_viscosity():
    # Section 4.1 in the paper's mesoscale units.  With the rotational force
    # on (spins relax to half the vorticity) the SDPD+a dissipative force
    # carries shear viscosity eta; the start-up profile of the
    # counter-flowing halves is fitted with the diffusion-equation series
    # for nu.  Noise off so the profile is deterministic.
    c = cases.poiseuille_meso(nx=8, ny=24, nz=8, kBT=0.0, jitter=0.0)
    p = c["params"]
    c["params"]["dt"] = 0.1 * p["r_c"] / math.sqrt(p["alpha"] * p["p0"] / p["rho0"])
    s = oracle.OracleSim(c)
    nsteps = 120
    s.run(nsteps)
    t = nsteps * c["params"]["dt"]
    st = s.state()
    L = p["box"][1]
    y = st["x"][:, 1]
    u = st["v"][:, 0]
    nb = 24
    b = np.clip((y / L * nb).astype(int), 0, nb - 1)
    yc = (np.arange(nb) + 0.5) * L / nb
    ub = np.array([u[b == k].mean() for k in range(nb)])
    nus = np.linspace(0.5, 2.0, 301) * p["eta"] / p["rho0"]
    errs = [np.sum((_transient_profile(yc, t, p["body_amp"], nu, L) - ub) ** 2) for nu in nus]
    nu_fit = nus[int(np.argmin(errs))]
    eta_fit = nu_fit * p["rho0"]
    assert eta_fit == pytest.approx(p["eta"], rel=0.06), eta_fit


@pytest.mark.slow
def test_without_rotational_force_viscosity_is_twelve_sevenths():
    # Continuum limit of Eq. FijD alone (xi = 20 eta/21, so gamma^a = gamma^b
    # = 20 eta/7 F/(d_i d_j)): the second moment of F gives an effective shear
    # viscosity gamma_a/2 + (gamma_a + 2 gamma_b)/30 = 12 eta / 7.  The
    # rotational force with relaxed spins removes gamma_a/4, giving eta.
    c = cases.poiseuille_meso(nx=8, ny=24, nz=8, kBT=0.0, jitter=0.0, coeff_r=0.0)
    p = c["params"]
    c["params"]["dt"] = 0.1 * p["r_c"] / math.sqrt(p["alpha"] * p["p0"] / p["rho0"])
    s = oracle.OracleSim(c)
    nsteps = 120
    s.run(nsteps)
    t = nsteps * c["params"]["dt"]
    st = s.state()
    L = p["box"][1]
    y = st["x"][:, 1]
    u = st["v"][:, 0]
    nb = 24
    b = np.clip((y / L * nb).astype(int), 0, nb - 1)
    yc = (np.arange(nb) + 0.5) * L / nb
    ub = np.array([u[b == k].mean() for k in range(nb)])
    nus = np.linspace(0.5, 3.0, 501) * p["eta"] / p["rho0"]
    errs = [np.sum((_transient_profile(yc, t, p["body_amp"], nu, L) - ub) ** 2) for nu in nus]
    eta_fit = nus[int(np.argmin(errs))] * p["rho0"]
    assert eta_fit == pytest.approx(12.0 / 7.0 * p["eta"], rel=0.06), eta_fit


@pytest.mark.slow
def test_equipartition():
    # Fluctuation-dissipation (Section 2.1): with the random and dissipative
    # forces in balance the kinetic temperature m<v^2>/3 equals kBT.
    # Rotational force off (its torque lever differs from SDPD+a, so only the
    # translational temperature is pinned).
    c = cases.poiseuille_meso(nx=8, ny=8, nz=8, amp=0.0, kBT=1.0, coeff_r=0.0)
    p = c["params"]
    c["params"]["dt"] = 0.02 * p["r_c"] / math.sqrt(p["alpha"] * p["p0"] / p["rho0"])
    s = oracle.OracleSim(c)
    s.run(150)
    temps = []
    for k in range(60):
        s.run(5)
        v = s.state()["v"]
        v = v - v.mean(axis=0)
        temps.append(np.mean(np.sum(v * v, axis=1)) / 3.0)
    T = np.mean(temps)
    assert T == pytest.approx(1.0, rel=0.05), T
