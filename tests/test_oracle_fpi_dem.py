"""Pins of the oracle's fluid-particle interaction (Section 2.4: Eqs. beta,
C_D, F_fpi_DG, F_fpi_DG_reac, fvfdef) and contact models (Sections 2.2-2.3)
against closed forms and textbook results."""
import math

import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import cases


def _sphere_drag(Re_target, mu=1e-3, rho=1000.0, d=4e-3):
    v = Re_target * mu / (rho * d)
    return v, mu, rho, d


@pytest.mark.parametrize("Re", [1e-4, 0.3, 5.0, 120.0, 999.0, 1500.0, 2.3e4])
def test_single_sphere_drag_at_eps_one(Re):
    # At eps = 1 the Wen-Yu branch is the drag of an isolated sphere,
    # 1/2 C_D rho (pi d^2/4) |u| u, with the Schiller-Naumann / Newton C_D.
    v, mu, rho, d = _sphere_drag(Re)
    Vs = math.pi * d ** 3 / 6
    F = oracle.drag_force(1.0, d, rho, mu, Vs, [0.0, 0.0, v])
    CD = 24.0 / Re * (1 + 0.15 * Re ** 0.687) if Re <= 1000 else 0.44
    ref = 0.5 * CD * rho * (math.pi * d * d / 4) * v * v
    assert F[2] == pytest.approx(ref, rel=1e-12)
    assert F[0] == 0.0 and F[1] == 0.0


@pytest.mark.parametrize("eps", [0.81, 0.9, 1.0])
def test_stokes_limit(eps):
    # Re_p -> 0: 3 pi mu d u eps^-2.65 (Stokes drag with Wen-Yu voidage).
    mu, rho, d = 1e-3, 1000.0, 4e-3
    u = 1e-9
    F = oracle.drag_force(eps, d, rho, mu, math.pi * d ** 3 / 6, [u, 0, 0])
    assert F[0] == pytest.approx(3 * math.pi * mu * d * u * eps ** -2.65, rel=1e-6)


def test_drag_branch_continuity_in_Re():
    # The two C_D branches meet at Re_p = 1000 within 0.4 % (published fit).
    mu, rho, d = 1e-3, 1000.0, 4e-3
    Vs = math.pi * d ** 3 / 6
    v1 = 1000 * mu / (rho * d)
    lo = oracle.drag_force(1.0, d, rho, mu, Vs, [v1 * (1 - 1e-9), 0, 0])[0]
    hi = oracle.drag_force(1.0, d, rho, mu, Vs, [v1 * (1 + 1e-9), 0, 0])[0]
    assert abs(lo - hi) / hi < 0.004


def test_ergun_viscous_limit_is_kozeny_carman():
    # Ergun branch, slow flow: per unit bed volume the drag is the
    # Kozeny-Carman pressure gradient 150 mu (1-eps)^2 U / (eps^3 d^2) at
    # superficial velocity U = eps u, shared by the (1-eps) solid volume
    # fraction: force per particle = dP/dx * V_s / (1 - eps).
    mu, rho, d, eps = 2e-3, 1000.0, 3e-3, 0.6
    Vs = math.pi * d ** 3 / 6
    u = 1e-10
    F = oracle.drag_force(eps, d, rho, mu, Vs, [u, 0, 0])[0]
    dPdx = 150 * mu * (1 - eps) ** 2 * (eps * u) / (eps ** 3 * d ** 2)
    assert F == pytest.approx(dPdx * Vs / (1 - eps), rel=1e-6)


def test_drag_opposes_slip():
    # F^DG on the solid points along (v_f - v_s): it reduces the slip.
    F = oracle.drag_force(0.9, 4e-3, 1000.0, 1e-3, 3e-8, [0.0, 0.0, -0.2])
    assert F[2] < 0  # dv = v_f - v_s negative -> force negative


def _two_rigid_case(x1, x2, v1, v2, R=1e-3, rho_s=2500.0, box=0.05, periodic=(1, 1, 1), **over):
    p = cases.base_params(dx=1e-3, **over)
    p.update(box=[box] * 3, periodic=list(periodic), kBT=0.0)
    for k, v in over.items():
        p[k] = v
    m = rho_s * 4 / 3 * math.pi * R ** 3
    return dict(params=p, x=np.array([x1, x2], float), v=np.array([v1, v2], float),
                w=np.zeros((2, 3)), type=np.array([1, 1], np.int32), radius=np.array([R, R]),
                mass=np.array([m, m]))


def test_head_on_restitution_and_contact_time():
    # Linear spring-dashpot (dem_law 1): the rebound speed ratio equals the
    # restitution coefficient and the contact lasts pi / omega_d,
    # omega_d = sqrt(kn/m* - (cn/2m*)^2).
    R = 1e-3
    e_in = 0.7
    v0 = 0.05
    c = _two_rigid_case([0.02, 0.025, 0.025], [0.02 + 2 * R + 1e-5, 0.025, 0.025], [v0, 0, 0],
                        [-v0, 0, 0], R=R, restitution=e_in, kn=1e3, dt=2e-7, eta=0.0)
    c["params"]["r_c"] = 1.5e-3  # no lubrication: spheres only in contact range
    s = oracle.OracleSim(c)
    m = c["mass"][0]
    mstar = m / 2
    kn = 1e3
    le = math.log(e_in)
    zeta = -le / math.sqrt(math.pi ** 2 + le ** 2)
    cn = 2 * zeta * math.sqrt(mstar * kn)
    wd = math.sqrt(kn / mstar - (cn / (2 * mstar)) ** 2)
    tc = math.pi / wd
    dt = c["params"]["dt"]
    in_contact = []
    for k in range(int(3 * tc / dt) + 400):
        s.run(1)
        st = s.state()
        L = np.linalg.norm(st["x"][0] - st["x"][1])
        in_contact.append(L < 2 * R)
    st = s.state()
    v_out = st["v"][1, 0] - st["v"][0, 0]
    assert v_out / (2 * v0) == pytest.approx(e_in, rel=0.01)
    steps = np.sum(in_contact)
    assert steps * dt == pytest.approx(tc, rel=0.02)
    assert np.allclose(st["v"].sum(axis=0), 0.0, atol=1e-15)


def test_sliding_sphere_ends_rolling_at_five_sevenths():
    # A sphere launched sliding without spin on a plane with Coulomb friction
    # ends up rolling at 5/7 of its initial speed (solid sphere, I = 2/5 m R^2).
    R = 2e-3
    p = cases.base_params(dx=1e-3)
    p.update(box=[0.2, 0.2, 0.02], periodic=[1, 1, 0], g=[0, 0, -9.81], kBT=0.0, eta=0.0,
             mu_fric=0.4, kn=2e3, restitution=0.5, dt=2e-6, r_c=3e-3)
    m = 2500 * 4 / 3 * math.pi * R ** 3
    overlap = m * 9.81 / 2e3
    c = dict(params=p, x=np.array([[0.05, 0.1, R - overlap]]), v=np.array([[0.2, 0, 0]]),
             w=np.zeros((1, 3)), type=np.array([1], np.int32), radius=np.array([R]),
             mass=np.array([m]))
    s = oracle.OracleSim(c)
    s.run(60000)
    st = s.state()
    v = st["v"][0, 0]
    w = st["w"][0, 1]
    assert v == pytest.approx(5 / 7 * 0.2, rel=0.02)
    assert w * R == pytest.approx(v, rel=0.03)  # rolling: v = w R


def test_lubrication_is_antisymmetric_and_dissipative():
    R = 1e-3
    c = _two_rigid_case([0.02, 0.02, 0.02], [0.02 + 2 * R + 3e-4, 0.02, 0.02], [0.01, 0.002, 0],
                        [-0.01, 0, 0.003], R=R, eta=1e-3)
    c["params"]["r_c"] = 3.9e-3
    s = oracle.OracleSim(c)
    s.evaluate(1)
    F = s.component("lub")
    assert np.array_equal(F[0], -F[1])
    vij = c["v"][0] - c["v"][1]
    assert np.dot(F[0], vij) < 0
    # force grows as the gap closes
    c2 = _two_rigid_case([0.02, 0.02, 0.02], [0.02 + 2 * R + 1e-4, 0.02, 0.02], [0.01, 0.002, 0],
                         [-0.01, 0, 0.003], R=R, eta=1e-3)
    c2["params"]["r_c"] = 3.9e-3
    s2 = oracle.OracleSim(c2)
    s2.evaluate(1)
    assert np.linalg.norm(s2.component("lub")[0]) == pytest.approx(3 * np.linalg.norm(F[0]), rel=1e-12)


@pytest.mark.parametrize("gap_frac", [0.05, 0.2, 0.6])
def test_lubrication_magnitude_is_reynolds_two_sphere_force(gap_frac):
    # Two equal spheres of radius a approaching along their line of centres
    # at relative speed V with a surface gap g << a: Reynolds lubrication
    # between the two near-contact spheres gives the squeeze force
    # 6 pi mu V a*^2 / g with the reduced radius a* = a a / (a + a) = a / 2
    # (textbook asymptote, e.g. Kim & Karrila, Microhydrodynamics, Ch. 9).
    # The paper's Eq. lubri with d = R_i + R_j (reading G22) is the same
    # force, so a wrong prefactor, d = 2R as the diameter of one sphere of a
    # different size, or d^2 in place of d, fails here.
    a, mu, V = 1e-3, 2.5e-3, 0.013
    g = gap_frac * a
    c = _two_rigid_case([0.02, 0.02, 0.02], [0.02 + 2 * a + g, 0.02, 0.02], [V / 2, 0, 0],
                        [-V / 2, 0, 0], R=a, eta=mu)
    c["params"]["r_c"] = 3.9e-3
    c["params"]["lub_gap_min"] = 0.01
    s = oracle.OracleSim(c)
    s.evaluate(1)
    F = s.component("lub")
    a_red = a * a / (a + a)
    ref = 6 * math.pi * mu * V * a_red ** 2 / g
    # the squeeze force pushes the approaching spheres apart
    assert F[0][0] == pytest.approx(-ref, rel=1e-12)
    assert F[1][0] == pytest.approx(ref, rel=1e-12)
    assert F[0][1] == 0.0 and F[0][2] == 0.0


def test_dem_coefficients_law1():
    p = cases.base_params()
    kn, kt, cn, ct = oracle.dem_coeffs(p, 1e-3, 1e-3, 2e-5, 2e-5)
    assert kn == 1e3 and kt == pytest.approx(1e3 / 2.5)
    # critical damping when e -> 0: c -> 2 sqrt(m* k)
    p["restitution"] = 1e-300
    _, _, cn0, _ = oracle.dem_coeffs(p, 1e-3, 1e-3, 2e-5, 2e-5)
    assert cn0 == pytest.approx(2 * math.sqrt(1e-5 * 1e3), rel=1e-2)


def _slurry_case(phi=0.15, n=10):
    return cases.viscometer_instance(2 * n ** 3, phi, 300.0, 1e-2, seed=5, mesoscale=True)


def test_drag_reaction_conserves_momentum():
    c = _slurry_case()
    rng = np.random.default_rng(0)
    c["v"] = rng.normal(0, 0.5, size=c["v"].shape)
    s = oracle.OracleSim(c)
    s.evaluate(1)
    dg = s.component("dg")
    rxn = s.component("rxn")
    assert np.abs(dg).sum() > 0
    tot = dg.sum(axis=0) + rxn.sum(axis=0)
    assert np.abs(tot).max() < 1e-12 * np.abs(dg).sum()


def test_eps_single_sphere():
    # One sphere of diameter 4 dx alone within h = 3.9 dx: eps = 1 - (2/3.9)^3.
    c = cases.sedimentation(nx=12, ny=12, nz=24)
    s = oracle.OracleSim(c)
    s.evaluate(1)
    eps, S = s.fpi()
    k = int(np.where(c["type"] == 1)[0][0])
    assert eps[k] == pytest.approx(1 - (2 / 3.9) ** 3, rel=1e-12)
    assert S[k] > 0
