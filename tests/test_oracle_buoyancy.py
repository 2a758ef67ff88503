"""Pins of the pressure-gradient force on a rigid particle (Section 2.4,
Eq. F_fpi_PG in reading G17: F^PG_s = V_s d_s sum_fluid (F^C + F^D)) and of the
pressure part of the fluid force (Eq. FijC) by hydrostatics.

A sphere at rest in fluid at rest under a hydrostatic pressure field
p(z) = p_c - rho0 g (z - z_c) feels Archimedes' buoyancy rho0 g V_s, upward,
whatever its density; a fluid particle in the same field carries its own
weight.  The field is imposed on a perfect cubic lattice (number density
1/dx^3, the value the kernel normalisation gives a perfect lattice), so the
only difference from the continuum is the lattice sum of z^2 F(r), which is
within 0.2 % of its integral at h = 3.9 dx.  A wrong V_s or d_s factor, a
sign, or a weighted mean in place of the sum fails by far more than the
0.5 % tolerance."""
import math

import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import cases

N = 12
DX = 1e-3
G = 9.81


def _column(rho_s):
    p = cases.base_params(dx=DX, kBT=0.0)
    p.update(box=[N * DX] * 3, periodic=[1, 1, 1], g=[0.0, 0.0, -G])
    x = cases.lattice(N, N, N, DX)
    centre = np.full(3, N * DX / 2)
    k = int(np.argmin(np.linalg.norm(x - centre, axis=1)))
    n = len(x)
    R = 2 * DX
    typ = np.zeros(n, np.int32)
    typ[k] = 1
    rad = np.zeros(n)
    rad[k] = R
    mass = np.full(n, p["rho0"] * DX ** 3)
    mass[k] = rho_s * 4 / 3 * math.pi * R ** 3
    case = dict(params=p, x=x, v=np.zeros((n, 3)), w=np.zeros((n, 3)), type=typ, radius=rad, mass=mass)
    s = oracle.OracleSim(case)
    s.neighbors()
    zc = x[k, 2]
    pr = 1000.0 - p["rho0"] * G * (x[:, 2] - zc)
    s.set_fields(d=np.full(n, 1.0 / DX ** 3), p=pr)
    s.forces(1)
    return s, k, case


@pytest.mark.parametrize("rho_s", [1000.0, 2700.0])
def test_pressure_gradient_force_is_archimedes_buoyancy(rho_s):
    s, k, case = _column(rho_s)
    Vs = 4 / 3 * math.pi * case["radius"][k] ** 3
    buoy = case["params"]["rho0"] * G * Vs
    pg = s.component("pg")[k]
    assert pg[2] == pytest.approx(buoy, rel=5e-3)
    assert abs(pg[0]) < 1e-9 * buoy and abs(pg[1]) < 1e-9 * buoy
    # the sphere at rest in fluid at rest feels no drag; its net force is
    # its weight less the buoyancy, the start of the settling ODE
    assert np.allclose(s.component("dg")[k], 0.0)
    net = s.state()["F"][k]
    assert abs(net[2] - (buoy - case["mass"][k] * G)) < 5e-3 * buoy


def test_fluid_particle_carries_its_weight_in_the_hydrostatic_field():
    s, k, case = _column(2700.0)
    x = case["x"]
    # the site half a box away along x, at the sphere's height (beyond h of it)
    target = x[k] + np.array([N * DX / 2, 0.0, 0.0])
    target[0] -= N * DX if target[0] > N * DX else 0.0
    i = int(np.argmin(np.linalg.norm(x - target, axis=1)))
    assert np.linalg.norm(x[i] - x[k]) > case["params"]["r_c"]
    F = s.state()["F"][i]
    w = case["mass"][i] * G
    assert abs(F[2]) < 5e-3 * w          # pressure force balances gravity
    assert abs(F[0]) < 1e-9 * w and abs(F[1]) < 1e-9 * w
    # and the pressure force alone is the weight, upward
    assert s.component("sdpd")[i][2] == pytest.approx(w, rel=5e-3)
