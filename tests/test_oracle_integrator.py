"""Pins of the oracle's time integration (Section 2.6, Eqs. newton1 and
newton2 with velocity Verlet, reading G9) and of its boundary treatment
(Section 2.5: periodic wrap, reflection at a wall axis) on a lone particle,
whose only force is the external one (Eq. govern, F^EXT).  Velocity Verlet
is exact for a constant force, so the trajectory must be the free-fall
parabola up to rounding."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import cases


def _lone(x0, v0, g, periodic, box=0.2, dt=1e-3, w0=(0.0, 0.0, 0.0), typ=0):
    p = cases.base_params(dx=1e-3)
    p.update(box=[box] * 3, periodic=list(periodic), kBT=0.0, g=list(g), dt=dt)
    return dict(params=p, x=np.array([x0], float), v=np.array([v0], float), w=np.array([w0], float),
                type=np.array([typ], np.int32), radius=np.array([0.5e-3]), mass=np.array([1e-6]))


def test_free_fall_is_the_parabola():
    x0, v0, g = np.array([0.1, 0.1, 0.15]), np.array([0.3, -0.2, 0.5]), np.array([0.0, 0.0, -9.81])
    c = _lone(x0, v0, g, (1, 1, 1))
    s = oracle.OracleSim(c)
    n, dt = 40, c["params"]["dt"]
    s.run(n)
    st = s.state()
    t = n * dt
    assert np.allclose(st["v"][0], v0 + g * t, rtol=1e-12, atol=1e-15)
    assert np.allclose(st["x"][0], x0 + v0 * t + 0.5 * g * t * t, rtol=1e-12, atol=1e-15)
    # no torque: the spin is unchanged
    assert np.array_equal(st["w"][0], c["w"][0])


def test_periodic_wrap_is_the_parabola_modulo_the_box():
    L = 0.2
    x0, v0, g = np.array([0.19, 0.005, 0.1]), np.array([0.6, -0.4, 0.0]), np.array([0.0, 0.0, 0.0])
    c = _lone(x0, v0, g, (1, 1, 1), box=L)
    s = oracle.OracleSim(c)
    n, dt = 50, c["params"]["dt"]
    s.run(n)
    x = s.state()["x"][0]
    ref = np.mod(x0 + v0 * n * dt, L)
    assert np.all((x >= 0.0) & (x < L))
    assert np.allclose(x, ref, rtol=0, atol=1e-14)


def test_reflection_at_a_wall_axis():
    # moving towards the lower wall of a non-periodic z axis at constant
    # speed: after the crossing the path is mirrored at z = 0 and the normal
    # velocity reversed; the other components are untouched
    x0, v0 = np.array([0.1, 0.1, 0.004]), np.array([0.01, 0.0, -0.3])
    c = _lone(x0, v0, (0.0, 0.0, 0.0), (1, 1, 0))
    s = oracle.OracleSim(c)
    n, dt = 30, c["params"]["dt"]
    s.run(n)
    st = s.state()
    t = n * dt
    z_free = x0[2] + v0[2] * t
    assert z_free < 0.0
    assert st["x"][0][2] == pytest.approx(-z_free, rel=1e-12)
    assert st["v"][0][2] == pytest.approx(-v0[2], rel=1e-15)
    assert st["x"][0][0] == pytest.approx(x0[0] + v0[0] * t, rel=1e-13)
    assert st["v"][0][0] == v0[0]
