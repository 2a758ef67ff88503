"""Pins of the oracle's collision-method artificial viscosity (Table 1's
enable_artvis option, Section 4.4; reading G25: mobile pairs closer than artvis_alpha dx that
approach each other collide inelastically with restitution artvis_e, every
correction from the pre-correction velocities) against the mechanics of a
two-body collision: the relative normal velocity is reversed and scaled by the
restitution coefficient, the tangential velocities are untouched and the
momentum is conserved.  These laws, not the oracle's formula, fix the
expected velocities."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import cases

DX = 1e-3


def _case(x, v, m, types, artvis=1, e_c=0.2):
    p = cases.base_params(dx=DX)
    p.update(box=[0.05] * 3, periodic=[1, 1, 1], kBT=0.0, artvis=artvis, artvis_e=e_c, artvis_alpha=0.5)
    n = len(x)
    return dict(params=p, x=np.array(x, float), v=np.array(v, float), w=np.zeros((n, 3)),
                type=np.array(types, np.int32), radius=np.full(n, 0.5 * DX), mass=np.array(m, float))


def _after(c):
    s = oracle.OracleSim(c)
    s.neighbors()
    s.artvis()
    return s.state()["v"]


@pytest.mark.parametrize("e_c", [0.0, 0.2, 1.0])
def test_two_body_collision_laws(e_c):
    rng = np.random.default_rng(3)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    x1 = np.array([0.02, 0.025, 0.025])
    x2 = x1 - 0.3 * DX * n           # e_12 = (x1 - x2) / |x1 - x2| = n
    m1, m2 = 1.0e-6, 2.7e-6
    v1 = rng.normal(size=3) * 1e-2
    v2 = v1 + (0.05 + rng.normal(size=3) * 1e-3)
    # make the pair approach: (v1 - v2) . n < 0
    if np.dot(v1 - v2, n) > 0:
        v2 = v1 - (v2 - v1)
    rel_n = np.dot(v1 - v2, n)
    assert rel_n < 0
    c = _case([x1, x2], [v1, v2], [m1, m2], [0, 0], e_c=e_c)
    w1, w2 = _after(c)
    # restitution: the relative normal velocity is reversed and scaled by e_c
    assert np.dot(w1 - w2, n) == pytest.approx(-e_c * rel_n, rel=1e-12, abs=1e-15)
    # the impulse is along the line of centres: tangential velocities unchanged
    for u, w in ((v1, w1), (v2, w2)):
        ut, wt = u - np.dot(u, n) * n, w - np.dot(w, n) * n
        assert np.allclose(wt, ut, rtol=0, atol=1e-16)
    # momentum is conserved
    assert np.allclose(m1 * w1 + m2 * w2, m1 * v1 + m2 * v2, rtol=1e-14, atol=1e-22)


def test_receding_far_and_wall_pairs_are_untouched():
    x1 = np.array([0.02, 0.025, 0.025])
    # receding (v_12 . e_12 > 0) within the collision radius
    c = _case([x1, x1 - [0.3 * DX, 0, 0]], [[1e-2, 0, 0], [-1e-2, 0, 0]], [1e-6, 1e-6], [0, 0])
    assert np.array_equal(_after(c), c["v"])
    # approaching, but beyond artvis_alpha dx
    c = _case([x1, x1 - [0.6 * DX, 0, 0]], [[-1e-2, 0, 0], [1e-2, 0, 0]], [1e-6, 1e-6], [0, 0])
    assert np.array_equal(_after(c), c["v"])
    # approaching a wall particle (not mobile)
    c = _case([x1, x1 - [0.3 * DX, 0, 0]], [[-1e-2, 0, 0], [0, 0, 0]], [1e-6, 1e-6], [0, 2])
    assert np.array_equal(_after(c), c["v"])
    # switched off
    c = _case([x1, x1 - [0.3 * DX, 0, 0]], [[-1e-2, 0, 0], [1e-2, 0, 0]], [1e-6, 1e-6], [0, 0], artvis=0)
    assert np.array_equal(_after(c), c["v"])


def test_cloud_conserves_momentum():
    # a dense random cloud: many overlapping collisions in one Jacobi pass
    rng = np.random.default_rng(11)
    n = 300
    x = 0.02 + rng.uniform(0, 4 * DX, size=(n, 3))
    v = rng.normal(size=(n, 3)) * 1e-2
    m = rng.uniform(0.5e-6, 2e-6, size=n)
    c = _case(x, v, m, [0] * n)
    w = _after(c)
    p0 = (m[:, None] * v).sum(axis=0)
    p1 = (m[:, None] * w).sum(axis=0)
    scale = (m[:, None] * np.abs(v)).sum()
    assert np.abs(p1 - p0).max() < 1e-14 * scale
    assert not np.array_equal(w, v)   # collisions happened
