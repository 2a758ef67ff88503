"""The collision-method artificial viscosity (reading G25: mobile pairs closer
than 0.5 dx that approach exchange momentum as an inelastic collision,
restitution 0.2, Jacobi update after the velver-2 kick) on the GPU path
against the oracle, one full step with several close approaching pairs.  The
density pass marks the particles that have a close neighbour and the
collision pass scans only those: a missed mark would show here."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _case(artvis):
    n = 12
    c = cases.poiseuille_meso(nx=n, ny=n, nz=n, amp=0.0, kBT=1e-3, seed=5, artvis=artvis)
    dx = c["params"]["dx"]
    rng = np.random.default_rng(6)
    x, v = c["x"], c["v"]
    # 16 pairs on well separated sites: j = the +x lattice neighbour of i,
    # moved to 0.3 dx from i along a random direction, both approaching
    sites = rng.choice(n * n * n, size=400, replace=False)
    used, pairs = set(), []
    for i in sites:
        i = int(i)
        if i % n >= n - 2 or len(pairs) == 16 or used & {i - 1, i, i + 1, i + 2}:
            continue
        used |= {i, i + 1}
        pairs.append((i, i + 1))
    for i, j in pairs:
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        x[j] = x[i] + 0.3 * dx * e
        v[i] = 0.8 * e
        v[j] = -0.8 * e
    return c, pairs


@pytest.mark.parametrize("precision,tol", [(B.SDPD_PREC_FP64, 1e-9), (B.SDPD_PREC_SPLIT, 1e-4)])
def test_collision_pass_matches_oracle(precision, tol):
    case, pairs = _case(artvis=1)
    assert len(pairs) == 16
    sim = B.Sim(case, precision=precision)
    sim.step(1)
    gv = sim.state(density=False)["v"]
    orc = oracle.OracleSim(case)
    orc.run(1)
    ov = orc.state()["v"]
    assert rel_l2(gv, ov) < tol
    # the collisions happened: without them the close pairs keep approaching
    off, _ = _case(artvis=0)
    o2 = oracle.OracleSim(off)
    o2.run(1)
    ov2 = o2.state()["v"]
    idx = np.array([p for pr in pairs for p in pr])
    assert np.linalg.norm(ov[idx] - ov2[idx]) > 0.1 * np.linalg.norm(ov2[idx])
    assert rel_l2(gv[idx], ov[idx]) < tol
