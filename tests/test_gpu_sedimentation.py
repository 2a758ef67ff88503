"""Single-particle sedimentation (Section 4.2) stepped on the GPU and on the
oracle from the same seeded inputs, with the random force off (kBT = 0), so
that both runs are deterministic: over 40 full steps the sphere's velocity
and position follow the oracle's (FP64 to summation-order rounding, the split
path within its force tolerance).  (Over these first steps the unrelaxed
column's pressure waves push the sphere about; it settles later.)  The
settling velocity is not compared with the drag ODE:
in the model the viscous part of the pressure-gradient force and the fluid
the sphere drags along change it (reading B7); those forces are pinned one by
one on the oracle (test_oracle_buoyancy.py, test_oracle_fpi_dem.py)."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu

STEPS = 40


@pytest.fixture(scope="module")
def oracle_run():
    case = cases.sedimentation(nx=12, ny=12, nz=24, kBT=0.0)
    k = int(np.where(case["type"] == 1)[0][0])
    s = oracle.OracleSim(case)
    hist = []
    for _ in range(STEPS):
        s.run(1)
        st = s.state()
        hist.append((st["x"][k].copy(), st["v"][k].copy()))
    return case, k, hist


@pytest.mark.parametrize("precision,tol", [(B.SDPD_PREC_FP64, 1e-9), (B.SDPD_PREC_SPLIT, 5e-3)])
def test_settling_sphere_follows_oracle(oracle_run, precision, tol):
    need_gpu()
    case, k, hist = oracle_run
    sim = B.Sim(case, precision=precision)
    scale = max(np.abs(h[1]).max() for h in hist)
    assert scale > 1e-3          # the sphere does move
    for n in range(STEPS):
        sim.step(1)
        st = sim.state(density=False)
        xo, vo = hist[n]
        assert np.max(np.abs(st["v"][k] - vo)) <= tol * scale, (n, st["v"][k], vo)
        assert np.max(np.abs(st["x"][k] - xo)) <= tol * case["params"]["dx"]
    sim.close()
