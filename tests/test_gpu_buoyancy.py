"""Buoyancy through the pressure-gradient force (Eq. F_fpi_PG, reading G17:
F^PG_s = V_s d_s sum_j (F^C + F^D)_sj): a neutrally buoyant sphere in a relaxed
hydrostatic column (mesoscale units, walls below and above) feels no net
force, i.e. F^PG balances its weight m_s g = rho_f V_s g.  A wrong volume or
density factor in F^PG, or its sign, leaves a net force of order m_s g."""
import numpy as np
import pytest

from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("precision", [B.SDPD_PREC_FP64, B.SDPD_PREC_SPLIT])
def test_neutrally_buoyant_sphere_feels_no_net_force(precision):
    case = cases.buoyancy_column()
    rig = np.where(case["type"] == 1)[0][0]
    ms, g = case["mass"][rig], -case["params"]["g"][2]
    sim = B.Sim(case, precision=precision)
    sim.step(600)                      # the column relaxes (about 7 viscous times)
    fz = []
    for _ in range(20):
        sim.step(10)
        fz.append(sim.state(density=False)["F"][rig, 2])
    # net vertical force on the sphere, averaged over the last 200 steps
    assert abs(np.mean(fz)) <= 0.05 * ms * g, (np.mean(fz), ms * g)
    # the weight alone would be -m g: F^PG carries +m g
    assert np.mean(fz) > -0.5 * ms * g
