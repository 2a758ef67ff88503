"""Uploading state into a running context (sdpd_upload_state) keeps the
neighbour lists while the particles stay within half the Verlet skin of their
build positions: the continuation equals the run without the round trip bit
for bit, and moved particles give the oracle's step at the new positions,
with or without the rebuild that larger moves trigger."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import need_gpu, rel_l2

pytestmark = pytest.mark.gpu
PRECISIONS = [B.SDPD_PREC_FP64, B.SDPD_PREC_SPLIT]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _case():
    return cases.sedimentation(nx=12, ny=12, nz=24)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_round_trip_changes_nothing(precision):
    case = _case()
    a = B.Sim(case, precision=precision)
    a.step(5)
    a.step(5)
    sa = a.state(density=False)
    b = B.Sim(case, precision=precision)
    b.step(5)
    N = b.N
    x = np.zeros((N, 3)); v = np.zeros((N, 3)); w = np.zeros((N, 3))
    b.download_state(x, v, w)
    b.check()
    b.upload_state(x, v, w)
    b.step(5)
    sb = b.state(density=False)
    for k in ("x", "v", "w", "F", "N"):
        assert np.array_equal(sa[k], sb[k]), k


@pytest.mark.parametrize("precision,tol", [(B.SDPD_PREC_FP64, 1e-9), (B.SDPD_PREC_SPLIT, 1e-4)])
@pytest.mark.parametrize("move", [0.002, 0.05])   # fractions of h: inside and beyond half the skin
def test_moved_particles_step_like_the_oracle(precision, tol, move):
    case = _case()
    sim = B.Sim(case, precision=precision)
    sim.step(3)
    N = sim.N
    x = np.zeros((N, 3)); v = np.zeros((N, 3)); w = np.zeros((N, 3))
    sim.download_state(x, v, w)
    sim.check()
    rng = np.random.default_rng(11)
    mob = case["type"] <= 1
    h = case["params"]["r_c"]
    d = rng.normal(size=(N, 3))
    d *= (move * h / np.linalg.norm(d, axis=1))[:, None]
    x[mob] += d[mob]
    sim.upload_state(x, v, w)
    sim.step(1)
    g = sim.state(density=False)
    orc = oracle.OracleSim(case)
    orc.step = 3
    orc.set_state(x=x, v=v, w=w)
    orc.run(1)
    o = orc.state()
    assert rel_l2(g["v"][mob], o["v"][mob]) < tol
    # positions move by dt v: the velocity difference, scaled by dt / |x|
    assert rel_l2(g["x"], o["x"]) < (1e-12 if precision == B.SDPD_PREC_FP64 else 1e-9)
