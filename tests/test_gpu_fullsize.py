"""Full-size workloads through the C ABI, in the configuration bench.py
times: forces of sampled particles against the oracle (which evaluates the
sample one by one on the full state), and properties of a few steps.

* dam break: 0.4 x 0.2 x 0.2 m column of 490,094 fluid particles with 10,000
  polydisperse spheres in a walled 1.0 x 0.2 x 0.6 m tank (~1.0 M particles),
  split precision;
* batched viscometer: 64 slurry instances (~8 M particles) in one context.
"""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import TOL_FORCE, check_per_type, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _sample(case, k, seed):
    rng = np.random.default_rng(seed)
    t = case["type"]
    fluid = np.where(t == 0)[0]
    rigid = np.where(t == 1)[0]
    idx = np.concatenate([rng.choice(fluid, min(k, len(fluid)), replace=False),
                          rng.choice(rigid, min(k // 10, len(rigid)), replace=False) if len(rigid) else []])
    return np.unique(idx.astype(np.int64))


def _moving(case, seed, scale=1e-3):
    """Seeded velocities and spins on the mobile particles, so that every
    force term (and the spheres' torques) is non-zero."""
    rng = np.random.default_rng(seed)
    mob = (case["type"] <= 1)[:, None]
    case["v"] = np.where(mob, rng.normal(0, scale, case["v"].shape), 0.0)
    case["w"] = np.where(mob, rng.normal(0, scale / case["params"]["dx"], case["w"].shape), 0.0)
    return case


def test_dam_break_full_size_sampled_parity():
    case = _moving(cases.dam_break(), 3)
    sim = B.Sim(case, precision=B.SDPD_PREC_SPLIT)
    sim.step_count = 7
    sim.evaluate(1)
    g = sim.state()
    idx = _sample(case, 400, 1)
    orc = oracle.OracleSim(case)
    orc.step = 7
    orc.set_sample(idx)
    orc.evaluate(1)
    o = orc.state()
    assert rel_l2(g["d"], o["d"]) < 1e-6
    assert rel_l2(g["F"][idx], o["F"][idx]) < TOL_FORCE[B.SDPD_PREC_SPLIT]
    assert rel_l2(g["N"][idx], o["N"][idx]) < TOL_FORCE[B.SDPD_PREC_SPLIT]
    errs = check_per_type(g, o, case["type"], TOL_FORCE[B.SDPD_PREC_SPLIT], idx)
    assert "rigid" in errs


def test_dam_break_full_size_steps():
    case = cases.dam_break()
    sim = B.Sim(case, precision=B.SDPD_PREC_SPLIT)
    sim.step(10)
    st = sim.state(density=False)
    mob = case["type"] <= 1
    lo = np.asarray(case["params"]["origin"])
    hi = lo + np.asarray(case["params"]["box"])
    x = st["x"][mob]
    assert np.all(x >= lo - 1e-12) and np.all(x <= hi + 1e-12)
    d = sim.diagnostics()
    assert d[8] == 0 and np.isfinite(d[5])
    # the column starts falling: gravity dominates the first steps
    v = st["v"][case["type"] == 0]
    assert v[:, 2].mean() < 0


def test_batched_viscometer_full_size():
    insts = [_moving(c, 100 + k) for k, c in enumerate(cases.viscometer_batch())]
    n = sum(len(c["x"]) for c in insts)
    assert n > 6_000_000
    sim = B.Sim(insts, precision=B.SDPD_PREC_SPLIT, max_neighbors=320)
    sim.step_count = 3
    sim.evaluate(1)
    sizes = np.array([len(c["x"]) for c in insts])
    for k in np.argsort(sizes)[:3]:
        case = insts[k]
        g = sim.state(int(k))
        idx = _sample(case, 300, int(k))
        orc = oracle.OracleSim(case, inst=int(k))
        orc.step = 3
        orc.set_sample(idx)
        orc.evaluate(1)
        o = orc.state()
        assert rel_l2(g["d"], o["d"]) < 1e-6
        assert rel_l2(g["F"][idx], o["F"][idx]) < TOL_FORCE[B.SDPD_PREC_SPLIT]
        check_per_type(g, o, case["type"], TOL_FORCE[B.SDPD_PREC_SPLIT], idx)
    sim.step(3)
    for k in range(len(insts)):
        assert sim.diagnostics(k)[8] == 0
