"""Force-pass variants that must agree bit for bit over whole trajectories
(both sub-steps, the normals cache filled at velver 1 and read back at velver
2, fluid-sphere pairs with the drag reaction, walls, several instances in one
context):
* the pair stream (modes 2 and 3: the direct pass with the pairs within h
  compacted through shared memory and evaluated 32 at a time) and the lean
  direct pass (mode 5: fewer registers, the partner's records loaded after
  the r < h decision, at velver 1 through an async shared-memory ring) add
  the same terms in the same order as the direct pass (mode 0);
* the Newton-3 pass with pushed results (mode 4) hands the partner the same
  bits as the one whose partner rebuilds them (mode 1).
Each also matches the oracle within the force tolerance."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import TOL_FORCE, check_per_type, need_gpu, rel_l2

pytestmark = pytest.mark.gpu

PRECISIONS = [B.SDPD_PREC_FP64, B.SDPD_PREC_SPLIT]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _moving(case, seed):
    c = dict(case)
    rng = np.random.default_rng(seed)
    mob = (c["type"] <= 1)[:, None]
    scale = 0.05 if c["params"]["dx"] == 1.0 else 1e-3
    c["v"] = np.where(mob, rng.normal(0, scale, c["v"].shape), 0.0)
    c["w"] = np.where(mob, rng.normal(0, scale / c["params"]["dx"], c["w"].shape), 0.0)
    return c


CASES = {
    "sediment_small": lambda: cases.sedimentation(nx=12, ny=12, nz=24),
    "dambreak_small": lambda: cases.dam_break(scale=0.15, n_spheres=40),
    "slurry_batch": lambda: [cases.viscometer_instance(6000, 0.2, 300.0, 1e-2, seed=9, mesoscale=True),
                             cases.viscometer_instance(5000, 0.1, 330.0, 1e-2, seed=3, mesoscale=True)],
}


def _run(insts, precision, mode, cache=True, steps=3):
    sim = B.Sim(insts, precision=precision)
    sim.set_force_mode(mode)
    sim.set_noise_cache(cache)
    sim.step_count = 4
    sim.step(steps)
    out = [sim.state(k, density=False) for k in range(len(sim.cases))]
    sim.check()
    sim.close()
    return out


@pytest.mark.parametrize("cache", [True, False])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name", list(CASES))
def test_equal_variants_bit_for_bit(name, precision, cache):
    made = CASES[name]()
    insts = [_moving(c, 7 + k) for k, c in enumerate(made if isinstance(made, list) else [made])]
    for ref_mode, modes in ((0, (2, 3, 5)), (1, (4,))):
        ref = _run(insts, precision, ref_mode, cache)
        for mode in modes:
            got = _run(insts, precision, mode, cache)
            for a, b in zip(got, ref):
                for q in ("x", "v", "w", "F", "N"):
                    assert np.array_equal(a[q], b[q]), (ref_mode, mode, q)


@pytest.mark.parametrize("mode", [2, 4, 5])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_variants_match_oracle(precision, mode):
    case = _moving(cases.dam_break(scale=0.15, n_spheres=40), 12)
    sim = B.Sim(case, precision=precision)
    sim.set_force_mode(mode)
    sim.step_count = 6
    sim.evaluate(1)
    g = sim.state()
    orc = oracle.OracleSim(case)
    orc.step = 6
    orc.evaluate(1)
    o = orc.state()
    assert rel_l2(g["F"], o["F"]) < TOL_FORCE[precision]
    check_per_type(g, o, case["type"], TOL_FORCE[precision])
    sim.close()


@pytest.mark.parametrize("tpp", [2, 4])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_lanes_per_particle_sum_order_only(precision, tpp):
    # several lanes per particle change the summation order of the direct
    # pass and nothing else; the same on every run
    made = CASES["dambreak_small"]()
    insts = [_moving(made, 3)]

    def run():
        sim = B.Sim(insts, precision=precision)
        sim.set_force_mode(0)
        sim.set_threads_per_particle(tpp)
        sim.step_count = 4
        sim.step(2)
        out = sim.state(0, density=False)
        sim.check()
        sim.close()
        return out

    ref = _run(insts, precision, 0, True, steps=2)[0]
    a, b = run(), run()
    for q in ("x", "v", "w", "F", "N"):
        assert np.array_equal(a[q], b[q]), q
    tol = 1e-12 if precision == B.SDPD_PREC_FP64 else 1e-5
    assert rel_l2(a["F"], ref["F"]) < tol and rel_l2(a["N"], ref["N"]) < tol
