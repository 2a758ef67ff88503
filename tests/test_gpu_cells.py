"""Half-size cells of the neighbour search (sdpd_set_cell_factor 2: a
125-cell stencil, lists built one lane per candidate) against the FP64
oracle: the pairs within h exactly, forces per particle type within the
parity tolerances for every force variant, contacts of dry granular matter,
trajectories equal to full-size cells up to summation order, capacity
overflow reported, the largest list capacity, a crowded cell, and spheres
crowded enough that the sphere kernel pools its DEM pairs over several rounds."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import TOL_FORCE, check_per_type, need_gpu, pair_set, rel_l2

pytestmark = pytest.mark.gpu

PRECISIONS = [B.SDPD_PREC_FP64, B.SDPD_PREC_SPLIT]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


CASES = {
    "periodic12": cases.poiseuille_si(nx=12, ny=12, nz=12),
    "config1_8192": cases.poiseuille_si(),
    "sediment_small": cases.sedimentation(nx=12, ny=12, nz=24),
    "dambreak_small": cases.dam_break(scale=0.15, n_spheres=40),
    "slurry_small": cases.viscometer_instance(6000, 0.2, 300.0, 1e-2, seed=9, mesoscale=True),
}


def _moving(case, seed):
    c = dict(case)
    rng = np.random.default_rng(seed)
    mob = (c["type"] <= 1)[:, None]
    scale = 0.05 if c["params"]["dx"] == 1.0 else 1e-3
    c["v"] = np.where(mob, rng.normal(0, scale, c["v"].shape), 0.0)
    c["w"] = np.where(mob, rng.normal(0, scale / c["params"]["dx"], c["w"].shape), 0.0)
    return c


def _half(case, precision, max_neighbors=0):
    sim = B.Sim(case, precision=precision, max_neighbors=max_neighbors)
    sim.set_cell_factor(2)
    return sim


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name", list(CASES))
def test_half_cells_pair_sets_exact(name, precision):
    case = CASES[name]
    sim = _half(case, precision)
    sim.evaluate(1)
    orc = oracle.OracleSim(case)
    orc.neighbors()
    assert pair_set(sim.pairs()) == pair_set(orc.pairs())
    sim.close()


@pytest.mark.parametrize("mode", [1, 0, 5])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name", ["sediment_small", "dambreak_small", "slurry_small"])
def test_half_cells_forces_per_type(name, precision, mode):
    if mode == 5 and precision == B.SDPD_PREC_FP64:
        pytest.skip("the lean direct pass is FP32-only (FP64 runs the direct pass)")
    case = _moving(CASES[name], 11)
    for velver in (1, 2):
        sim = _half(case, precision)
        sim.set_force_mode(mode)
        sim.step_count = 4
        sim.evaluate(velver)
        orc = oracle.OracleSim(case)
        orc.step = 4
        orc.evaluate(velver)
        errs = check_per_type(sim.state(), orc.state(), case["type"], TOL_FORCE[precision])
        assert "fluid" in errs
        g, o = sim.state(), orc.state()
        tol_d = 1e-12 if precision == B.SDPD_PREC_FP64 else 1e-6
        assert rel_l2(g["d"], o["d"]) < tol_d
        sim.close()


@pytest.mark.parametrize("tpp", [2, 4])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_half_cells_lanes_per_particle(precision, tpp):
    # the direct pass with several lanes per particle on half-size cells
    case = _moving(CASES["sediment_small"], 5)
    sim = _half(case, precision)
    sim.set_force_mode(0)
    sim.set_threads_per_particle(tpp)
    sim.step_count = 2
    sim.evaluate(1)
    orc = oracle.OracleSim(case)
    orc.step = 2
    orc.evaluate(1)
    check_per_type(sim.state(), orc.state(), case["type"], TOL_FORCE[precision])
    sim.close()


def test_half_cells_dry_granular_contacts():
    # spheres only, some touching: contact-range entries (beyond h) and
    # their tangential history must be listed exactly as with full cells
    c = cases.viscometer_instance(6000, 0.3, 300.0, 0.0, seed=9, mesoscale=True)
    keep = c["type"] == 1
    c = dict(c, x=c["x"][keep], v=c["v"][keep], w=c["w"][keep], type=c["type"][keep],
             radius=c["radius"][keep], mass=c["mass"][keep])
    rng = np.random.default_rng(4)
    c["v"] = rng.normal(0, 0.5, c["v"].shape)
    sim = _half(c, B.SDPD_PREC_FP64)
    sim.step(6)
    o = oracle.OracleSim(c)
    o.run(6)
    g, so = sim.state(density=False), o.state()
    assert rel_l2(g["v"], so["v"]) < 1e-9
    scale = np.linalg.norm(so["v"]) / np.mean(c["radius"])
    assert np.linalg.norm(g["w"] - so["w"]) <= 1e-9 * scale


@pytest.mark.parametrize("precision", PRECISIONS)
def test_half_cells_trajectory_equals_full_cells(precision):
    # rebuilds inside the steps (skin list reuse, then drift past the skin):
    # the same pairs every evaluation, so the trajectories differ only by
    # summation order (split: also by the cell-relative FP32 coordinates)
    case = dict(CASES["dambreak_small"])
    rng = np.random.default_rng(8)
    mob = case["type"] <= 1
    case["v"] = np.where(mob[:, None], rng.normal(0, 0.05, case["v"].shape), 0.0)
    out = []
    for cells in (1, 2):
        sim = B.Sim(case, precision=precision)
        sim.set_cell_factor(cells)
        sim.step(8)
        out.append(sim.state(density=False))
        if cells == 2:
            orc = oracle.OracleSim(dict(case, x=out[-1]["x"], v=out[-1]["v"], w=out[-1]["w"]))
            orc.neighbors()
            assert pair_set(sim.pairs()) == pair_set(orc.pairs())
        sim.close()
    tol = 1e-10 if precision == B.SDPD_PREC_FP64 else 1e-4
    assert rel_l2(out[1]["v"], out[0]["v"]) < tol
    assert rel_l2(out[1]["x"], out[0]["x"]) < 1e-12


@pytest.mark.parametrize("mode", [1, 0])
def test_half_cells_batched_equals_single(mode):
    # an instance's lists and sums do not depend on the batch it is in (the
    # random stream is keyed by the instance index: the second one draws none)
    a = _moving(CASES["sediment_small"], 3)
    b = cases.poiseuille_si(nx=12, ny=12, nz=12, seed=2, coeff_t=0.0)
    batch = _half([a, b], B.SDPD_PREC_SPLIT)
    batch.set_force_mode(mode)
    batch.step(3)
    for k, single_case in ((0, a), (1, b)):
        single = _half(single_case, B.SDPD_PREC_SPLIT)
        single.set_force_mode(mode)
        single.step(3)
        sb, ss = batch.state(k, density=False), single.state(density=False)
        for key in ("x", "v", "w"):
            assert np.array_equal(sb[key], ss[key]), (k, key)
        single.close()
    batch.close()


def test_half_cells_overflow_is_reported():
    sim = _half(CASES["periodic12"], B.SDPD_PREC_SPLIT, max_neighbors=50)
    with pytest.raises(B.SdpdError) as e:
        sim.step(1)
    assert e.value.code == 4


def test_half_cells_largest_capacity():
    # at the largest list capacity the kernel's list buffers leave room for
    # one warp per block: the same lists, so the same forces bit for bit
    case = CASES["periodic12"]
    sim = _half(case, B.SDPD_PREC_FP64, max_neighbors=B.SDPD_MAX_NEIGHBORS)
    sim.evaluate(1)
    orc = oracle.OracleSim(case)
    orc.neighbors()
    assert pair_set(sim.pairs()) == pair_set(orc.pairs())
    ref = _half(case, B.SDPD_PREC_FP64)
    ref.evaluate(1)
    assert np.array_equal(sim.state()["F"], ref.state()["F"])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_half_cells_crowded_cell(precision):
    # a cluster of 300 particles inside one half cell: more than the 8-bit
    # cell offsets of the list buffer hold, so the cells around it are
    # scanned one lane per particle; the lists stay exact, the forces match
    base = cases.tiny_box(n=8, r_c_dx=1.6, jitter=0.1, seed=5)
    rng = np.random.default_rng(6)
    k = 300
    blob = 2.8 + rng.uniform(0.0, 0.5, (k, 3))   # inside cell 3 of 9 (width 8/9) per axis
    case = dict(base)
    case["x"] = np.concatenate([base["x"], blob])
    for key, fill in (("v", 0.0), ("w", 0.0)):
        case[key] = np.concatenate([base[key], np.full((k, 3), fill)])
    for key in ("type", "radius", "mass"):
        case[key] = np.concatenate([base[key], np.full(k, base[key][0])])
    sim = _half(case, precision, max_neighbors=1024)
    sim.evaluate(1)
    orc = oracle.OracleSim(case)
    orc.neighbors()
    assert pair_set(sim.pairs()) == pair_set(orc.pairs())
    orc.evaluate(1)
    assert rel_l2(sim.state()["F"], orc.state()["F"]) < TOL_FORCE[precision]
    sim.close()


@pytest.mark.parametrize("cells", [1, 2])
def test_crowded_spheres_pool_over_several_rounds(cells):
    # spheres only, about 71 sphere neighbours each (kernel radius 2.5
    # spacings), many in contact: a block's four spheres pool about 280 sphere
    # pairs, so the pooled DEM and lubrication run over several rounds and the
    # history slots continue across them
    c = cases.tiny_box(n=8, r_c_dx=2.5, jitter=0.15, seed=7)
    n = len(c["x"])
    c = dict(c, type=np.ones(n, dtype=c["type"].dtype), radius=np.full(n, 0.55),
             mass=np.full(n, c["params"]["rho0"] * 4.0 / 3.0 * np.pi * 0.55 ** 3 * 2.7))
    c["v"] = np.random.default_rng(3).normal(0, 0.05, (n, 3))
    sim = B.Sim(c, precision=B.SDPD_PREC_FP64)
    sim.set_cell_factor(cells)
    sim.step(6)
    o = oracle.OracleSim(c)
    o.run(6)
    g, so = sim.state(density=False), o.state()
    assert rel_l2(g["v"], so["v"]) < 1e-9
    scale = np.linalg.norm(so["v"]) / 0.55
    assert np.linalg.norm(g["w"] - so["w"]) <= 1e-9 * scale
    sim.close()


def test_cell_factor_rejects_other_values():
    sim = B.Sim(CASES["periodic12"], precision=B.SDPD_PREC_SPLIT)
    for bad in (0, 3, -1):
        with pytest.raises(B.SdpdError) as e:
            sim.set_cell_factor(bad)
        assert e.value.code == B.SDPD_E_INVALID
    sim.set_cell_factor(1)
    sim.step(1)
