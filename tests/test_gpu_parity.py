"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs: neighbour sets bit-exact, density / pressure / forces / torques within
the stated tolerances, exact integrator, batched == single."""
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


def _cases_small():
    return {
        "periodic12": cases.poiseuille_si(nx=12, ny=12, nz=12),
        "config1_8192": cases.poiseuille_si(),
        "sediment_small": cases.sedimentation(nx=12, ny=12, nz=24),
        "dambreak_small": cases.dam_break(scale=0.15, n_spheres=40),
        "slurry_small": cases.viscometer_instance(6000, 0.2, 300.0, 1e-2, seed=9, mesoscale=True),
    }


CASES = _cases_small()


def _oracle_eval(case, velver=1, step=0):
    s = oracle.OracleSim(case)
    s.step = step
    s.evaluate(velver)
    return s


def _gpu_eval(case, precision, velver=1, step=0):
    sim = B.Sim(case, precision=precision)
    sim.step_count = step
    sim.evaluate(velver)
    return sim


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name", list(CASES))
def test_neighbour_sets_bit_exact(name, precision):
    case = CASES[name]
    sim = _gpu_eval(case, precision)
    orc = oracle.OracleSim(case)
    orc.neighbors()
    assert pair_set(sim.pairs()) == pair_set(orc.pairs())


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name", list(CASES))
def test_density_pressure_forces(name, precision):
    case = CASES[name]
    sim = _gpu_eval(case, precision, step=3)
    orc = _oracle_eval(case, step=3)
    g = sim.state()
    o = orc.state()
    # split: float kernel values (a few ulp each) under a compensated sum
    tol_d = 1e-12 if precision == B.SDPD_PREC_FP64 else 1e-6
    assert rel_l2(g["d"], o["d"]) < tol_d
    # pressure is a small difference of large terms: judged against p0
    p0 = case["params"]["p0"]
    assert np.max(np.abs(g["p"] - o["p"])) < (1e-9 if precision == 0 else 2e-4) * p0
    assert rel_l2(g["F"], o["F"]) < TOL_FORCE[precision]
    assert rel_l2(g["N"], o["N"]) < TOL_FORCE[precision]


def _moving(case, seed):
    """The case with random velocities and spins on its mobile particles, so
    that every term of the pair forces (dissipative, rotational, drag,
    lubrication) is non-zero."""
    c = dict(case)
    rng = np.random.default_rng(seed)
    mob = (c["type"] <= 1)[:, None]
    scale = 0.05 if c["params"]["dx"] == 1.0 else 1e-3
    c["v"] = np.where(mob, rng.normal(0, scale, c["v"].shape), 0.0)
    c["w"] = np.where(mob, rng.normal(0, scale / c["params"]["dx"], c["w"].shape), 0.0)
    return c


@pytest.mark.parametrize("velver", [1, 2])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name", ["sediment_small", "dambreak_small", "slurry_small"])
def test_forces_per_particle_type(name, precision, velver):
    # fluid and rigid particles judged separately (force and torque), so the
    # few spheres' pressure-gradient force, torque, drag reaction and contact
    # forces are held to the tolerance on their own
    case = _moving(CASES[name], 11)
    sim = _gpu_eval(case, precision, velver=velver, step=4)
    orc = _oracle_eval(case, velver=velver, step=4)
    errs = check_per_type(sim.state(), orc.state(), case["type"], TOL_FORCE[precision])
    assert "rigid" in errs and "fluid" in errs
    sim.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_forces_velver2_with_history(precision):
    case = CASES["dambreak_small"]
    sim = _gpu_eval(case, precision, velver=2, step=5)
    orc = _oracle_eval(case, velver=2, step=5)
    assert rel_l2(sim.state()["F"], orc.state()["F"]) < TOL_FORCE[precision]


@pytest.mark.parametrize("precision,tol_f", [(B.SDPD_PREC_FP64, 1e-11), (B.SDPD_PREC_SPLIT, 1e-5)])
@pytest.mark.parametrize("name", ["sediment_small", "slurry_small", "dambreak_small"])
def test_drag_parity(name, precision, tol_f):
    # eps from the rigid volumes (FP64, exact decisions) in both precisions;
    # the kernel-weighted fluid velocity in FP32 on the split path
    case = dict(CASES[name])
    rng = np.random.default_rng(4)
    case["v"] = np.where((case["type"] <= 1)[:, None], rng.normal(0, 0.05, case["v"].shape), 0.0)
    sim = _gpu_eval(case, precision)
    orc = _oracle_eval(case)
    eps_g, F_g = sim.drag()
    eps_o, _ = orc.fpi()
    rig = np.where(case["type"] == 1)[0]
    assert np.allclose(eps_g, eps_o[rig], rtol=1e-13, atol=0)
    assert rel_l2(F_g, orc.component("dg")[rig]) < tol_f


def test_config2_full_size_parity():
    # the benchmark workload (65,535 fluid + 1 sphere + 8,192 wall particles)
    case = cases.sedimentation()
    rng = np.random.default_rng(5)
    mob = case["type"] <= 1
    case["v"] = np.where(mob[:, None], rng.normal(0, 1e-3, case["v"].shape), 0.0)
    orc = _oracle_eval(case, step=11)
    o = orc.state()
    for precision in PRECISIONS:
        sim = _gpu_eval(case, precision, step=11)
        g = sim.state()
        assert pair_set(sim.pairs()) == pair_set(orc.pairs())
        assert rel_l2(g["F"], o["F"]) < TOL_FORCE[precision]
        assert rel_l2(g["N"], o["N"]) < TOL_FORCE[precision]
        check_per_type(g, o, case["type"], TOL_FORCE[precision])
        sim.close()


def test_integrator_is_bit_exact():
    # pair forces off, body force and boundaries on: both sides see the same
    # forces exactly, so velocity Verlet + wrap / reflection must agree bit
    # for bit over many steps.
    case = cases.sedimentation(nx=12, ny=12, nz=24, coeff_c=0.0, coeff_d=0.0, coeff_r=0.0,
                               coeff_t=0.0, artvis=0)
    case["params"]["g"] = [0.3, -0.2, -9.81]
    rng = np.random.default_rng(6)
    mob = case["type"] == 0
    case["v"] = np.where(mob[:, None], rng.normal(0, 0.5, case["v"].shape), 0.0)
    case["w"] = np.where(mob[:, None], rng.normal(0, 5.0, case["w"].shape), 0.0)
    # no sphere: DEM forces would differ in summation order
    keep = case["type"] != 1
    case = {k: (v[keep] if isinstance(v, np.ndarray) else v) for k, v in case.items()}
    sim = B.Sim(case, precision=B.SDPD_PREC_FP64)
    sim.step(40)
    orc = oracle.OracleSim(case)
    orc.run(40)
    g, o = sim.state(density=False), orc.state()
    assert np.array_equal(g["x"], o["x"])
    assert np.array_equal(g["v"], o["v"])
    assert np.array_equal(g["w"], o["w"])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_few_steps_track_oracle(precision):
    case = CASES["config1_8192"]
    sim = B.Sim(case, precision=precision)
    sim.step(3)
    orc = oracle.OracleSim(case)
    orc.run(3)
    g, o = sim.state(), orc.state()
    dx_g = g["x"] - case["x"]
    dx_o = o["x"] - case["x"]
    assert rel_l2(g["v"], o["v"]) < (1e-8 if precision == 0 else 5e-4)
    assert rel_l2(dx_g, dx_o) < (1e-8 if precision == 0 else 5e-4)


def test_stage_api_equals_step():
    # the graph reuses the skin list between sub-steps, the stage calls rebuild
    # every time: same pairs, summation order may differ
    case = CASES["sediment_small"]
    a = B.Sim(case, precision=B.SDPD_PREC_FP64)
    a.step(2)
    b = B.Sim(case, precision=B.SDPD_PREC_FP64)
    for _ in range(2):
        for velver in (1, 2):
            b.evaluate(velver)
            b.integrate(velver)
    sa, sb = a.state(density=False), b.state(density=False)
    assert rel_l2(sa["x"] - case["x"], sb["x"] - case["x"]) < 1e-10
    assert rel_l2(sa["v"], sb["v"]) < 1e-10
    assert a.step_count == b.step_count == 2


@pytest.mark.parametrize("precision", PRECISIONS)
def test_skin_list_reuse_keeps_exact_pairs(precision):
    # after several steps on a reused skin list the pairs within h are exactly
    # the oracle's at the current positions, and the trajectory does not
    # depend on the skin (rebuild every drift with skin 0)
    case = dict(CASES["dambreak_small"])
    rng = np.random.default_rng(8)
    mob = case["type"] <= 1
    case["v"] = np.where(mob[:, None], rng.normal(0, 0.05, case["v"].shape), 0.0)
    a = B.Sim(case, precision=precision)
    a.step(6)
    st = a.state()
    orc = oracle.OracleSim(dict(case, x=st["x"], v=st["v"], w=st["w"]))
    orc.neighbors()
    assert pair_set(a.pairs()) == pair_set(orc.pairs())
    b = B.Sim(case, precision=precision)
    b.set_skin(0.0)
    b.step(6)
    sb = b.state()
    tol = 1e-10 if precision == B.SDPD_PREC_FP64 else 1e-4
    assert rel_l2(st["v"], sb["v"]) < tol


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("newton3", [1, 0])
def test_noise_cache_equals_recomputation(precision, newton3):
    # the second evaluation of a step reads the normals of the first from the
    # cache (same counter, same bits): the trajectory equals the one that
    # draws them again, bit for bit, in both force passes
    case = CASES["periodic12"]
    case = dict(case, params=dict(case["params"], kBT=4.1e-15))
    out = []
    for on in (1, 0):
        sim = B.Sim(case, precision=precision)
        sim.set_force_mode(newton3)
        sim.set_noise_cache(on)
        sim.step(4)
        out.append(sim.state(density=False))
        sim.close()
    for k in ("x", "v", "w", "F", "N"):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_force_modes_agree():
    # Newton-3 half pairs and the direct pass: same trajectory up to rounding
    case = CASES["periodic12"]
    case = dict(case, params=dict(case["params"], kBT=4.1e-15))
    a = B.Sim(case, precision=B.SDPD_PREC_FP64)
    a.step(4)
    b = B.Sim(case, precision=B.SDPD_PREC_FP64)
    b.set_force_mode(0)
    b.step(4)
    assert rel_l2(a.state(density=False)["v"], b.state(density=False)["v"]) < 1e-10


@pytest.mark.parametrize("precision", PRECISIONS)
def test_deterministic(precision):
    case = CASES["dambreak_small"]
    outs = []
    for _ in range(2):
        sim = B.Sim(case, precision=precision)
        sim.step(5)
        outs.append(sim.state(density=False))
        sim.close()
    for k in ("x", "v", "w", "F", "N"):
        assert np.array_equal(outs[0][k], outs[1][k])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_batched_equals_single_and_oracle(precision):
    # Instances of one context are independent: with the noise off (its key
    # carries the instance number) every instance reproduces its own
    # single-instance context bit for bit; with the noise on, each matches the
    # oracle keyed with the same instance number.
    quiet = [dict(c, params=dict(c["params"], coeff_t=0.0))
             for c in (CASES["periodic12"], CASES["sediment_small"], CASES["slurry_small"])]
    multi = B.Sim(quiet, precision=precision)
    multi.step_count = 2
    multi.evaluate(1)
    for k, case in enumerate(quiet):
        single = _gpu_eval(case, precision, step=2)
        a, b = multi.state(k), single.state()
        assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["N"], b["N"])
        single.close()
    noisy = [CASES["periodic12"], CASES["sediment_small"], CASES["slurry_small"]]
    multi = B.Sim(noisy, precision=precision)
    multi.step_count = 2
    multi.evaluate(1)
    for k, case in enumerate(noisy):
        orc = oracle.OracleSim(case, inst=k)
        orc.step = 2
        orc.evaluate(1)
        o = orc.state()
        assert rel_l2(multi.state(k)["F"], o["F"]) < TOL_FORCE[precision]
        assert rel_l2(multi.state(k)["N"], o["N"]) < TOL_FORCE[precision]


def test_momentum_conserved_over_steps():
    case = cases.poiseuille_si(nx=12, ny=12, nz=12, g_amp=0.0, kBT=4.1e-15)
    sim = B.Sim(case, precision=B.SDPD_PREC_FP64)
    sim.step(200)
    d = sim.diagnostics()
    m = case["mass"][0]
    vth = np.sqrt(4.1e-15 / m)
    assert np.abs(d[:3]).max() < 1e-10 * m * vth * len(case["x"])
    assert d[8] == 0


def test_viscosity_probe_matches_oracle():
    case = cases.poiseuille_meso(nx=12, ny=24, nz=12)
    rng = np.random.default_rng(7)
    case["v"] = rng.normal(0, 1.0, case["v"].shape)
    sim = B.Sim(case)
    prof_g, mu_g = sim.viscosity_probe(0, 24)
    orc = oracle.OracleSim(case)
    prof_o, mu_o = orc.profile(24)
    assert np.allclose(prof_g, prof_o, rtol=1e-12, atol=1e-14)
    assert mu_g == pytest.approx(mu_o, rel=1e-12)


def test_count_pairs():
    case = CASES["config1_8192"]
    sim = _gpu_eval(case, B.SDPD_PREC_SPLIT)
    assert sim.count_pairs() == len(sim.pairs()) == 1_024_000


def test_capacity_overflow_is_reported():
    sim = B.Sim(CASES["periodic12"], max_neighbors=50)
    with pytest.raises(B.SdpdError) as e:
        sim.step(1)
    assert e.value.code == 4


def test_invalid_parameters_rejected():
    case = cases.poiseuille_si(nx=12, ny=12, nz=12)
    case["params"]["xi"] = 10 * case["params"]["eta"]  # gamma^a < 0
    with pytest.raises(B.SdpdError) as e:
        B.Sim(case)
    assert e.value.code == 1
    case = cases.poiseuille_si(nx=8, ny=12, nz=12)  # 8 dx < 3 h on x
    with pytest.raises(B.SdpdError) as e:
        B.Sim(case).step(1)
    assert e.value.code == 1


def test_stage_order_enforced():
    sim = B.Sim(CASES["periodic12"])
    with pytest.raises(B.SdpdError) as e:
        sim.compute_forces(1)
    assert e.value.code == 8


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name", ["config1_8192", "sediment_small", "dambreak_small"])
def test_newton3_equals_direct(name, precision):
    # the half-pair pass evaluates each unordered pair once; the direct pass
    # from both sides: same forces up to summation order
    case = CASES[name]
    a = _gpu_eval(case, precision, step=4)
    b = B.Sim(case, precision=precision)
    b.set_force_mode(0)
    b.step_count = 4
    b.evaluate(1)
    sa, sb = a.state(), b.state()
    if precision == B.SDPD_PREC_FP64:
        # the FP64 density of the half-pair path sums the same terms in the
        # same order as the full-list pass: identical
        assert np.array_equal(sa["d"], sb["d"])
    tol = 1e-12 if precision == B.SDPD_PREC_FP64 else 2e-5
    assert rel_l2(sa["F"], sb["F"]) < tol
    assert rel_l2(sa["N"], sb["N"]) < tol
    orc = _oracle_eval(case, step=4)
    assert rel_l2(sb["F"], orc.state()["F"]) < TOL_FORCE[precision]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name", ["periodic12", "dambreak_small"])
def test_density_reinit_matches_oracle(name, precision):
    # reading B5: Shepard reinitialisation of the summation density before
    # the pressure filter; densities, pressures and forces against the oracle
    case = dict(CASES[name])
    case["params"] = dict(case["params"], density_reinit=1)
    orc = _oracle_eval(case, step=2)
    sim = _gpu_eval(case, precision, step=2)
    so, sg = orc.state(), sim.state()
    tol_d = 1e-12 if precision == B.SDPD_PREC_FP64 else 1e-6
    assert rel_l2(sg["d"], so["d"]) < tol_d
    # the reinitialisation changed something on the free surface
    base = _oracle_eval(CASES[name], step=2).state()["d"]
    if name == "dambreak_small":
        assert rel_l2(so["d"], base) > 1e-6
    assert rel_l2(sg["F"], so["F"]) < TOL_FORCE[precision]
