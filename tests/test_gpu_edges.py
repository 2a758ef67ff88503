"""Edge cases of the GPU path against the oracle: a single particle, pairs
placed within a few ulp of the support radius h (the r < h decision must be
the oracle's), an empty instance inside a batch, a dry granular case (rigid
particles only: DEM, lubrication, contact history), and the surrogate network
on empty, single-row and single-sample inputs."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import TOL_FORCE, need_gpu, pair_set, rel_l2

pytestmark = pytest.mark.gpu
PRECISIONS = [B.SDPD_PREC_FP64, B.SDPD_PREC_SPLIT]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _subset(case, keep):
    out = dict(case)
    for k in ("x", "v", "w", "type", "radius", "mass"):
        out[k] = np.ascontiguousarray(case[k][keep])
    out["params"] = dict(case["params"])
    return out


@pytest.mark.parametrize("precision", PRECISIONS)
def test_single_particle(precision):
    c = cases.poiseuille_si(nx=12, ny=12, nz=12)
    c = _subset(c, np.array([5]))
    sim = B.Sim(c, precision=precision)
    sim.step_count = 1
    sim.evaluate(1)
    g = sim.state()
    o = oracle.OracleSim(c)
    o.step = 1
    o.evaluate(1)
    so = o.state()
    assert sim.pairs().shape[0] == 0
    # the self term W(0) alone; the split path sums in FP32
    tol = 1e-12 if precision == B.SDPD_PREC_FP64 else 1e-6
    assert g["d"][0] == pytest.approx(so["d"][0], rel=tol)
    np.testing.assert_allclose(g["F"], so["F"], rtol=tol, atol=0)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_pairs_straddling_h(precision):
    # a centre particle and neighbours at h (1 + delta) along random
    # directions, delta from a few ulp to 1e-7 on both sides
    c = cases.poiseuille_si(nx=16, ny=16, nz=16, jitter=0.0)
    p = c["params"]
    h = p["r_c"]
    centre = np.array(p["box"]) * 0.5 + 0.123e-3
    rng = np.random.default_rng(3)
    deltas = np.array([-1e-7, -1e-12, -4e-16, -2.2e-16, 0.0, 2.2e-16, 4e-16, 1e-12, 1e-7])
    pts = [centre]
    for dlt in deltas:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pts.append(centre + h * (1.0 + dlt) * u)
    x = np.array(pts)
    n = len(x)
    case = dict(c, x=x, v=rng.normal(0, 1e-3, (n, 3)), w=np.zeros((n, 3)), type=np.zeros(n, dtype=np.int32),
                radius=np.full(n, 0.5 * p["dx"]), mass=np.full(n, c["mass"][0]))
    sim = B.Sim(case, precision=precision)
    sim.step_count = 2
    sim.evaluate(1)
    o = oracle.OracleSim(case)
    o.step = 2
    o.evaluate(1)
    assert pair_set(sim.pairs()) == pair_set(o.pairs())
    assert rel_l2(sim.state()["F"], o.state()["F"]) < TOL_FORCE[precision]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_empty_instance_in_a_batch(precision):
    # the random stream is keyed by the instance index: without it the
    # instances of the batch repeat their single runs bit for bit
    a = cases.poiseuille_si(nx=12, ny=12, nz=12, seed=2, coeff_t=0.0)
    b = cases.sedimentation(nx=12, ny=12, nz=24, coeff_t=0.0)
    empty = _subset(cases.poiseuille_si(nx=12, ny=12, nz=12, seed=3), np.array([], dtype=np.int64))
    batch = B.Sim([a, empty, b], precision=precision)
    batch.step(3)
    for k, single_case in ((0, a), (2, b)):
        single = B.Sim(single_case, precision=precision)
        single.step(3)
        sb, ss = batch.state(k, density=False), single.state(density=False)
        for key in ("x", "v", "w"):
            assert np.array_equal(sb[key], ss[key]), (k, key)
    assert batch.state(1, density=False)["x"].shape == (0, 3)


def test_dry_granular_matches_oracle():
    # rigid particles only (spheres on random lattice sites, some touching),
    # random velocities: DEM contacts with history and lubrication
    c = cases.viscometer_instance(6000, 0.3, 300.0, 0.0, seed=9, mesoscale=True)
    c = _subset(c, c["type"] == 1)
    rng = np.random.default_rng(4)
    c["v"] = rng.normal(0, 0.5, c["v"].shape)
    sim = B.Sim(c, precision=B.SDPD_PREC_FP64)
    sim.step(6)
    o = oracle.OracleSim(c)
    o.run(6)
    g, so = sim.state(density=False), o.state()
    assert rel_l2(g["v"], so["v"]) < 1e-9
    # spins may stay at rounding level (no sliding contact yet): compare on
    # the scale of v / R
    scale = np.linalg.norm(so["v"]) / np.mean(c["radius"])
    assert np.linalg.norm(g["w"] - so["w"]) <= 1e-9 * scale


def test_network_on_empty_single_and_one_row():
    import torch
    from oracle import mlp_oracle as M
    order = ["W0", "b0", "W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]
    p = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in M.init_params(5).items()}
    net = B.Mlp(seed=0, batch_max=256)
    net.set_params(np.concatenate([p[k].reshape(-1) for k in order]))
    X0 = torch.empty((0, 3), device="cuda")
    net.infer(X0, torch.empty(0, device="cuda"))     # nothing to do, no error
    x = np.array([[0.3, 0.7, 0.1]], dtype=np.float32)
    Y = torch.empty(1, device="cuda")
    net.infer(torch.tensor(x, device="cuda"), Y)
    net.check()
    y_ref, cache = M.forward(p, x.astype(np.float64), "bf16")
    assert abs(Y.item() - y_ref[0]) <= 1e-3 * max(1.0, abs(y_ref[0]))
    t = np.array([0.5], dtype=np.float32)
    net.gradients(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    g = net.grads().astype(np.float64)
    g_ref = M.backward(p, cache, y_ref, t.astype(np.float64))
    gr = np.concatenate([g_ref[k].reshape(-1) for k in order])
    assert rel_l2(g, gr) < 5e-3
