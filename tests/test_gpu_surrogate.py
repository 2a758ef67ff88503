"""What the trained surrogate gains over the viscometer without it.

Training data: apparent viscosities of Sobol-sampled viscometer instances
(solid fraction, temperature, forcing) run as uneven batches on the engine,
in the paper's mesoscale units (Section 4.1; slurries of Section 4.3).  The
network is trained by the tensor-core kernels.  Checked:
  * data: the read-out at zero solids follows the input viscosity law, and
    the relative viscosity rises with the solid fraction (Section 4.3);
  * accuracy: on held-out sweep points the surrogate's error is well below
    that of the method's own answer without simulation (the pure-fluid
    viscosity law mu(T), ignoring the solids);
  * cost: one surrogate query costs less than 1e-6 of one simulated point;
  * proposals: for a target viscosity, the surrogate's proposals, re-checked
    by the simulation, land far closer to the target than as many sweep
    points chosen without it, and the simulation confirms the surrogate's
    predictions there."""
import time

import numpy as np
import pytest

from paper_2002_03120_gb300 import cases
from paper_2002_03120_gb300 import surrogate as S

from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu

N_TRAIN = 384


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _eta(pts):
    return np.array([25.0 * cases.arrhenius_viscosity(T) / cases.arrhenius_viscosity(293.15) for T in pts[:, 1]])


@pytest.fixture(scope="module")
def trained():
    import torch
    pts = S.sweep_points(N_TRAIN, skip=1)
    t0 = time.perf_counter()
    mu = S.simulate(pts, seed=1)
    t_sim = (time.perf_counter() - t0) / len(pts)
    ok = np.isfinite(mu)
    ens = S.Ensemble(members=2, seed=3)
    ens.fit(S.features(pts[ok]), S.target(mu[ok]), epochs=400)
    torch.cuda.synchronize()
    hp = S.sweep_points(32, skip=1 + N_TRAIN)
    hmu = S.simulate(hp, seed=10 ** 6)
    return dict(pts=pts, mu=mu, ok=ok, ens=ens, hp=hp, hmu=hmu, t_sim=t_sim)


def test_sweep_data_follow_the_physics(trained):
    pts, mu, ok = trained["pts"], trained["mu"], trained["ok"]
    assert ok.mean() > 0.98
    rel = mu / _eta(pts)
    lo = ok & (pts[:, 0] < 0.05)
    hi = ok & (pts[:, 0] > 0.2)
    # without solids the viscometer reads back the fluid viscosity law
    assert np.median(rel[lo]) == pytest.approx(1.0, abs=0.1)
    # solids raise the apparent viscosity
    assert np.median(rel[hi]) > np.median(rel[lo]) + 0.05


def test_surrogate_beats_the_fluid_law_on_held_out_points(trained):
    import torch
    hp, hmu, ens = trained["hp"], trained["hmu"], trained["ens"]
    m = np.isfinite(hmu)
    pm, _ = ens.predict(torch.as_tensor(S.features(hp[m]), device="cuda"))
    err_s = np.abs(S.from_target(pm.cpu().numpy()) / hmu[m] - 1.0)
    err_law = np.abs(_eta(hp[m]) / hmu[m] - 1.0)
    assert np.median(err_s) < 0.5 * np.median(err_law), (np.median(err_s), np.median(err_law))
    assert np.median(err_s) < 0.1


def test_query_cost_and_proposals(trained):
    import torch
    ens = trained["ens"]
    X = torch.rand(1_000_000, 3, device="cuda")
    Y = torch.empty(1_000_000, device="cuda")
    ens.nets[0].infer(X, Y)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    ens.nets[0].infer(X, Y)
    b.record()
    b.synchronize()
    per_query = a.elapsed_time(b) / 1e3 / 1e6
    assert per_query < 1e-6 * trained["t_sim"], (per_query, trained["t_sim"])
    target = 30.0
    pt, pred, _, _ = S.propose(ens, target, k_target=8, k_explore=0)
    mu_p = S.simulate(pt, seed=2 * 10 ** 6)
    miss_p = np.nanmedian(np.abs(mu_p / target - 1.0))
    # the same simulation budget without the surrogate: the next sweep points
    miss_sobol = np.nanmedian(np.abs(trained["hmu"][:8] / target - 1.0))
    assert miss_p < 0.5 * miss_sobol, (miss_p, miss_sobol, mu_p)
    assert miss_p < 0.15
    # the simulation judges the surrogate: its predictions at the proposals
    assert np.nanmedian(np.abs(S.from_target(pred) / mu_p - 1.0)) < 0.15
