"""Apparent-viscosity surrogate workflow on top of the batched viscometer.

The paper measures the apparent viscosity of a slurry with the
reverse-Poiseuille viscometer (Section 4.1, Eqs. poiseuanasol and poiseuave;
slurries in Section 4.3).  This module adds a learned layer the paper does
not have:

  1. Sobol-sampled sweep points (solid fraction phi, temperature T, forcing
     amplitude g) run as uneven batches of viscometer instances in one
     graph-captured engine each (the batched path of the C ABI);
  2. the tensor-core network (mlp_* entry points) trained on log(mu_app / 25)
     with Adam, batch 256;
  3. inference on 10^6 query points on the tensor cores;
  4. proposal of sweep points (a target viscosity, or the largest ensemble
     disagreement), every proposal re-checked by the simulation, which stays
     both the fallback and the arbiter of the surrogate's error.

Instances are in the paper's mesoscale units (rho0 = 3, p0 = beta = 100,
alpha = 7, r_c = 3.9 dx); the viscosity follows an Arrhenius law in T scaled to
eta = 25 at 293.15 K, kBT = kbt_scale * T / 293.15, spheres of diameter 3 dx
and density 2.7 rho0 on random lattice sites, lubrication gap floored at
0.1 d.  The forcing amplitude spans one decade, 0.1 to 1: the peak velocity
of the lowest viscosity stays below 0.2 of the artificial sound speed, and at
the highest viscosity it stays above the thermal velocity sqrt(kBT/m).

Run as a program it generates a data set, trains, times the inference and
proposes points:  python -m paper_2002_03120_gb300.surrogate --runs 2000
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import binding as B
from . import cases
from .sobol import sobol

PHI = (0.0, 0.3)
TEMP = (280.0, 350.0)
AMP = (0.1, 1.0)
ETA_REF = 25.0


def points_from_unit(u: np.ndarray) -> np.ndarray:
    """Unit-cube points -> (phi, T, g): phi and T uniform, g log-uniform."""
    u = np.asarray(u, dtype=np.float64).reshape(-1, 3)
    phi = PHI[0] + u[:, 0] * (PHI[1] - PHI[0])
    T = TEMP[0] + u[:, 1] * (TEMP[1] - TEMP[0])
    g = AMP[0] * (AMP[1] / AMP[0]) ** u[:, 2]
    return np.stack([phi, T, g], axis=1)


def features(pts: np.ndarray) -> np.ndarray:
    """(phi, T, g) -> network inputs in [0, 1]^3 (inverse of points_from_unit)."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    u0 = (pts[:, 0] - PHI[0]) / (PHI[1] - PHI[0])
    u1 = (pts[:, 1] - TEMP[0]) / (TEMP[1] - TEMP[0])
    u2 = np.log(pts[:, 2] / AMP[0]) / math.log(AMP[1] / AMP[0])
    return np.stack([u0, u1, u2], axis=1).astype(np.float32)


def sweep_points(n: int, skip: int = 0) -> np.ndarray:
    return points_from_unit(sobol(n, 3, skip=skip))


def meso_dt(p) -> float:
    """Time step of a mesoscale instance: the acoustic limit 0.1 r_c / c and
    the explicit limit of the velocity-proportional pair forces.  The
    dissipative friction rate of one particle is about 3.7 eta at rho0 = 3
    and r_c = 3.9 dx (sum over ~250 neighbours of gamma_a (1 + 1/3) x 2);
    the drag and lubrication rates of a sphere (Ergun at eps ~ 0.5, gap at its
    floor of 0.1 d, several partners) scale with eta as well.  Velocity
    Verlet applied to a force -k v is stable for k dt < 4 and free of
    overshoot for k dt < 2; dt = 0.2 / eta keeps the fluid at 0.74 and the
    stiffest sphere configurations below 2."""
    c = math.sqrt(p["alpha"] * p["p0"] / p["rho0"])
    return min(0.1 * p["r_c"] / c, 0.2 / p["eta"])


def instance(pt, seed: int, n: int = 12, kbt_scale: float = 0.01) -> dict:
    phi, T, g = (float(v) for v in pt)
    c = cases.viscometer_instance(2 * n ** 3, phi, T, g, seed=seed, mesoscale=True,
                                  kBT=kbt_scale * T / 293.15, lub_gap_min=0.1)
    p = c["params"]
    p["dt"] = meso_dt(p)
    return c


def simulate(pts, seed: int = 0, n: int = 12, steps: int = 1500, avg: int = 500, every: int = 25,
             batch: int = 64, precision: int = B.SDPD_PREC_SPLIT, kbt_scale: float = 0.01,
             n_bins: int = 24) -> np.ndarray:
    """Apparent viscosity of every sweep point: run `steps` steps, average the
    probe over the last `avg` (one read-out every `every` steps).  Points run
    as batches of `batch` instances, one engine (one graph) per batch, with
    the autotuner's setting for the batch shape.  Non-finite or non-positive
    read-outs come back as NaN."""
    from . import autotune
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    mu = np.full(len(pts), np.nan)
    for b0 in range(0, len(pts), batch):
        chunk = pts[b0:b0 + batch]
        insts = [instance(pt, seed + b0 + k, n=n, kbt_scale=kbt_scale) for k, pt in enumerate(chunk)]
        # force variant, skin and block size for this batch shape (cached
        # after the first measurement of the size class)
        setting = autotune.tune(insts, precision=precision)
        sim = B.Sim(insts, precision=precision)
        autotune.apply(sim, setting)
        sim.step(steps - avg)
        acc = np.zeros(len(chunk))
        reads = 0
        for _ in range(avg // every):
            sim.step(every)
            acc += [sim.viscosity_probe(k, n_bins)[1] for k in range(len(chunk))]
            reads += 1
        m = acc / max(reads, 1)
        m[~np.isfinite(m) | (m <= 0)] = np.nan
        mu[b0:b0 + len(chunk)] = m
        sim.close()
    return mu


def target(mu):
    return np.log(np.asarray(mu, dtype=np.float64) / ETA_REF).astype(np.float32)


def from_target(y):
    return ETA_REF * np.exp(np.asarray(y, dtype=np.float64))


class Ensemble:
    """M independently initialised networks trained on the same data (each
    epoch in its own shuffled order); the spread of their predictions is the
    disagreement used to propose exploratory points."""

    def __init__(self, members: int = 4, seed: int = 0, batch: int = 256):
        self.batch = batch
        self.nets = [B.Mlp(seed=seed + 977 * m, batch_max=batch) for m in range(members)]

    def fit(self, X, y, epochs: int = 400, lr: float = 1e-3, seed: int = 0):
        import torch
        Xd = torch.as_tensor(np.asarray(X, dtype=np.float32), device="cuda")
        yd = torch.as_tensor(np.asarray(y, dtype=np.float32), device="cuda")
        n = Xd.shape[0]
        gen = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        for net in self.nets:
            for ep in range(epochs):
                order = torch.randperm(n, generator=gen).to("cuda")
                Xs, ys = Xd[order].contiguous(), yd[order].contiguous()
                for b0 in range(0, n, self.batch):
                    net.train_step(Xs[b0:b0 + self.batch], ys[b0:b0 + self.batch], lr=lr,
                                   want_loss=False)
            net.check()
            losses.append(float(((self.predict_one(net, Xd) - yd) ** 2).mean()))
        return losses

    @staticmethod
    def predict_one(net, Xd):
        import torch
        Y = torch.empty(Xd.shape[0], dtype=torch.float32, device="cuda")
        net.infer(Xd, Y)
        return Y

    def predict(self, Xd):
        """Mean and standard deviation over the members ([n] device tensors)."""
        import torch
        Ys = torch.stack([self.predict_one(net, Xd) for net in self.nets])
        return Ys.mean(0), Ys.std(0) if len(self.nets) > 1 else torch.zeros_like(Ys[0])


def propose(ens: Ensemble, mu_target: float, n_query: int = 1_000_000, k_target: int = 8,
            k_explore: int = 8, seed: int = 0):
    """Score n_query uniform points with the ensemble; return the k_target
    points whose predicted viscosity is closest to mu_target among the most
    confident half, and the k_explore points of largest disagreement."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    U = torch.rand(n_query, 3, generator=g).to("cuda")
    mean, std = ens.predict(U)
    yt = float(np.log(mu_target / ETA_REF))
    conf = std <= torch.quantile(std[: min(n_query, 1 << 20)], 0.5)
    miss = (mean - yt).abs() + torch.where(conf, 0.0, float("inf"))
    it = torch.topk(-miss, k_target).indices
    ie = torch.topk(std, k_explore).indices
    Uc = U.cpu().numpy().astype(np.float64)
    return (points_from_unit(Uc[it.cpu().numpy()]), mean[it].cpu().numpy(),
            points_from_unit(Uc[ie.cpu().numpy()]), mean[ie].cpu().numpy())


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--runs", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=128)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--avg", type=int, default=500)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--members", type=int, default=4)
    ap.add_argument("--target", type=float, default=40.0)
    ap.add_argument("--out", default=None, help="write the data set (npz) here")
    a = ap.parse_args(argv)
    import torch
    t0 = time.time()
    pts = sweep_points(a.runs, skip=1)
    mu = simulate(pts, seed=1, steps=a.steps, avg=a.avg)
    t_data = time.time() - t0
    ok = np.isfinite(mu)
    hpts = sweep_points(a.heldout, skip=1 + a.runs)
    hmu = simulate(hpts, seed=10 ** 6, steps=a.steps, avg=a.avg)
    if a.out:
        np.savez(a.out, pts=pts, mu=mu, hpts=hpts, hmu=hmu)
    t1 = time.time()
    ens = Ensemble(a.members, seed=3)
    losses = ens.fit(features(pts[ok]), target(mu[ok]), epochs=a.epochs)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    hok = np.isfinite(hmu)
    hm, _ = ens.predict(torch.as_tensor(features(hpts[hok]), device="cuda"))
    herr = np.abs(from_target(hm.cpu().numpy()) / hmu[hok] - 1.0)
    # without the surrogate: the fluid viscosity law mu(T) (solids ignored)
    eta_T = np.array([ETA_REF * cases.arrhenius_viscosity(T) / cases.arrhenius_viscosity(293.15)
                      for T in hpts[hok][:, 1]])
    lerr = np.abs(eta_T / hmu[hok] - 1.0)
    # 1e6-query inference, one network, CUDA events
    U = torch.rand(1_000_000, 3, device="cuda")
    Y = torch.empty(1_000_000, device="cuda")
    for _ in range(3):
        ens.nets[0].infer(U, Y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        ens.nets[0].infer(U, Y)
    e1.record()
    torch.cuda.synchronize()
    t_inf = e0.elapsed_time(e1) / 20 / 1e3
    pt_t, pred_t, pt_e, pred_e = propose(ens, a.target)
    mu_t = simulate(pt_t, seed=2 * 10 ** 6, steps=a.steps, avg=a.avg)
    mu_e = simulate(pt_e, seed=3 * 10 ** 6, steps=a.steps, avg=a.avg)
    rep = dict(runs=a.runs, valid=int(ok.sum()), data_s=t_data, train_s=t_train,
               train_mse=losses, heldout=int(hok.sum()),
               heldout_rel_err_median=float(np.median(herr)), heldout_rel_err_p90=float(np.quantile(herr, 0.9)),
               fluid_law_rel_err_median=float(np.median(lerr)), fluid_law_rel_err_p90=float(np.quantile(lerr, 0.9)),
               target_miss_median=float(np.nanmedian(np.abs(mu_t / a.target - 1.0))),
               sobol_target_miss_median=float(np.nanmedian(np.abs(hmu[:len(mu_t)] / a.target - 1.0))),
               infer_1e6_ms=t_inf * 1e3, infer_tflops=1e6 * flops_per_query() / t_inf / 1e12,
               target=a.target, proposed=pt_t.tolist(), predicted=from_target(pred_t).tolist(),
               simulated=mu_t.tolist(),
               proposal_rel_err=(np.abs(from_target(pred_t) / mu_t - 1.0)).tolist(),
               explore=pt_e.tolist(), explore_pred=from_target(pred_e).tolist(), explore_sim=mu_e.tolist())
    print(json.dumps(rep))
    return rep


def flops_per_query() -> int:
    """Multiply-adds x 2 of one forward pass (3 -> 4 x 128 -> 1)."""
    return 2 * (3 * 128 + 3 * 128 * 128 + 128)


if __name__ == "__main__":
    main()
