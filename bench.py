#!/usr/bin/env python
"""Benchmark of the SDPD-DEM per-timestep interaction step on GB300.

Workload: single-particle sedimentation, 32 x 32 x 64 fluid lattice
(65,535 fluid + 1 DEM sphere, d = 4 dx, rho_s = 2500) with 4-layer
dummy-particle walls in z (8,192 wall particles), dx = 1 mm, h = 3.9 dx,
dt = 1e-5 s; synthetic seeded inputs.  A step is one full velocity-Verlet step
(both sub-steps: neighbour build, density, drag, forces, integration,
artificial viscosity).

Metric: SDPD-DEM pair updates/s = unordered pairs within h evaluated by the
force pass x 2 evaluations per step x steps / time; also timesteps/s.  The
headline runs the FP64 path; the split-precision path (FP32 pair arithmetic,
FP64 state) is measured beside it on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Multi-GPU (torchrun): every rank runs its own replica of the workload (the
instances are independent; no collective on the data path), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SDPD-DEM pair updates/s & timesteps/s on 1 GB300, vs plain FP64 GPU path"
UNIT = "pair updates/s"
WORKLOADS = {
    "sedimentation": "single-particle sedimentation 32x32x64 (65,535 fluid + 1 sphere + 8,192 wall)",
    "poiseuille": "reverse-Poiseuille 16x32x16 (8,192 fluid), fully periodic",
    "dambreak": "dam break 126x63x63 column (490,094 fluid + 10,000 spheres + 501,903 wall)",
    "batch": "batched viscometer sweep: 64 slurry instances, N_f log-uniform 20k-400k",
    "surrogate": "apparent-viscosity MLP 3-128-128-128-128-1 (GELU, BF16 tensor cores): "
                 "1e6-query inference; training epoch of 2,000 samples, batch 256",
}
# algorithmic flops of one evaluation of one unordered pair by the force pass
# (Eqs. FijC, FijD, FijR, FijT incl. Box-Muller; transcendentals counted as 1)
FLOPS_PER_PAIR = 160.0
# algorithmic bytes of the velver-1 update (kick + drift) of one mobile
# particle: read x, v, w, F, N (5 x 24 B) and m, I (2 x 8 B), write x, v, w
# (3 x 24 B)
INTEGRATE_BYTES = 208.0
# nominal ALU peaks from unit counts x maximum SM clock (152 SMs, 2070 MHz):
# FP64 2 DFMA/clk/SM, FP32 128 FFMA/clk/SM, 2 flops per FMA
FP64_PEAK_TF = 152 * 2 * 2 * 2070e6 / 1e12
FP32_PEAK_TF = 152 * 128 * 2 * 2070e6 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "split"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="sedimentation", choices=sorted(WORKLOADS))
    ap.add_argument("--paths", default="both", choices=["both", "main"],
                    help="also time the other precision path (both) or not")
    ap.add_argument("--max-neighbors", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (force variant, skin, block size) and use the defaults")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_case(workload="sedimentation"):
    from paper_2002_03120_gb300 import cases
    if workload == "sedimentation":
        return cases.sedimentation()
    if workload == "poiseuille":
        return cases.poiseuille_si()
    if workload == "dambreak":
        return cases.dam_break()
    return cases.viscometer_batch()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ------------------------------------------------------------------ native
def time_native(args, ws, rank, local):
    import torch
    import torch.distributed as dist

    from paper_2002_03120_gb300 import binding as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    case = make_case(args.workload)
    prec = B.SDPD_PREC_FP64 if args.precision == "fp64" else B.SDPD_PREC_SPLIT

    def run_path(precision):
        setting = None
        if not args.no_tune:
            from paper_2002_03120_gb300 import autotune
            setting = autotune.tune(case, precision=precision, max_neighbors=args.max_neighbors)
        sim = B.Sim(case, precision=precision, max_neighbors=args.max_neighbors)
        if setting:
            autotune.apply(sim, setting)
        sim.build_cells(stream)
        torch.cuda.synchronize()
        pairs = sim.count_pairs()
        with torch.cuda.stream(stream):
            sim.step(args.warmup, stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ms = []
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                sim.step(1, stream)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        total_ms = float(sum(ms))
        kernels = sim.graph_kernels()
        # dominant kernel (force pass, velver 1) timed alone on the stream it
        # is launched on, L2 flushed before each launch
        fms = []
        for _ in range(5):
            sim.evaluate(1, stream)  # build, density, drag for the current state
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.compute_forces(1, stream)
            b.record(stream)
            b.synchronize()
            fms.append(a.elapsed_time(b))
        # the density pass (density, EOS, and the filter or reinitialisation
        # where the workload has them) timed alone after a list build
        dms = []
        for _ in range(5):
            sim.build_cells(stream)
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.compute_density(stream)
            b.record(stream)
            b.synchronize()
            dms.append(a.elapsed_time(b))
        sim.couple_drag(stream)   # leave the stage sequence complete
        torch.cuda.synchronize()
        # the HBM-bound update kernel alone (velocity Verlet, velver 1: kick
        # and drift; the velver-2 call also runs the collision pass)
        ims = []
        for _ in range(5):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.integrate(1, stream)
            b.record(stream)
            b.synchronize()
            ims.append(a.elapsed_time(b))
        # end-to-end through the C ABI with host buffers: upload the step's
        # state from pinned memory, run the step, read the result back
        N = sim.N
        hx = torch.empty((N, 3), dtype=torch.float64, pin_memory=True)
        hv = torch.empty_like(hx)
        hw = torch.empty_like(hx)
        sim.download_state(hx, hv, hw, stream=stream)
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(max(3, args.steps // 2)):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.upload_state(hx, hv, hw, stream=stream)
            sim.step(1, stream)
            sim.download_state(hx, hv, hw, stream=stream)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        mobile = int(sum(int(np.sum(c["type"] <= 1)) for c in sim.cases))
        out = dict(pairs=pairs, ms=total_ms, per_step=ms, kernels=kernels,
                   force_ms=float(np.median(fms)), density_ms=float(np.median(dms)),
                   e2e_ms=float(np.mean(e2e_ms)),
                   integrate_ms=float(np.median(ims)), mobile=mobile, setting=setting,
                   e2e_bytes=3 * N * 3 * 8, clocks=clk.summary(), N=N)
        sim.close()
        return out

    main = run_path(prec)
    other = None
    if args.paths == "both":
        other = run_path(B.SDPD_PREC_SPLIT if prec == B.SDPD_PREC_FP64 else B.SDPD_PREC_FP64)
    return main, other


def time_surrogate(args, ws, rank, local):
    """The surrogate network: one step = one 10^6-query inference launch
    (inputs in HBM, L2 flushed before each); training throughput measured
    beside it on 2,000 Sobol samples with a smooth synthetic target."""
    import torch
    from paper_2002_03120_gb300 import binding as B
    from paper_2002_03120_gb300 import surrogate as S
    from paper_2002_03120_gb300.sobol import sobol
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    nq = 1_000_000
    g = torch.Generator(device="cpu").manual_seed(5 + rank)
    Xh = torch.rand(nq, 3, generator=g).pin_memory()
    X = Xh.to(dev)
    Y = torch.empty(nq, dtype=torch.float32, device=dev)
    Yh = torch.empty(nq, dtype=torch.float32).pin_memory()
    net = B.Mlp(seed=11, batch_max=256)
    U = sobol(2000, 3, skip=1).astype(np.float32)
    T = (np.sin(3 * U[:, 0]) + U[:, 1] * U[:, 2] - 0.5 * U[:, 2] ** 2).astype(np.float32)
    Ud, Td = torch.as_tensor(U, device=dev), torch.as_tensor(T, device=dev)
    torch.cuda.synchronize()

    def epoch():
        for b0 in range(0, 2000, 256):
            net.train_step(Ud[b0:b0 + 256], Td[b0:b0 + 256], lr=1e-3, stream=stream, want_loss=False)

    for _ in range(args.warmup):
        epoch()
        net.infer(X, Y, stream)
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            net.infer(X, Y, stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    tr = []
    for _ in range(max(3, args.steps // 4)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        epoch()
        b.record(stream)
        b.synchronize()
        tr.append(a.elapsed_time(b))
    e2e = []
    for _ in range(max(3, args.steps // 2)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            X.copy_(Xh, non_blocking=True)
            net.infer(X, Y, stream)
            Yh.copy_(Y, non_blocking=True)
            b.record(stream)
        b.synchronize()
        e2e.append(a.elapsed_time(b))
    net.check()
    t_ms = max_over_ranks(float(sum(ms)), ws)
    per = t_ms / args.steps
    fq = S.flops_per_query()
    achieved = nq * fq / (per / 1e3) / 1e12
    peak = measured_peaks().get("bf16_tflops") or 1900.0
    cnt = ncu_counters("counters_surrogate")
    rec = {
        "metric": "surrogate inference queries/s", "value": nq * args.steps * ws / (t_ms / 1e3),
        "unit": "queries/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 GEMM operands / f32 accumulate", "data": "synthetic",
        "config": {"workload": WORKLOADS["surrogate"], "queries_per_step": nq,
                   "l2": "flushed (256 MB write) before every timed launch",
                   "parallelism": f"replicas x{ws}"},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "roofline": {"kernel": "k_mlp_forward", "bound": "tensor", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": cnt.get("k_mlp_forward", {}).get("dram_bytes_per_launch"),
                     "flop_per_query": fq,
                     "pipe_util_ncu": None if not cnt else {
                         k: cnt["k_mlp_forward"][k + "_pct"] / 100.0
                         for k in ("tensor_pipe", "fma_pipe", "alu_pipe", "issue_active")},
                     "note": "peak = measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"},
        "e2e": {"value": nq / (float(np.mean(e2e)) / 1e3), "unit": "queries/s",
                "h2d_bytes_per_step": nq * 12, "d2h_bytes_per_step": nq * 4},
        "training": {"samples_per_s": 2000 / (float(np.median(tr)) / 1e3), "epoch_ms": float(np.median(tr)),
                     "adam_steps_per_epoch": 8, "batch": 256},
    }
    if rank == 0:
        print(json.dumps(rec))


def max_over_ranks(v, ws):
    """The largest value over the ranks (the job's time is its slowest
    rank's)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(seconds=15.0):
    """The FP64 oracle timed on this host's cores on a bounded sample of the
    workload: full steps of a 16x16x32 sedimentation box (1/8 of the lattice,
    same physics), until `seconds` of CPU time have elapsed."""
    import oracle
    from paper_2002_03120_gb300 import cases
    case = cases.sedimentation(nx=16, ny=16, nz=32)
    sim = oracle.OracleSim(case)
    sim.neighbors()
    pairs = _oracle_pairs(sim, case)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        sim.run(1)
        steps += 1
    dt = time.perf_counter() - t0
    return dict(value=pairs * 2 * steps / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"{steps} full steps of sedimentation 16x16x32 ({len(case['x'])} particles, "
                       f"{pairs} pairs/evaluation), FP64, single thread",
                steps_per_s=steps / dt)


def _oracle_pairs(sim, case):
    ij = sim.pairs()
    mob = case["type"] <= 1
    return int(np.sum(mob[ij[:, 0]] | mob[ij[:, 1]]))


def sources_sha(paths):
    """First 16 hex digits of the SHA-256 of the files' bytes, concatenated in order."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def ncu_counters(name="counters_sedimentation"):
    """ncu counters of profiled kernels (profiles/<name>.json), used only
    while the kernel source and the headers it compiles ("sources") are the
    ones that were profiled."""
    try:
        c = json.load(open(os.path.join(ROOT, "profiles", name + ".json")))
        if "sources" in c:
            ok = sources_sha(c["sources"]) == c["sources_sha256_16"]
        else:
            ok = sources_sha([c["source"]]) == c["source_sha256_16"]
        return c if ok else {}
    except Exception:
        return {}


def pipe_util(c, fp64):
    if not c:
        return None
    if fp64:
        return {"fp64_pipe": c["fp64_pipe_pct"] / 100.0, "lanes_active": c["threads_per_inst"] / 32.0}
    return {"fma_pipe": c["fma_pipe_pct"] / 100.0, "alu_pipe": c["alu_pipe_pct"] / 100.0,
            "issue_active": c["issue_active_pct"] / 100.0, "lanes_active": c["threads_per_inst"] / 32.0}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def main():
    args = parse()
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "native" else "gloo")
    if args.impl == "reference":
        if rank != 0:
            return
        ms = []
        import oracle
        from paper_2002_03120_gb300 import cases
        case = cases.sedimentation(nx=16, ny=16, nz=32)
        sim = oracle.OracleSim(case)
        sim.neighbors()
        pairs = _oracle_pairs(sim, case)
        for _ in range(args.warmup):
            sim.run(1)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            sim.run(1)
            ms.append((time.perf_counter() - t0) * 1e3)
        tot = sum(ms) / 1e3
        val = pairs * 2 * args.steps / tot
        sample = (f"sedimentation 16x16x32 ({len(case['x'])} particles) per step, the 32x32x64 "
                  f"workload's physics at 1/8 of its lattice; FP64 oracle, single thread")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ms)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS["sedimentation"], "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if args.workload == "surrogate":
        time_surrogate(args, ws, rank, local)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    main_r, other_r = time_native(args, ws, rank, local)
    t_max = max_over_ranks(main_r["ms"], ws)
    pairs = main_r["pairs"]
    value = pairs * 2 * args.steps * ws / (t_max / 1e3)
    steps_per_s = args.steps / (t_max / 1e3)
    other_val = other_r["pairs"] * 2 * args.steps / (other_r["ms"] / 1e3) if other_r else None
    peaks = measured_peaks()
    # ncu counters of the profiled kernels of this workload (the dam break's
    # were taken at half scale, DRAM bytes scaled by the particle ratio)
    cnt = ncu_counters({"sedimentation": "counters_sedimentation",
                        "dambreak": "counters_dambreak"}.get(args.workload, "none"))
    fp64 = args.precision == "fp64"
    integ_cnt = ncu_counters("counters_integrate").get(f"k_integrate<{'double' if fp64 else 'float'}>", {})
    # dominant kernel: the force pass (k_force_half + k_force_gather + the
    # sphere kernel), ALU bound; algorithmic flops = 160 per unordered pair
    force_flops = FLOPS_PER_PAIR * pairs
    achieved_tf = force_flops / (main_r["force_ms"] / 1e3) / 1e12
    other_tf = FLOPS_PER_PAIR * other_r["pairs"] / (other_r["force_ms"] / 1e3) / 1e12 if other_r else None
    def force_kernel(res, double):
        # the phase-1 kernel of the Newton-3 pass, or the direct pass
        n3 = (res or {}).get("setting") or {}
        name = "k_force_half" if n3.get("newton3", 1) else "k_force_fluid"
        return f"{name}<{'double' if double else 'float'}>"
    main_k = force_kernel(main_r, fp64)
    other_k = force_kernel(other_r, not fp64)
    fp64_peak_tf = FP64_PEAK_TF if fp64 else FP32_PEAK_TF
    rec = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32 pairs / f64 state",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "particles": main_r["N"], "pairs_per_eval": pairs,
                   "evals_per_step": 2, "precision": args.precision,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{ws}",
                   "tuning": main_r["setting"] or "defaults (newton3 1, skin 0.03, block 128)"},
        "timesteps_per_s": steps_per_s,
        "density_pass": {"ms_per_launch": main_r["density_ms"], "pairs": pairs,
                         "pair_evals_per_s": pairs / (main_r["density_ms"] / 1e3),
                         "note": "density + EOS (+ filter or reinitialisation where the workload "
                                 "has them) after a list build, L2 flushed, events on the stream"},
        "step_ms": {"min": float(np.min(main_r["per_step"])), "median": float(np.median(main_r["per_step"])),
                    "max": float(np.max(main_r["per_step"]))},
        "gpu_launches": main_r["kernels"] * args.steps,
        "clocks": main_r["clocks"],
        "roofline": {"kernel": ("force pass (k_force_half + k_force_gather + k_force_rigid), velver 1"
                                if main_k.startswith("k_force_half") else
                                "force pass (k_force_fluid + k_force_rigid), velver 1"),
                     "bound": "alu", "achieved": achieved_tf, "peak": fp64_peak_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / fp64_peak_tf,
                     "traffic": cnt.get(main_k, {}).get("dram_bytes_per_launch"),
                     "ms_per_launch": main_r["force_ms"],
                     "pipe_util_ncu": pipe_util(cnt.get(main_k), fp64),
                     "note": ("peak = %s nominal from unit counts x max clock (2070 MHz); "
                              "achieved counts 160 flop per unordered pair (both directions of the "
                              "direct pass count once); traffic = ncu DRAM bytes of %s per launch "
                              "(profiles/)") % ("FP64" if fp64 else "FP32", main_k)},
        "hbm_kernel": {"kernel": "k_integrate (velver 1: kick + drift)", "bound": "hbm",
                       "achieved": main_r["mobile"] * INTEGRATE_BYTES / (main_r["integrate_ms"] / 1e3) / 1e9,
                       "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                       "frac": (main_r["mobile"] * INTEGRATE_BYTES / (main_r["integrate_ms"] / 1e3) / 1e9
                                / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None,
                       "bytes_per_particle": INTEGRATE_BYTES, "particles": main_r["mobile"],
                       "ms_per_launch": main_r["integrate_ms"],
                       "fp64_pipe_ncu": integ_cnt.get("fp64_pipe_pct", 100.0) / 100.0 if integ_cnt else None,
                       "note": "peak = measured copy bandwidth (MEASURED_PEAKS.json); the kernel also "
                               "keeps the cell-relative mirrors current (xl64, dsp, A32, A64: about 190 B "
                               "more per particle), which the algorithmic bytes do not count.  Its bound "
                               "is the FP64 pipe, not HBM: the kicks (with the exactly rounded division), "
                               "the drift and the mirror updates are FP64 (fp64_pipe_ncu: busy fraction "
                               "from profiles/counters_integrate.json)"},
        "e2e": {"value": pairs * 2 / (main_r["e2e_ms"] / 1e3) * ws, "unit": UNIT,
                "h2d_bytes_per_step": main_r["e2e_bytes"], "d2h_bytes_per_step": main_r["e2e_bytes"]},
        "split_precision" if fp64 else "fp64_path": None if other_r is None else {
            "value": other_val, "unit": UNIT, "ms_per_step": other_r["ms"] / args.steps,
            "force_ms_per_launch": other_r["force_ms"], "tuning": other_r["setting"],
            "speedup_vs_fp64": (other_val / (value / ws)) if fp64 else None,
            "roofline": {"bound": "alu", "achieved": other_tf,
                         "peak": FP32_PEAK_TF if fp64 else FP64_PEAK_TF, "unit": "TFLOP/s",
                         "frac": other_tf / (FP32_PEAK_TF if fp64 else FP64_PEAK_TF),
                         "traffic": cnt.get(other_k, {}).get("dram_bytes_per_launch"),
                         "pipe_util_ncu": pipe_util(cnt.get(other_k), not fp64)}},
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")},
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == "sedimentation":
        rec["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(rec))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
