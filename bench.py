#!/usr/bin/env python
"""Benchmark of the SDPD-DEM per-timestep interaction step on GB300.

Default workload: the batched viscometer sweep, 64 reverse-Poiseuille slurry
instances (fluid counts log-uniform in 20k-400k, solid fraction 0-30 % of
DEM spheres of diameter 3 dx, temperature 280-350 K, forcing 1e-3-1e-1 m/s^2;
about 9.46M particles) in one context, FP32 pair forces on FP64 state, one
graph-captured launch sequence per step, autotuned; synthetic seeded inputs.
A step is one full velocity-Verlet step (both sub-steps: neighbour build,
density, drag, forces, integration) of every instance.

Metric: SDPD-DEM pair updates/s = unordered pairs within h evaluated by the
force pass x 2 evaluations per step x steps / time; also timesteps/s.  The
plain FP64 GPU path (double pair arithmetic, one context per instance, stage
calls without a graph, default tuning) is timed beside it on the same GPU.
Other workloads: --workload sedimentation | poiseuille | dambreak | surrogate.

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
# nominal ALU peaks from unit counts x maximum SM clock (152 SMs, 2070 MHz),
# context only: the rooflines divide by the rates sdpd_alu_peaks measures;
# FP64 2 DFMA/clk/SM, FP32 128 FFMA/clk/SM, 2 flops per FMA
FP64_PEAK_TF = 152 * 2 * 2 * 2070e6 / 1e12
FP32_PEAK_TF = 152 * 128 * 2 * 2070e6 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # the viscometers start from rest; by about step 25 the lists need a
    # rebuild every few steps, so the default window runs past that point
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="batch", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "split"],
                    help="pair arithmetic of the timed path (auto: the workload's own, "
                         "split for the batch and the dam break, fp64 otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", default="both", choices=["both", "main"],
                    help="also time the comparison path (both) or not")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the plain FP64 comparison path (per instance)")
    ap.add_argument("--max-neighbors", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (force variant, skin, block size) and use the defaults")
    ap.add_argument("--cells", type=int, default=0, choices=[0, 1, 2],
                    help="cell factor of the neighbour search (1 full, 2 half-size cells); "
                         "0: the autotuner's choice (1 with --no-tune)")
    a = ap.parse_args()
    if a.precision == "auto":
        a.precision = "split" if a.workload in ("batch", "dambreak") else "fp64"
    return a


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
def _timed(stream, fn, flush=None):
    """Milliseconds of fn() on `stream` by CUDA events, L2 flushed before."""
    import torch
    if flush is not None:
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


def time_graph_path(case, precision, args, local, stream, flush, ws):
    """The product path: one context holding every instance of the workload,
    autotuned, whole steps replayed from the captured CUDA graph.  Also times
    the dominant kernel (force pass), the density pass and the update alone,
    and the end-to-end step through the C ABI with host buffers."""
    import torch
    import torch.distributed as dist

    from paper_2002_03120_gb300 import binding as B
    setting = None
    if not args.no_tune:
        from paper_2002_03120_gb300 import autotune
        setting = autotune.tune(case, precision=precision, max_neighbors=args.max_neighbors)
    sim = B.Sim(case, precision=precision, max_neighbors=args.max_neighbors)
    if setting:
        from paper_2002_03120_gb300 import autotune
        autotune.apply(sim, setting)
    if args.cells:
        sim.set_cell_factor(args.cells)
        setting = dict(setting or {}, cells=args.cells)
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
    builds0 = sim.build_count()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            ms.append(_timed(stream, lambda: sim.step(1, stream), flush))
    builds = sim.build_count() - builds0   # list builds the skin triggered inside the timed steps
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    kernels = sim.graph_kernels()
    # end-to-end through the C ABI with host buffers, right after the timed
    # steps (the loops below move the state in ways a run would not): upload
    # the step's state from pinned memory, run the step, read the result back
    N = sim.N
    hx = torch.empty((N, 3), dtype=torch.float64, pin_memory=True)
    hv = torch.empty_like(hx)
    hw = torch.empty_like(hx)
    sim.download_state(hx, hv, hw, stream=stream)
    torch.cuda.synchronize()

    def e2e_step():
        sim.upload_state(hx, hv, hw, stream=stream)
        sim.step(1, stream)
        sim.download_state(hx, hv, hw, stream=stream)
    e2e_ms = [_timed(stream, e2e_step, flush) for _ in range(max(3, args.steps // 2))]
    # dominant kernel (force pass, velver 1) timed alone on the stream it is
    # launched on, L2 flushed before each launch
    fms = []
    for _ in range(5):
        sim.evaluate(1, stream)  # build, density, drag for the current state
        fms.append(_timed(stream, lambda: sim.compute_forces(1, stream), flush))
    # the density pass (density, EOS, and the filter or reinitialisation
    # where the workload has them) timed alone after a list build
    dms = []
    for _ in range(5):
        sim.build_cells(stream)
        dms.append(_timed(stream, lambda: sim.compute_density(stream), flush))
    # the list build alone (counting sort, mirrors, lists; reverse index for
    # the Newton-3 passes), forced
    bms = [_timed(stream, lambda: sim.build_cells(stream), flush) for _ in range(5)]
    sim.compute_density(stream)
    sim.couple_drag(stream)   # leave the stage sequence complete
    torch.cuda.synchronize()
    # the HBM-bound update kernel alone (velocity Verlet, velver 1)
    ims = [_timed(stream, lambda: sim.integrate(1, stream), flush) for _ in range(5)]
    mobile = int(sum(int(np.sum(c["type"] <= 1)) for c in sim.cases))
    out = dict(pairs=pairs, ms=float(sum(ms)), per_step=ms, kernels=kernels,
               force_ms=float(np.median(fms)), density_ms=float(np.median(dms)),
               build_ms=float(np.median(bms)),
               e2e_ms=float(np.mean(e2e_ms)), e2e_per_step=[float(t) for t in e2e_ms], builds=builds,
               integrate_ms=float(np.median(ims)), mobile=mobile,
               setting=setting, e2e_bytes=3 * N * 3 * 8, clocks=clk.summary(), N=N,
               instances=len(sim.cases))
    sim.close()
    return out


def time_plain_fp64(case, args, stream, flush):
    """The plain FP64 GPU path the metric compares with: the same kernels with
    double pair arithmetic, each instance in a context of its own, the stages
    launched one by one (no CUDA graph), default tuning.  Returns the summed
    per-step time over the instances and the pairs evaluated per step."""
    import torch

    from paper_2002_03120_gb300 import binding as B
    insts = case if isinstance(case, list) else [case]
    steps = max(1, args.fp64_steps)
    tot_ms = 0.0
    pairs = 0
    for c in insts:
        sim = B.Sim(c, precision=B.SDPD_PREC_FP64, max_neighbors=args.max_neighbors)

        def one_step():
            for velver in (1, 2):
                sim.build_cells(stream)
                sim.compute_density(stream)
                sim.couple_drag(stream)
                sim.compute_forces(velver, stream)
                sim.integrate(velver, stream)
        sim.build_cells(stream)
        torch.cuda.synchronize()
        pairs += sim.count_pairs()
        one_step()   # warm-up
        tot_ms += sum(_timed(stream, one_step, flush) for _ in range(steps)) / steps
        sim.check()
        sim.close()
    return dict(ms_per_step=tot_ms, pairs=pairs, steps=steps, instances=len(insts))


def force_kernel_name(mode, split):
    """The pair kernel that does the arithmetic of a force mode (the phase-1
    kernel of the Newton-3 passes), as ncu names it."""
    r = "float" if split else "double"
    if mode in (1, 4):
        return f"k_force_half<{r}, {'true' if mode == 4 or not split else 'false'}>"
    if mode in (2, 3):
        return f"k_force_stream<{r}, {mode if split else 1}>"
    if mode == 5 and split:
        return "k_force_fluid_lean<float, 5, 2, 0>"   # velver 1: with the async record ring
    return f"k_force_fluid<{r}, 0>"


def time_native(args, ws, rank, local):
    import torch

    from paper_2002_03120_gb300 import binding as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    case = make_case(args.workload)
    peaks = B.alu_peaks()   # this GPU's FP32 / FP64 / INT32 rates at its current clock
    prec = B.SDPD_PREC_FP64 if args.precision == "fp64" else B.SDPD_PREC_SPLIT
    main = time_graph_path(case, prec, args, local, stream, flush, ws)
    other = None
    if args.paths == "both":
        if prec == B.SDPD_PREC_SPLIT:
            other = time_plain_fp64(case, args, stream, flush)
        else:
            other = time_graph_path(case, B.SDPD_PREC_SPLIT, args, local, stream, flush, 1)
    return main, other, peaks


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


def oracle_sample(workload, case=None):
    """A bounded sample of the workload the oracle can step in seconds: the
    smallest instance of the batch (full size), or a smaller box of the
    single-instance workloads with the same physics."""
    from paper_2002_03120_gb300 import cases
    if workload == "batch":
        insts = case if case is not None else cases.viscometer_batch()
        sizes = [len(c["x"]) for c in insts]
        k = int(np.argmin(sizes))
        return insts[k], k, f"instance {k} of the 64-instance batch ({sizes[k]} particles, full size)"
    if workload == "dambreak":
        c = cases.dam_break(scale=0.25, n_spheres=156)
        return c, 0, f"dam break at 1/4 linear scale ({len(c['x'])} particles, 156 spheres)"
    if workload == "poiseuille":
        c = cases.poiseuille_si()
        return c, 0, f"reverse Poiseuille 16x32x16 ({len(c['x'])} particles, full size)"
    c = cases.sedimentation(nx=16, ny=16, nz=32)
    return c, 0, f"sedimentation 16x16x32 ({len(c['x'])} particles, 1/8 of the lattice)"


def cpu_baseline(workload, seconds=12.0, case=None):
    """The FP64 oracle, as it stands, timed on this host's cores on a bounded
    sample of the workload: full steps of oracle_sample() until `seconds`
    have elapsed, once on one thread and once on every core (OpenMP over
    particles; the same results)."""
    import oracle
    case, inst, what = oracle_sample(workload, case)
    nproc = os.cpu_count() or 1
    runs = {}
    for nt in (1, nproc):
        used = oracle.threads(nt)
        sim = oracle.OracleSim(case, inst=inst)
        sim.neighbors()
        pairs = _oracle_pairs(sim, case)
        sim.run(1)   # warm-up step
        t0 = time.perf_counter()
        steps = 0
        while time.perf_counter() - t0 < seconds or steps == 0:
            sim.run(1)
            steps += 1
        dt = time.perf_counter() - t0
        runs[nt] = dict(value=pairs * 2 * steps / dt, steps=steps, seconds=dt, threads=used,
                        steps_per_s=steps / dt, pairs=pairs)
    allc = runs[nproc]
    one = runs[1]
    return dict(value=allc["value"], unit=UNIT, cores=allc["threads"], kind="oracle",
                sample=f"{allc['steps']} full steps of {what}, {allc['pairs']} pairs/evaluation, FP64, "
                       f"{allc['threads']} threads (all host cores)",
                steps_per_s=allc["steps_per_s"], host_cores=nproc, host_cpu=_cpu_name(),
                single_thread={"value": one["value"], "unit": UNIT, "cores": 1,
                               "sample": f"{one['steps']} full steps of the same sample, 1 thread",
                               "steps_per_s": one["steps_per_s"]})


def _cpu_name():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


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
    """Pipe utilisation of a profiled kernel (fractions), from whatever the
    counters file holds for it; None without a capture."""
    if not c:
        return None
    keys = ({"fp64_pipe": "fp64_pipe_pct", "lanes_active": "threads_per_inst"} if fp64 else
            {"fma_pipe": "fma_pipe_pct", "alu_pipe": "alu_pipe_pct", "issue_active": "issue_active_pct",
             "lanes_active": "threads_per_inst"})
    out = {k: c[v] / (32.0 if v == "threads_per_inst" else 100.0) for k, v in keys.items() if v in c}
    return out or None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def reference_arm(args):
    """bench.py --impl reference: the oracle, as it stands, on every host core,
    each step one full step of the bounded sample of the workload."""
    import oracle
    case, inst, what = oracle_sample(args.workload)
    cores = oracle.threads(os.cpu_count() or 1)
    sim = oracle.OracleSim(case, inst=inst)
    sim.neighbors()
    pairs = _oracle_pairs(sim, case)
    for _ in range(args.warmup):
        sim.run(1)
    ms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sim.run(1)
        ms.append((time.perf_counter() - t0) * 1e3)
    tot = sum(ms) / 1e3
    val = pairs * 2 * args.steps / tot
    sample = f"{what} per step; FP64 oracle on {cores} threads (all host cores)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ms)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample": sample},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    args = parse()
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "native" else "gloo")
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    if args.workload == "surrogate":
        time_surrogate(args, ws, rank, local)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    main_r, other_r, alu = time_native(args, ws, rank, local)
    t_max = max_over_ranks(main_r["ms"], ws)
    pairs = main_r["pairs"]
    value = pairs * 2 * args.steps * ws / (t_max / 1e3)
    split = args.precision == "split"
    peaks = measured_peaks()
    # ncu counters of the profiled kernels of this workload (captured on a
    # reduced case, DRAM bytes scaled by the particle ratio; see profiles/)
    cnt = ncu_counters({"sedimentation": "counters_sedimentation", "dambreak": "counters_dambreak",
                        "batch": "counters_batch"}.get(args.workload, "none"))
    integ_cnt = ncu_counters("counters_integrate").get(f"k_integrate<{'float' if split else 'double'}>", {})
    main_k = force_kernel_name((main_r.get("setting") or {}).get("newton3", 1), split)
    # the force pass is bound by arithmetic issue: algorithmic flops = 160 per
    # unordered pair, against this GPU's measured FMA rate of the path's
    # precision (sdpd_alu_peaks, run at the start of this bench)
    peak_tf = alu["fp32_tflops"] if split else alu["fp64_tflops"]
    achieved_tf = FLOPS_PER_PAIR * pairs / (main_r["force_ms"] / 1e3) / 1e12
    rec = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 pairs / f64 state" if split else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "instances": main_r["instances"],
                   "particles": main_r["N"], "pairs_per_eval": pairs, "evals_per_step": 2,
                   "precision": args.precision,
                   "l2": "inputs larger than L2, and L2 flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{ws}",
                   "tuning": main_r["setting"] or "defaults (newton3 1, skin 0.03, block 128)"},
        "timesteps_per_s": args.steps / (t_max / 1e3),
        "density_pass": {"ms_per_launch": main_r["density_ms"], "pairs": pairs,
                         "pair_evals_per_s": pairs / (main_r["density_ms"] / 1e3),
                         "note": "density + EOS (+ filter or reinitialisation where the workload "
                                 "has them) after a list build, L2 flushed, events on the stream"},
        "list_build": {"ms_per_build": main_r["build_ms"], "builds_in_timed_steps": main_r["builds"],
                       "note": "one forced build (cell sort, mirrors, neighbour lists, reverse index "
                               "where the force variant needs it), L2 flushed, events on the stream; "
                               "inside the timed steps builds run only when the skin is exceeded"},
        "step_ms": {"samples": [round(float(t), 3) for t in main_r["per_step"]],
                    "min": float(np.min(main_r["per_step"])), "median": float(np.median(main_r["per_step"])),
                    "max": float(np.max(main_r["per_step"]))},
        "gpu_launches": main_r["kernels"] * args.steps,
        "clocks": main_r["clocks"],
        "roofline": {"kernel": f"force pass ({main_k} with the sphere kernel), velver 1",
                     "bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / peak_tf,
                     "traffic": cnt.get(main_k, {}).get("dram_bytes_per_launch"),
                     "ms_per_launch": main_r["force_ms"],
                     "pipe_util_ncu": pipe_util(cnt.get(main_k), not split),
                     "note": ("peak = this GPU's %s FMA rate measured by sdpd_alu_peaks at the start of "
                              "this run (register-resident FMA chains, CUDA events); achieved counts 160 "
                              "flop per unordered pair (both directions of the direct pass count once); "
                              "the Philox integer work is on top (see alu_peaks.int32_tops); traffic = ncu "
                              "DRAM bytes of %s per launch (profiles/)") % ("FP32" if split else "FP64", main_k)},
        "alu_peaks": {**alu, "nominal_fp32_tflops": FP32_PEAK_TF, "nominal_fp64_tflops": FP64_PEAK_TF,
                      "note": "measured at the clock of this run; nominal = unit counts x 2070 MHz"},
        "hbm_kernel": {"kernel": "k_integrate (velver 1: kick + drift)", "bound": "hbm",
                       "achieved": main_r["mobile"] * INTEGRATE_BYTES / (main_r["integrate_ms"] / 1e3) / 1e9,
                       "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                       "frac": (main_r["mobile"] * INTEGRATE_BYTES / (main_r["integrate_ms"] / 1e3) / 1e9
                                / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None,
                       "bytes_per_particle": INTEGRATE_BYTES, "particles": main_r["mobile"],
                       "ms_per_launch": main_r["integrate_ms"],
                       "fp64_pipe_ncu": integ_cnt.get("fp64_pipe_pct", 100.0) / 100.0 if integ_cnt else None,
                       "note": "peak = measured copy bandwidth (MEASURED_PEAKS.json); algorithmic bytes: "
                               "read x, v, w, F, N, m, I and write x, v, w of each mobile particle"},
        "e2e": {"value": pairs * 2 / (main_r["e2e_ms"] / 1e3) * ws, "unit": UNIT,
                "h2d_bytes_per_step": main_r["e2e_bytes"], "d2h_bytes_per_step": main_r["e2e_bytes"],
                "ms_per_step": main_r["e2e_ms"], "ms_samples": main_r["e2e_per_step"]},
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")},
    }
    if other_r is not None and split:
        fp64_val = other_r["pairs"] * 2 / (other_r["ms_per_step"] / 1e3)
        rec["fp64_path"] = {
            "value": fp64_val, "unit": UNIT, "ms_per_step": other_r["ms_per_step"],
            "timesteps_per_s": 1e3 / other_r["ms_per_step"], "steps_timed": other_r["steps"],
            "speedup_of_value": (value / ws) / fp64_val,
            "note": "plain FP64 GPU path: double pair arithmetic, each of the %d instances in its own "
                    "context, stage calls without a graph, default tuning; per-step time summed over "
                    "the instances" % other_r["instances"]}
    elif other_r is not None:
        other_val = other_r["pairs"] * 2 * args.steps / (other_r["ms"] / 1e3)
        otf = FLOPS_PER_PAIR * other_r["pairs"] / (other_r["force_ms"] / 1e3) / 1e12
        rec["split_precision"] = {
            "value": other_val, "unit": UNIT, "ms_per_step": other_r["ms"] / args.steps,
            "force_ms_per_launch": other_r["force_ms"], "tuning": other_r["setting"],
            "speedup_vs_fp64": other_val / (value / ws),
            "roofline": {"bound": "alu", "achieved": otf, "peak": alu["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": otf / alu["fp32_tflops"]}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = cpu_baseline(args.workload, case=None)
    if rank == 0:
        print(json.dumps(rec))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
