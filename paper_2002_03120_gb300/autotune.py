"""Autotuner of the per-workload launch choices of libsdpd.

For one workload (a list of instances and a precision) it times full steps
under each candidate setting -- force-pass variant (Newton-3 half pairs,
direct, or the pair stream through shared memory at two register caps),
Verlet skin, pair-kernel block size, lanes per particle of the direct pass,
full- or half-size cells of the neighbour search -- picks the fastest, and keeps
the choice in a JSON file keyed by GPU name, precision and size class (total
particles rounded to a power of two, number of instances), so later contexts
of the same class reuse it without measuring again.

The measurement uses CUDA events on one stream after warm-up steps, with one
forced list build in each measured window of `steps` steps (runs rebuild the
lists every few steps once the particles move, and the settings differ in its
cost); the choice never changes results beyond summation order (all settings
evaluate the same pairs exactly).
"""
from __future__ import annotations

import itertools
import json
import math
import os

from . import binding as B

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sdpd_gb300", "autotune.json")
# force-pass variants (sdpd_set_force_mode): 1 Newton 3, 0 direct, 5 direct
# with fewer registers (FP32 only).  Not sampled by default, because they
# measured slower on every workload here: 2 and 3 (the pair stream: its
# shared-memory compaction buys nothing where lanes are already busy, and
# costs L1 and instructions) and 4 (Newton 3 with pushed results: the
# scattered stores cost more than the coalesced gather saves)
CANDIDATES = {
    "newton3": (1, 0, 5),
    "skin": (0.0, 0.03, 0.06, 0.12),
    "block": (64, 128, 256),
    "tpp": (1, 2, 4),   # lanes per particle of the direct pass
    "cells": (1, 2),    # cells per minimum cell width of the neighbour search
}


def size_class(n_particles: int, n_instances: int, precision: int) -> str:
    return f"p{precision}_n2^{int(round(math.log2(max(n_particles, 1))))}_i{n_instances}"


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _sampled(setting, candidates, precision):
    """Settings measured, with full-size cells: the Newton-3 passes over the
    whole grid (the push variant for FP32 pairs only); the direct pass at the
    default block (every skin) and without skin (every block), its lean form
    (FP32 only, 128 threads) at the three smaller skins; the pair stream,
    when asked for, at the two larger blocks and the two middle skins, the
    three-block variant for FP32 pairs only.  Half-size cells: the Newton-3,
    direct and lean direct passes at the default block and the three smaller
    skins, and the direct pass with several lanes per particle at the default
    block and skin."""
    mode, skin, block = setting["newton3"], setting["skin"], setting["block"]
    skins = candidates["skin"]
    if setting.get("cells", 1) != 1:
        # half-size cells: the default block, the three smaller skins; Newton
        # 3, direct and lean direct (FP32) with one lane per particle, and
        # the direct pass with several lanes at the default skin
        if block != 128 or skin not in skins[:3]:
            return False
        if setting.get("tpp", 1) != 1:
            return mode == 0 and skin == skins[min(1, len(skins) - 1)]
        return mode in (0, 1) or (mode == 5 and precision != B.SDPD_PREC_FP64)
    if setting.get("tpp", 1) != 1:
        # several lanes per particle: the direct pass at the default block
        # and the default skin
        return mode == 0 and block == 128 and skin == skins[min(1, len(skins) - 1)]
    if mode in (4, 5) and precision == B.SDPD_PREC_FP64:
        return False
    if mode == 5:
        return block == 128 and skin in skins[:3]
    if mode == 0:
        return skin == skins[0] or block == 128
    if mode in (2, 3):
        if mode == 3 and precision == B.SDPD_PREC_FP64:
            return False
        return block in (128, 256) and skin in skins[1:3]
    return True


def search(measure, candidates=CANDIDATES, precision=None):
    """Search over the sampled candidate grid; `measure(setting)` returns a
    time in ms (or None when the setting is not usable).  Returns
    (best_setting, table of all results)."""
    keys = sorted(candidates)
    table = []
    best, best_t = None, float("inf")
    for values in itertools.product(*(candidates[k] for k in keys)):
        setting = dict(zip(keys, values))
        if not _sampled(setting, candidates, precision):
            continue
        t = measure(setting)
        table.append({**setting, "ms": t})
        if t is not None and t < best_t:
            best, best_t = setting, t
    return best, table


def apply(sim: "B.Sim", setting: dict) -> None:
    sim.set_force_mode(int(setting["newton3"]))
    sim.set_threads_per_particle(int(setting.get("tpp", 1)))
    sim.set_skin(float(setting["skin"]))
    sim.set_cell_factor(int(setting.get("cells", 1)))
    sim.set_block_size(int(setting["block"]))


def tune(cases, precision=B.SDPD_PREC_SPLIT, steps=10, warmup=3, cache_path=DEFAULT_CACHE,
         force=False, max_neighbors=0, candidates=CANDIDATES):
    """Measure (or read from the cache) the fastest setting for this workload."""
    import torch
    if isinstance(cases, dict):
        cases = [cases]
    n = sum(len(c["x"]) for c in cases)
    key = f"{_gpu_name()}|{size_class(n, len(cases), precision)}"
    cache = load_cache(cache_path)
    if not force and key in cache:
        return cache[key]["best"]
    stream = torch.cuda.Stream()
    # one context for every setting: the starting state is restored from a
    # checkpoint image before each measurement (no re-upload of the particles)
    sim = B.Sim(cases, precision=precision, max_neighbors=max_neighbors)
    image = sim.checkpoint()

    def measure(setting):
        try:
            apply(sim, setting)
            sim.restore(image)
            sim.step(warmup, stream)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            # one list build per measured window: a run rebuilds every few
            # steps once the particles move, and the settings differ in its cost
            sim.build_cells(stream)
            sim.step(steps, stream)
            b.record(stream)
            b.synchronize()
            return a.elapsed_time(b) / steps
        except B.SdpdError:
            return None

    try:
        best, table = search(measure, candidates, precision)
    finally:
        sim.close()
    cache[key] = {"best": best, "table": table, "particles": n, "instances": len(cases)}
    save_cache(cache, cache_path)
    return best
