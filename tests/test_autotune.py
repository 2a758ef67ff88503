"""Autotuner: search logic and cache on the CPU (fake timings), and one real
tuning run through the C ABI on the GPU."""
import json

import pytest

from paper_2002_03120_gb300 import autotune


def test_search_picks_fastest_and_skips_nothing_required():
    times = {}

    mode_cost = {1: 7.0, 4: 7.5, 0: 10.0, 2: 8.0, 3: 8.5, 5: 9.0}

    def fake(setting):
        t = mode_cost[setting["newton3"]] - 10 * setting["skin"] + abs(setting["block"] - 128) / 64 \
            + 0.1 * setting.get("tpp", 1) + 0.05 * setting.get("cells", 1)
        times[tuple(sorted(setting.items()))] = t
        return t

    best, table = autotune.search(fake)
    assert best == {"newton3": 1, "skin": 0.12, "block": 128, "tpp": 1, "cells": 1}
    # several lanes per particle only for the direct pass, default block and skin
    assert {(r["newton3"], r["block"], r["skin"]) for r in table if r["tpp"] != 1} == {(0, 128, 0.03)}
    # half-size cells: default block, the smaller skins; several lanes per
    # particle only for the direct pass at the default skin
    half = [r for r in table if r["cells"] == 2]
    assert {r["block"] for r in half} == {128}
    assert {r["skin"] for r in half} == {0.0, 0.03, 0.06}
    assert {r["newton3"] for r in half} == {0, 1, 5}
    assert {(r["newton3"], r["skin"]) for r in half if r["tpp"] != 1} == {(0, 0.03)}
    assert min(r["ms"] for r in table) == pytest.approx(fake(best))
    assert {r["newton3"] for r in table} == {0, 1, 5}
    # asked for, the pair stream is sampled at the two larger blocks and
    # middle skins
    cand = dict(autotune.CANDIDATES, newton3=(1, 4, 0, 2, 3, 5))
    _, t32 = autotune.search(fake, cand, precision=1)
    assert {(r["block"], r["skin"]) for r in t32 if r["newton3"] == 2} == \
        {(128, 0.03), (256, 0.03), (128, 0.06), (256, 0.06)}
    # the push variant, the three-block stream and the lean direct pass are
    # FP32-only
    _, t64 = autotune.search(fake, cand, precision=0)
    assert not any(r["newton3"] in (3, 4, 5) for r in t64)


def test_search_ignores_unusable_settings():
    best, table = autotune.search(lambda s: None if s["block"] == 64 else 1.0 + s["skin"] + s["tpp"])
    assert best["block"] != 64 and best["skin"] == 0.0 and best["cells"] == 1


def test_cache_roundtrip(tmp_path):
    p = tmp_path / "t.json"
    autotune.save_cache({"k": {"best": {"newton3": 1}}}, str(p))
    assert autotune.load_cache(str(p))["k"]["best"]["newton3"] == 1
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
    assert autotune.size_class(73728, 1, 0) == "p0_n2^16_i1"


@pytest.mark.gpu
def test_tune_on_gpu(tmp_path):
    from _gpu_common import need_gpu
    need_gpu()
    from paper_2002_03120_gb300 import binding as B
    from paper_2002_03120_gb300 import cases
    case = cases.sedimentation(nx=16, ny=16, nz=32)
    cache = str(tmp_path / "tune.json")
    cand = {"newton3": (1, 0, 2), "skin": (0.0, 0.03, 0.06), "block": (128, 256), "tpp": (1, 2),
            "cells": (1, 2)}
    best = autotune.tune(case, precision=B.SDPD_PREC_SPLIT, steps=3, warmup=2, cache_path=cache,
                         candidates=cand)
    assert best["block"] in (128, 256) and best["newton3"] in (0, 1, 2)
    data = json.load(open(cache))
    (entry,) = data.values()
    assert all(r["ms"] is not None and r["ms"] > 0 for r in entry["table"])
    # a second call is served from the cache
    assert autotune.tune(case, precision=B.SDPD_PREC_SPLIT, cache_path=cache, candidates=cand) == best
