"""The oracle's per-particle loops may run on several threads (OpenMP, for
the all-cores CPU baseline); every particle owns its list and its sums, so the
state after full steps is bit for bit the same at any thread count."""
import numpy as np

import oracle
from paper_2002_03120_gb300 import cases


def test_results_do_not_depend_on_thread_count():
    c = cases.dam_break(scale=0.12, n_spheres=30)
    rng = np.random.default_rng(2)
    mob = (c["type"] <= 1)[:, None]
    c["v"] = np.where(mob, rng.normal(0, 0.01, c["v"].shape), 0.0)
    prev = oracle.threads()
    out = {}
    try:
        for nt in (1, 3):
            oracle.threads(nt)
            s = oracle.OracleSim(c)
            s.step = 2
            s.run(2)
            out[nt] = (s.state(), s.history(), s.pairs())
    finally:
        oracle.threads(prev)
    a, b = out[1], out[3]
    for k in ("x", "v", "w", "F", "N", "d", "p"):
        assert np.array_equal(a[0][k], b[0][k]), k
    for u, v in zip(a[1], b[1]):
        assert np.array_equal(u, v)
    assert np.array_equal(a[2], b[2])
