"""sdpd_density_noalloc: the allocation-free density entry point.

It serves callers that cannot let a library allocate device memory (an
application whose allocator owns the whole GPU, code that cannot take the
synchronisation of cudaMalloc/cudaFree).  Its scratch is a fixed file-scope
device array; here its output is checked against the context-based entry
points (sdpd_build_cells + sdpd_compute_density, FP64) on two calls in a row,
with the tolerances of the density parity tests."""
import numpy as np
import pytest

from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def _noalloc(case):
    import torch
    x = torch.tensor(case["x"], dtype=torch.float64, device="cuda")
    t = torch.tensor(case["type"], dtype=torch.int32, device="cuda")
    d = torch.full((x.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    p = torch.full_like(d, float("nan"))
    B.density_noalloc(case["params"], x, t, d, p)
    torch.cuda.synchronize()
    return d.cpu().numpy(), p.cpu().numpy()


def _context(case):
    sim = B.Sim(case, precision=B.SDPD_PREC_FP64)
    sim.build_cells()
    sim.compute_density()
    st = sim.state()
    sim.close()
    return st["d"], st["p"]


def test_noalloc_matches_context_on_two_calls_in_a_row():
    need_gpu()
    runs = [cases.sedimentation(nx=16, ny=16, nz=32), cases.poiseuille_si()]
    got = [_noalloc(c) for c in runs]          # two calls back to back
    for case, (d, p) in zip(runs, got):
        d_ref, p_ref = _context(case)
        assert rel_l2(d, d_ref) < 1e-12
        assert np.max(np.abs(p - p_ref)) < 1e-9 * case["params"]["p0"]


def test_noalloc_rejects_oversize_input():
    need_gpu()
    import torch
    n = B.NOALLOC_MAX_PARTICLES + 1
    case = cases.poiseuille_si()
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SdpdError) as e:
        B.density_noalloc(case["params"], x, t, d, d)
    assert e.value.code == 1 and "static scratch limit" in str(e.value)


def _bad_box_params(case, axis, value):
    prm = dict(case["params"])
    box = list(prm["box"])
    box[axis] = value
    prm["box"] = box
    return prm


@pytest.mark.parametrize("value", [-1.0, 0.0, float("nan"), float("inf"), 1e300])
def test_noalloc_rejects_bad_box_before_launch(value):
    # a wall axis (z of the sedimentation box) and a periodic axis (x) with a
    # box that is not a finite positive length, or one with far too many cells
    need_gpu()
    import torch
    case = cases.sedimentation(nx=8, ny=8, nz=16)
    n = len(case["x"])
    x = torch.tensor(case["x"], dtype=torch.float64, device="cuda")
    t = torch.tensor(case["type"], dtype=torch.int32, device="cuda")
    d = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    p = torch.full_like(d, 7.0)
    for axis in (2, 0):
        with pytest.raises(B.SdpdError) as e:
            B.density_noalloc(_bad_box_params(case, axis, value), x, t, d, p)
        assert e.value.code == 1
    torch.cuda.synchronize()
    assert bool(torch.all(d == 7.0)) and bool(torch.all(p == 7.0))   # nothing was launched


def test_noalloc_folds_periodic_positions_and_isolates_nonfinite():
    # positions shifted by whole boxes along the periodic axes give the same
    # density; a particle with a NaN position gets NaN and leaves the others
    # as they are without it
    need_gpu()
    case = cases.poiseuille_si()
    d0, p0 = _noalloc(case)
    box = np.asarray(case["params"]["box"])
    moved = dict(case)
    xs = case["x"].copy()
    xs[::3, 0] += box[0]
    xs[1::3, 1] -= 2.0 * box[1]
    xs[2::5, 2] += 3.0 * box[2]
    moved["x"] = xs
    d1, p1 = _noalloc(moved)
    assert rel_l2(d1, d0) < 1e-12
    assert np.max(np.abs(p1 - p0)) < 1e-9 * case["params"]["p0"]
    k = 100
    gone = dict(case)
    xg = case["x"].copy()
    xg[k] = np.nan
    gone["x"] = xg
    d2, p2 = _noalloc(gone)
    assert np.isnan(d2[k]) and np.isnan(p2[k])
    keep = np.arange(len(xg)) != k
    without = dict(case)
    for key in ("x", "v", "w", "type", "radius", "mass"):
        without[key] = case[key][keep]
    d3, p3 = _noalloc(without)
    assert rel_l2(d2[keep], d3) < 1e-12
