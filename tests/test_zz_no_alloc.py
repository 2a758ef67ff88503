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
