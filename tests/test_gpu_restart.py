"""Checkpoint and restart (the restart files of Section 3.1) through the C
ABI: a run continued from a checkpoint image in a fresh context is bit for
bit the run that wrote it (state, step counter keying the random stream,
tangential contact histories of the spheres)."""
import numpy as np
import pytest

from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


CASES = {
    "sediment_small": lambda: cases.sedimentation(nx=12, ny=12, nz=24),
    "slurry_small": lambda: cases.viscometer_instance(6000, 0.2, 300.0, 1e-2, seed=9, mesoscale=True),
    "dambreak_small": lambda: cases.dam_break(scale=0.15, n_spheres=40),
}


@pytest.mark.parametrize("precision", [B.SDPD_PREC_FP64, B.SDPD_PREC_SPLIT])
@pytest.mark.parametrize("name", list(CASES))
def test_restart_is_bit_identical(name, precision):
    case = CASES[name]()
    a = B.Sim(case, precision=precision)
    a.step(6)
    image = a.checkpoint()
    a.step(9)
    sa = a.state(density=False)
    b = B.Sim(case, precision=precision)
    b.restore(image)
    assert b.step_count == 6
    b.step(9)
    sb = b.state(density=False)
    for k in ("x", "v", "w", "F", "N"):
        assert np.array_equal(sa[k], sb[k]), k
    # an image of another context shape is refused
    other = B.Sim(cases.poiseuille_si(nx=12, ny=12, nz=12), precision=precision)
    with pytest.raises(B.SdpdError):
        other.restore(image)
