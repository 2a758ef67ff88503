"""The read-out entry points against the oracle's plain counterparts on the
same seeded inputs: sdpd_diagnostics (momentum, kinetic energy and
temperature, density range, non-finite count) and sdpd_viscosity_fit (the
least-squares parabola of Section 4.1, reading B6) with sdpd_viscosity_probe
(Eq. poiseuave).  Both sides read the same state; only summation order
differs (the GPU sums with atomics)."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B
from paper_2002_03120_gb300 import cases

from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _close(a, b, rel, scale=None):
    a, b = np.asarray(a, float), np.asarray(b, float)
    s = np.abs(b) if scale is None else scale
    return np.all(np.abs(a - b) <= rel * np.maximum(s, 1e-300))


@pytest.mark.parametrize("precision", [B.SDPD_PREC_FP64, B.SDPD_PREC_SPLIT])
def test_diagnostics_match_oracle(precision):
    insts = [cases.viscometer_instance(6000, 0.2, 300.0, 1e-2, seed=9, mesoscale=True),
             cases.sedimentation(nx=12, ny=12, nz=24)]
    rng = np.random.default_rng(21)
    for c in insts:
        mob = (c["type"] <= 1)[:, None]
        c["v"] = np.where(mob, rng.normal(0.01, 0.05, c["v"].shape) * c["params"]["dx"], 0.0)
    sim = B.Sim(insts, precision=precision)
    sim.build_cells()
    sim.compute_density()
    for k, c in enumerate(insts):
        g = sim.diagnostics(k)
        orc = oracle.OracleSim(c, inst=k)
        orc.neighbors()
        orc.density()
        o = orc.diagnostics()
        mom = np.linalg.norm(o[0:3]) + np.sqrt(2 * o[3] * c["mass"][c["type"] <= 1].sum())
        assert _close(g[0:3], o[0:3], 1e-12, scale=mom)
        assert _close(g[3:6], o[3:6], 1e-12)
        # densities: FP64 pair sums agree to 1e-12; the split path's FP32
        # kernel values to the density tolerance of the parity tests
        assert _close(g[6:8], o[6:8], 1e-12 if precision == B.SDPD_PREC_FP64 else 1e-6)
        assert g[8] == o[8] == 0
    sim.close()


def test_viscosity_fit_and_probe_match_oracle():
    c = cases.poiseuille_meso(nx=12, ny=48, nz=12)   # periodic axes >= 3 h
    p = c["params"]
    mu, a, rho = p["eta"], p["body_amp"], p["rho0"]
    D = 0.5 * p["box"][1]
    y = c["x"][:, 1]
    z = np.where(y < D, y, y - D)
    prof = rho * a / (2 * mu) * (z * D - z * z) + 0.2
    rng = np.random.default_rng(3)
    c["v"][:, 0] = np.where(y < D, prof, -prof) + rng.normal(0, 0.02, len(y))
    c["v"][:, 1:] = rng.normal(0, 0.02, (len(y), 2))
    sim = B.Sim(c, precision=B.SDPD_PREC_FP64)
    orc = oracle.OracleSim(c)
    for nb in (16, 24):
        prof_g, mu_g = sim.viscosity_probe(0, nb)
        prof_o, mu_o = orc.profile(nb)
        assert np.allclose(prof_g, prof_o, rtol=1e-12, atol=1e-12 * np.abs(prof_o).max())
        assert mu_g == pytest.approx(mu_o, rel=1e-12)
        # the GPU's fit solves the normal equations (Cramer's rule), the
        # oracle's numpy's least squares: their rounding differs by the
        # squared conditioning of [1 t t^2] over the slabs (~1e4)
        fit_g = sim.viscosity_fit(0, nb)
        fit_o = orc.viscosity_fit(nb)
        assert fit_g == pytest.approx(fit_o, rel=1e-10)
        assert fit_o == pytest.approx(mu, rel=0.05)
    sim.close()
