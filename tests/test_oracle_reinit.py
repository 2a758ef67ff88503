"""Pins of the oracle's density reinitialisation (reading B5: the Shepard
form d~_i = (W(0) + sum_j W_ij) / (W(0)/d_i + sum_j W_ij/d_j), after
Colagrossi and Landrini, named in the text under Algorithm 1)."""
import numpy as np

import oracle
from paper_2002_03120_gb300 import cases


def test_reinit_leaves_a_perfect_lattice_unchanged():
    c = cases.poiseuille_si(nx=12, ny=12, nz=12, jitter=0.0)
    c["params"]["density_reinit"] = 1
    o = oracle.OracleSim(c)
    o.neighbors()
    o.density()
    d0 = o.state()["d"].copy()
    o.reinit()
    assert np.max(np.abs(o.state()["d"] / d0 - 1.0)) < 1e-13


def test_reinit_is_a_weighted_harmonic_mean_of_the_neighbourhood():
    # a free-surface block: the summation density varies near the surface;
    # the reinitialised value of each particle lies between the smallest and
    # the largest density of itself and its neighbours, and differs from the
    # summation density somewhere
    c = cases.dam_break(scale=0.1, n_spheres=0)
    c["params"]["density_reinit"] = 1
    o = oracle.OracleSim(c)
    o.neighbors()
    o.density()
    d0 = o.state()["d"].copy()
    ij = o.pairs()
    lo, hi = d0.copy(), d0.copy()
    for a, b in ((0, 1), (1, 0)):
        np.minimum.at(lo, ij[:, a], d0[ij[:, b]])
        np.maximum.at(hi, ij[:, a], d0[ij[:, b]])
    o.reinit()
    d1 = o.state()["d"]
    inner = c["type"] != 3
    assert np.all(d1[inner] >= lo[inner] * (1 - 1e-12))
    assert np.all(d1[inner] <= hi[inner] * (1 + 1e-12))
    assert np.all(d1[~inner] == d0[~inner])
    assert np.max(np.abs(d1 / d0 - 1.0)) > 1e-3
    # pressure follows the new density through the equation of state
    p = o.state()["p"]
    P = c["params"]
    rho = P["rho0"] * P["dx"] ** 3 * d1
    pe = P["p0"] * (rho / P["rho0"]) ** P["alpha"] - P["beta_p"]
    if P["clamp_negative_p"]:
        pe = np.maximum(pe, 0.0)
    assert np.allclose(p[inner], pe[inner], rtol=1e-12, atol=1e-9 * P["p0"])
