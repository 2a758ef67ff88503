"""Seeded synthetic workloads for the SDPD-DEM viscometer step.

This module only places particles and fills parameter dictionaries.  It holds
none of the method's arithmetic (no kernel, density, force or integrator), so
both the CUDA path and the CPU oracle can be fed from it.

Every case is a dict with
  params : physical and numerical parameters (Table 1 of the paper plus the
           readings' constants); all lengths in metres unless stated,
  x, v, w: float64 [n, 3] positions, velocities, spin angular velocities,
  type   : int32 [n]  0 fluid, 1 rigid, 2 inner wall, 3 outer wall,
  radius : float64 [n] (rigid radius; dx/2 otherwise),
  mass   : float64 [n].
Particle index = global id (gid) used by the counter-based noise.

Workloads (shapes, sizes and distributions of the paper's Section 4 cases):
  poiseuille_si        reverse-Poiseuille flow, SDPD only, fully periodic
                       (16x32x16 lattice, dx = 1 mm, water)
  sedimentation        single sphere settling between dummy-particle walls
                       (32x32x64 lattice, d = 4 dx, rho_s = 2500)
  dam_break            water column with polydisperse spheres in a walled tank
  viscometer_instance  one reverse-Poiseuille slurry instance of the batched
                       sweep (log-uniform size, solid fraction, temperature,
                       forcing)
  poiseuille_meso      the reverse-Poiseuille case in the paper's mesoscale
                       units (rho0 = 3, eta = 25, xi = 20 eta / 21,
                       p0 = beta = 100), for viscosity read-outs
"""
from __future__ import annotations

import math

import numpy as np

T_FLUID, T_RIGID, T_INNER_WALL, T_OUTER_WALL = 0, 1, 2, 3
K_BOLTZMANN = 1.380649e-23


def base_params(**over) -> dict:
    """Default parameter set (SI water at 293 K, dx = 1 mm)."""
    dx = over.get("dx", 1e-3)
    rho0 = over.get("rho0", 1000.0)
    c = over.get("c_sound", 10.0)
    alpha = over.get("alpha", 7.0)
    eta = over.get("eta", 1e-3)
    p0 = rho0 * c * c / alpha
    p = dict(
        dx=dx, r_c=3.9 * dx, dt=1e-5,
        rho0=rho0, p0=p0, alpha=alpha, beta_p=p0,
        eta=eta, xi=20.0 * eta / 21.0, kBT=4.1e-21,
        coeff_c=1.0, coeff_d=1.0, coeff_r=1.0, coeff_t=1.0,
        origin=[0.0, 0.0, 0.0], box=[1.0, 1.0, 1.0], g=[0.0, 0.0, 0.0],
        body_amp=0.0, artvis_alpha=0.5, artvis_e=0.2,
        kn=1e3, restitution=0.9, nu_p=0.25, E_p=7e10, mu_fric=0.0,
        lub_gap_min=0.01, eps_min=0.05,
        periodic=[1, 1, 1], body_axis=0, split_axis=1,
        pressure_filter=0, clamp_negative_p=0, artvis=0, dem_law=1,
        seed=1,
    )
    for k, v in over.items():
        if k in ("c_sound",):
            continue
        p[k] = v
    if "xi" not in over:
        p["xi"] = 20.0 * p["eta"] / 21.0
    if "p0" not in over and ("c_sound" in over or "rho0" in over or "alpha" in over):
        p["p0"] = p["rho0"] * c * c / p["alpha"]
        p["beta_p"] = p["p0"]
    if "r_c" not in over:
        p["r_c"] = 3.9 * p["dx"]
    return p


def lattice(nx: int, ny: int, nz: int, dx: float, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Cubic lattice sites origin + (i + 1/2) dx, x fastest."""
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    pts = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64)
    return (pts + 0.5) * dx + np.asarray(origin, dtype=np.float64)


def _jitter(x: np.ndarray, amp: float, rng: np.random.Generator) -> np.ndarray:
    return x + rng.uniform(-amp, amp, size=x.shape)


def _assemble(params, parts, name):
    x = np.concatenate([p[0] for p in parts], axis=0)
    t = np.concatenate([np.full(len(p[0]), p[1], dtype=np.int32) for p in parts])
    R = np.concatenate([p[2] for p in parts])
    m = np.concatenate([p[3] for p in parts])
    n = len(x)
    return dict(name=name, params=params, x=np.ascontiguousarray(x), v=np.zeros((n, 3)),
                w=np.zeros((n, 3)), type=t, radius=R, mass=m)


def _wall_layers(nxyz, dx, origin, layers, axes_sides, top_open=False):
    """Dummy-particle layers outside the fluid box on the given (axis, side)
    faces; layer 0 is the inner wall, the rest outer wall.  Columns of the
    walls on one axis extend over the walls of the other wall axes so corners
    are filled."""
    nx, ny, nz = nxyz
    n = [nx, ny, nz]
    wall_axes = sorted({a for a, _ in axes_sides})
    lo = [0] * 3
    hi = list(n)
    for a in wall_axes:
        sides = {s for b, s in axes_sides if b == a}
        if 0 in sides:
            lo[a] = -layers
        if 1 in sides:
            hi[a] = n[a] + layers
    ii = [np.arange(lo[a], hi[a]) for a in range(3)]
    K, J, I = np.meshgrid(ii[2], ii[1], ii[0], indexing="ij")
    idx = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    # distance (in layers) outside the fluid box, per axis
    out = np.zeros(len(idx), dtype=np.int64)
    for a in range(3):
        below = np.where(idx[:, a] < 0, -idx[:, a], 0)
        above = np.where(idx[:, a] >= n[a], idx[:, a] - n[a] + 1, 0)
        out = np.maximum(out, np.maximum(below, above))
    keep = out > 0
    idx = idx[keep]
    out = out[keep]
    x = (idx.astype(np.float64) + 0.5) * dx + np.asarray(origin)
    t = np.where(out == 1, T_INNER_WALL, T_OUTER_WALL).astype(np.int32)
    return x, t


def poiseuille_si(nx=16, ny=32, nz=16, dx=1e-3, g_amp=1e-2, seed=1, jitter=0.01,
                  dt=1e-5, **over) -> dict:
    """Reverse-Poiseuille flow, SDPD only, fully periodic (Section 4.1 in SI
    water units): forcing +-g_amp along x in the two y-halves."""
    params = base_params(dx=dx, dt=dt, **over)
    params.update(box=[nx * dx, ny * dx, nz * dx], periodic=[1, 1, 1], body_amp=g_amp,
                  body_axis=0, split_axis=1, seed=seed)
    rng = np.random.default_rng(seed)
    x = _jitter(lattice(nx, ny, nz, dx), jitter * dx, rng)
    n = len(x)
    mf = params["rho0"] * dx ** 3
    return _assemble(params, [(x, T_FLUID, np.full(n, 0.5 * dx), np.full(n, mf))],
                     f"poiseuille_si_{nx}x{ny}x{nz}")


def poiseuille_meso(nx=12, ny=24, nz=12, rho0=3.0, eta=25.0, amp=1.5, kBT=1.0, alpha=7.0,
                    p0=100.0, dt=None, seed=1, jitter=0.01, **over) -> dict:
    """Reverse Poiseuille in the paper's mesoscale units (Section 4.1: unit
    mass, length and energy; rho0 = 3, eta = 25, xi = 20 eta/21,
    p0 = beta = 100, forcing 1.5 per unit mass); particle mass 1 so
    dx = rho0^(-1/3)."""
    dx = rho0 ** (-1.0 / 3.0)
    r_c = 3.9 * dx
    if dt is None:
        c = math.sqrt(alpha * p0 / rho0)
        nu = eta / rho0
        dt = min(0.1 * r_c / c, 0.05 * dx * dx / nu)
    params = base_params(dx=dx, rho0=rho0, eta=eta, alpha=alpha, dt=dt, **over)
    params.update(p0=p0, beta_p=p0, kBT=kBT, r_c=r_c, box=[nx * dx, ny * dx, nz * dx],
                  periodic=[1, 1, 1], body_amp=amp, body_axis=0, split_axis=1, seed=seed)
    for k, v in over.items():
        params[k] = v
    rng = np.random.default_rng(seed)
    x = _jitter(lattice(nx, ny, nz, dx), jitter * dx, rng)
    n = len(x)
    return _assemble(params, [(x, T_FLUID, np.full(n, 0.5 * dx), np.full(n, 1.0))],
                     f"poiseuille_meso_{nx}x{ny}x{nz}")


def poiseuille_meso_walls(nx=12, ny=24, nz=12, layers=4, **kw) -> dict:
    """Reverse Poiseuille with the wall-periodic hybrid boundaries of Section
    4.1: the mesoscale case of poiseuille_meso, but with dummy-particle walls
    (`layers` layers, the first inner) on both faces of the split axis (y) and
    periodic boundaries in x and z.  Each half is then a Poiseuille flow
    between a wall and the mid-plane, read by the same Eq. poiseuave."""
    case = poiseuille_meso(nx=nx, ny=ny, nz=nz, **kw)
    p = case["params"]
    p["periodic"] = [1, 0, 1]
    dx = p["dx"]
    wx, wt = _wall_layers((nx, ny, nz), dx, (0, 0, 0), layers, [(1, 0), (1, 1)])
    nw = len(wx)
    m = float(case["mass"][0])
    case["x"] = np.concatenate([case["x"], wx])
    case["type"] = np.concatenate([case["type"], wt])
    case["radius"] = np.concatenate([case["radius"], np.full(nw, 0.5 * dx)])
    case["mass"] = np.concatenate([case["mass"], np.full(nw, m)])
    case["v"] = np.zeros_like(case["x"])
    case["w"] = np.zeros_like(case["x"])
    case["name"] = f"poiseuille_meso_walls_{nx}x{ny}x{nz}"
    return case


def buoyancy_column(nx=14, ny=14, nz=24, layers=4, g=0.5, rho_ratio=1.0, diam_dx=4.0, eta=25.0,
                    kBT=1e-4, seed=1, **over) -> dict:
    """A fluid column in the paper's mesoscale units (rho0 = 3, p0 = beta = 100,
    alpha = 7, unit mass), periodic in x and y, with dummy-particle walls below
    and above in z, gravity -g along z, and one sphere of diameter diam_dx dx
    and density rho_ratio rho0 at mid-height replacing the nearest lattice
    site (the buoyancy check of the pressure-gradient force, Eq. F_fpi_PG)."""
    rho0 = 3.0
    dx = rho0 ** (-1.0 / 3.0)
    params = base_params(dx=dx, rho0=rho0, eta=eta, alpha=7.0, **over)
    params.update(p0=100.0, beta_p=100.0, kBT=kBT, r_c=3.9 * dx, box=[nx * dx, ny * dx, nz * dx],
                  periodic=[1, 1, 0], g=[0.0, 0.0, -g], seed=seed, dem_law=1, kn=1e3, restitution=0.9)
    c = math.sqrt(params["alpha"] * params["p0"] / rho0)
    params["dt"] = min(0.1 * params["r_c"] / c, 0.3 / eta)
    for k, v in over.items():
        params[k] = v
    rng = np.random.default_rng(seed)
    sites = lattice(nx, ny, nz, dx)
    target = np.array([0.5 * nx * dx, 0.5 * ny * dx, 0.5 * nz * dx])
    s = int(np.argmin(np.sum((sites - target) ** 2, axis=1)))
    centre = sites[s].copy()
    fluid = _jitter(np.delete(sites, s, axis=0), 0.01 * dx, rng)
    wx, wt = _wall_layers((nx, ny, nz), dx, (0, 0, 0), layers, [(2, 0), (2, 1)])
    R = 0.5 * diam_dx * dx
    ms = rho_ratio * rho0 * 4.0 / 3.0 * math.pi * R ** 3
    nf = len(fluid)
    parts = [
        (fluid, T_FLUID, np.full(nf, 0.5 * dx), np.full(nf, 1.0)),
        (centre[None, :], T_RIGID, np.array([R]), np.array([ms])),
    ]
    case = _assemble(params, parts, f"buoyancy_column_{nx}x{ny}x{nz}")
    nw = len(wx)
    case["x"] = np.concatenate([case["x"], wx])
    case["type"] = np.concatenate([case["type"], wt])
    case["radius"] = np.concatenate([case["radius"], np.full(nw, 0.5 * dx)])
    case["mass"] = np.concatenate([case["mass"], np.full(nw, 1.0)])
    case["v"] = np.zeros_like(case["x"])
    case["w"] = np.zeros_like(case["x"])
    return case


def _place_spheres_on_sites(nxyz, n_target: int, diam_dx: np.ndarray, periodic,
                            rng: np.random.Generator):
    """Random sequential addition on the sites of an nx x ny x nz lattice
    (index (k*ny + j)*nx + i, spacing 1): visit sites in random order and
    accept a sphere when no accepted sphere is closer than the sum of the two
    radii (checked conservatively against the largest diameter).  Returns the
    accepted site indices and their diameters in lattice units."""
    nx, ny, nz = nxyz
    blocked = np.zeros((nz, ny, nx), dtype=bool)
    dmax = float(np.max(diam_dx)) if len(diam_dx) else 1.0
    acc = []
    acc_d = []
    order = rng.permutation(nx * ny * nz)
    for s in order:
        if len(acc) >= n_target:
            break
        i = s % nx
        j = (s // nx) % ny
        k = s // (nx * ny)
        if blocked[k, j, i]:
            continue
        d = float(diam_dx[len(acc) % len(diam_dx)])
        lim = 0.5 * (d + dmax)
        rr = int(math.ceil(lim))
        off = np.arange(-rr, rr + 1)
        OZ, OY, OX = np.meshgrid(off, off, off, indexing="ij")
        near = (OX * OX + OY * OY + OZ * OZ) < lim * lim
        ii, jj, kk = i + OX[near], j + OY[near], k + OZ[near]
        ok = np.ones(ii.shape, dtype=bool)
        for arr, nn, per in ((ii, nx, periodic[0]), (jj, ny, periodic[1]), (kk, nz, periodic[2])):
            if per:
                arr %= nn
            else:
                ok &= (arr >= 0) & (arr < nn)
        blocked[kk[ok], jj[ok], ii[ok]] = True
        acc.append(int(s))
        acc_d.append(d)
    return np.asarray(acc, dtype=np.int64), np.asarray(acc_d)


def sedimentation(nx=32, ny=32, nz=64, dx=1e-3, layers=4, diam_dx=4.0, rho_s=2500.0,
                  height=0.75, dt=1e-5, seed=1, jitter=0.01, **over) -> dict:
    """Single-particle sedimentation (Section 4.2): fluid lattice periodic in
    x, y with dummy-particle walls in z, one sphere released from rest at
    `height` of the box, replacing the nearest lattice site (Section 3.1,
    --enable_load_rp)."""
    params = base_params(dx=dx, dt=dt, **over)
    params.update(box=[nx * dx, ny * dx, nz * dx], periodic=[1, 1, 0], g=[0.0, 0.0, -9.81],
                  artvis=1, dem_law=1, kn=1e3, restitution=0.9, seed=seed)
    for k, v in over.items():
        params[k] = v
    rng = np.random.default_rng(seed)
    sites = lattice(nx, ny, nz, dx)
    target = np.array([0.5 * nx * dx, 0.5 * ny * dx, height * nz * dx])
    s = int(np.argmin(np.sum((sites - target) ** 2, axis=1)))
    fluid = np.delete(sites, s, axis=0)
    fluid = _jitter(fluid, jitter * dx, rng)
    wx, wt = _wall_layers((nx, ny, nz), dx, (0, 0, 0), layers, [(2, 0), (2, 1)])
    mf = params["rho0"] * dx ** 3
    R = 0.5 * diam_dx * dx
    ms = rho_s * 4.0 / 3.0 * math.pi * R ** 3
    nf = len(fluid)
    parts = [
        (fluid, T_FLUID, np.full(nf, 0.5 * dx), np.full(nf, mf)),
        (target[None, :], T_RIGID, np.array([R]), np.array([ms])),
    ]
    case = _assemble(params, parts, f"sedimentation_{nx}x{ny}x{nz}")
    # walls carry their own types (inner/outer)
    case["x"] = np.concatenate([case["x"], wx])
    case["type"] = np.concatenate([case["type"], wt])
    nw = len(wx)
    case["radius"] = np.concatenate([case["radius"], np.full(nw, 0.5 * dx)])
    case["mass"] = np.concatenate([case["mass"], np.full(nw, mf)])
    case["v"] = np.zeros_like(case["x"])
    case["w"] = np.zeros_like(case["x"])
    return case


def dam_break(scale=1.0, n_spheres=10000, layers=3, dt=2e-5, seed=1, jitter=0.01, d_lo=3e-3,
              d_hi=5e-3, rho_s=2600.0, precision_note="split", **over) -> dict:
    """Dam break with rigid particles (Section 4.4): a 0.4 x 0.2 x 0.2 m water
    column (126 x 63 x 63 lattice at scale 1) at x in [0, 0.4] of a
    1.0 x 0.2 x 0.6 m tank with `layers` dummy-particle layers on the bottom
    and the four sides (open top), plus polydisperse spheres randomly placed
    in the column on lattice sites.  `scale` < 1 shrinks the lattice (same
    tank aspect) for small test cases."""
    ny = max(4, int(round(63 * scale)))
    dx = 0.2 / ny
    dscale = dx / (0.2 / 63)            # sphere sizes keep their ratio to dx
    nxc, nyc, nzc = 2 * ny, ny, ny
    nxt, nzt = 5 * ny, 3 * ny
    c = 20.0
    params = base_params(dx=dx, dt=dt, c_sound=c, **over)
    params.update(box=[nxt * dx, nyc * dx, nzt * dx], periodic=[0, 0, 0], g=[0.0, 0.0, -9.81],
                  artvis=1, pressure_filter=1, clamp_negative_p=1, dem_law=1, kn=1e3,
                  restitution=0.9, mu_fric=0.3, seed=seed)
    for k, v in over.items():
        params[k] = v
    rng = np.random.default_rng(seed)
    sites = lattice(nxc, nyc, nzc, dx)
    diam = rng.uniform(d_lo * dscale, d_hi * dscale, size=max(n_spheres, 1))
    acc, acc_d = _place_spheres_on_sites((nxc, nyc, nzc), n_spheres, diam / dx, [0, 0, 0], rng)
    acc_d = acc_d * dx
    mask = np.ones(len(sites), dtype=bool)
    mask[acc] = False
    fluid = _jitter(sites[mask], jitter * dx, rng)
    spheres = sites[acc]
    mf = params["rho0"] * dx ** 3
    Rs = 0.5 * acc_d
    ms = rho_s * 4.0 / 3.0 * math.pi * Rs ** 3
    wx, wt = _wall_layers((nxt, nyc, nzt), dx, (0, 0, 0), layers,
                          [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0)])
    nf = len(fluid)
    case = _assemble(params, [(fluid, T_FLUID, np.full(nf, 0.5 * dx), np.full(nf, mf)),
                              (spheres, T_RIGID, Rs, ms)], f"dam_break_s{scale}")
    nw = len(wx)
    case["x"] = np.concatenate([case["x"], wx])
    case["type"] = np.concatenate([case["type"], wt])
    case["radius"] = np.concatenate([case["radius"], np.full(nw, 0.5 * dx)])
    case["mass"] = np.concatenate([case["mass"], np.full(nw, mf)])
    case["v"] = np.zeros_like(case["x"])
    case["w"] = np.zeros_like(case["x"])
    return case


def arrhenius_viscosity(T: float, mu_ref=1e-3, T_ref=293.15, Ea_over_R=1900.0) -> float:
    """Water-like viscosity mu(T) = mu_ref exp[Ea/R (1/T - 1/T_ref)]."""
    return mu_ref * math.exp(Ea_over_R * (1.0 / T - 1.0 / T_ref))


def viscometer_instance(n_fluid_target: int, phi: float, T: float, g_amp: float, seed: int,
                        dx=1e-3, sphere_diam_dx=3.0, rho_ratio=2.7, jitter=0.01, dt=1e-5,
                        mesoscale=False, **over) -> dict:
    """One reverse-Poiseuille slurry instance of the batched sweep: an
    n x 2n x n periodic lattice (n = round((N_f/2)^(1/3))), spheres of
    diameter 3 dx and density 2.7 rho0 on random lattice sites up to solid
    volume fraction phi, viscosity from an Arrhenius law at temperature T,
    forcing amplitude g_amp.  With mesoscale=True the paper's units are used
    (rho0 = 3, eta = 25 mu(T)/mu(293 K), kBT = T/293.15)."""
    n = max(8, int(round((n_fluid_target / 2.0) ** (1.0 / 3.0))))
    if mesoscale:
        mu_ratio = arrhenius_viscosity(T) / arrhenius_viscosity(293.15)
        case = poiseuille_meso(nx=n, ny=2 * n, nz=n, eta=25.0 * mu_ratio, amp=g_amp,
                               kBT=T / 293.15, seed=seed, jitter=jitter)
        dx = case["params"]["dx"]
    else:
        eta = arrhenius_viscosity(T)
        case = poiseuille_si(nx=n, ny=2 * n, nz=n, dx=dx, g_amp=g_amp, seed=seed, jitter=jitter,
                             dt=dt, eta=eta, xi=20.0 * eta / 21.0, kBT=K_BOLTZMANN * T)
    for k, v in over.items():
        case["params"][k] = v
    params = case["params"]
    x = case["x"]
    R = 0.5 * sphere_diam_dx * dx
    Vs = 4.0 / 3.0 * math.pi * R ** 3
    Vbox = float(np.prod(params["box"]))
    n_sph = int(round(phi * Vbox / Vs))
    if n_sph > 0:
        rng = np.random.default_rng(seed + 7919)
        acc, _ = _place_spheres_on_sites((n, 2 * n, n), n_sph, np.array([sphere_diam_dx]),
                                         params["periodic"], rng)
        case["type"][acc] = T_RIGID
        case["radius"][acc] = R
        case["mass"][acc] = rho_ratio * params["rho0"] * Vs
    case["name"] = f"viscometer_n{n}_phi{phi:.3f}"
    case["meta"] = dict(phi_target=phi, T=T, g_amp=g_amp, n_spheres=int((case["type"] == T_RIGID).sum()))
    return case


def viscometer_batch(n_instances=64, seed=4, n_lo=20_000, n_hi=400_000, phi_hi=0.3,
                     T_lo=280.0, T_hi=350.0, g_lo=1e-3, g_hi=1e-1, mesoscale=False, **over):
    """The batched sweep: log-uniform fluid counts, uniform solid fraction and
    temperature, log-uniform forcing."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_instances):
        nf = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        phi = rng.uniform(0.0, phi_hi)
        T = rng.uniform(T_lo, T_hi)
        g = math.exp(rng.uniform(math.log(g_lo), math.log(g_hi)))
        out.append(viscometer_instance(int(nf), phi, T, g, seed=seed * 1000 + k,
                                       mesoscale=mesoscale, **over))
    return out


def tiny_box(n=6, dx=1.0, periodic=(1, 1, 1), r_c_dx=1.6, jitter=0.1, seed=3) -> dict:
    """A small jittered lattice for brute-force checks of the neighbour
    search (kernel radius r_c_dx spacings)."""
    params = base_params(dx=dx, r_c=r_c_dx * dx)
    params.update(box=[n * dx] * 3, periodic=list(periodic))
    rng = np.random.default_rng(seed)
    x = _jitter(lattice(n, n, n, dx), jitter * dx, rng)
    if not all(periodic):
        for a in range(3):
            if not periodic[a]:
                x[:, a] = np.clip(x[:, a], 0.0, n * dx)
    m = len(x)
    return _assemble(params, [(x, T_FLUID, np.full(m, 0.5 * dx), np.full(m, params["rho0"] * dx ** 3))],
                     "tiny_box")
