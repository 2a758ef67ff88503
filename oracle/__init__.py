"""Plain FP64 CPU oracle of the SDPD-DEM interaction step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and this package never imports the product.

The arithmetic lives in ``sdpd_oracle.c`` (Algorithms 1 and 2 and the
equations of Section 2 of the paper, in their order); this module compiles it
with gcc (``-O2 -ffp-contract=off``) on first use and marshals numpy arrays.

Parity pins (tests/test_oracle_*.py): every function here is checked
against something other than itself -- closed forms (Lucy kernel integral,
perfect-lattice density, drag laws, Reynolds lubrication, Archimedes'
buoyancy, the viscous part of the pressure-gradient force on a moving
sphere, restitution and rolling of DEM contacts, free fall, the Poiseuille
profile and its read-outs), brute force (neighbour sets), invariants
(antisymmetry, momentum, dissipation, fluctuation-dissipation, equipartition)
and published known-answer vectors (Philox4x32-10).  Parity unpinned, at the
level of whole trajectories only: the absolute viscosity of the viscometer
with solids and the dam-break run (the paper prints no data for them), and
the settling velocity of the sedimentation case (its ODE does not hold for
the model as printed); their forces are pinned one by one, and only
invariants are checked for the runs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdpd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

T_FLUID, T_RIGID, T_INNER_WALL, T_OUTER_WALL = 0, 1, 2, 3


class OrcParams(C.Structure):
    _fields_ = [
        ("dx", C.c_double), ("r_c", C.c_double), ("dt", C.c_double),
        ("rho0", C.c_double), ("p0", C.c_double), ("alpha", C.c_double), ("beta_p", C.c_double),
        ("eta", C.c_double), ("xi", C.c_double), ("kBT", C.c_double),
        ("coeff_c", C.c_double), ("coeff_d", C.c_double), ("coeff_r", C.c_double),
        ("coeff_t", C.c_double),
        ("origin", C.c_double * 3), ("box", C.c_double * 3), ("g", C.c_double * 3),
        ("body_amp", C.c_double),
        ("artvis_alpha", C.c_double), ("artvis_e", C.c_double),
        ("kn", C.c_double), ("restitution", C.c_double), ("nu_p", C.c_double),
        ("E_p", C.c_double), ("mu_fric", C.c_double),
        ("lub_gap_min", C.c_double), ("eps_min", C.c_double),
        ("periodic", C.c_int * 3),
        ("body_axis", C.c_int), ("split_axis", C.c_int),
        ("pressure_filter", C.c_int), ("clamp_negative_p", C.c_int), ("artvis", C.c_int),
        ("dem_law", C.c_int), ("density_reinit", C.c_int),
        ("seed", C.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent).  With OpenMP where the
    compiler has it (the per-particle loops may then run on several threads;
    results do not depend on their number), else without."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB + f".tmp{os.getpid()}"
            base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99"]
            r = subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
            if r.returncode != 0:
                subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        up = C.POINTER(C.c_uint32)
        L.orc_W.restype = C.c_double
        L.orc_W.argtypes = [C.c_double, C.c_double]
        L.orc_Fk.restype = C.c_double
        L.orc_Fk.argtypes = [C.c_double, C.c_double]
        L.orc_kernel_norm.restype = C.c_double
        L.orc_kernel_norm.argtypes = [C.c_double, C.c_double]
        L.orc_eos.restype = C.c_double
        L.orc_eos.argtypes = [C.c_double] * 5
        L.orc_philox4x32_10.argtypes = [up, up, up]
        L.orc_pair_normals.argtypes = [C.c_uint64, C.c_int, C.c_uint32, C.c_uint32, C.c_longlong, dp]
        L.orc_noise_vector.argtypes = [dp, C.c_double, C.c_double, dp, dp]
        L.orc_drag_force.argtypes = [C.c_double] * 5 + [dp, dp]
        L.orc_dem_coeffs.argtypes = [C.POINTER(OrcParams), C.c_double, C.c_double, C.c_double,
                                     C.c_double, dp]
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcParams), C.c_int, C.c_int, dp, dp, dp, ip, dp, dp,
                                 C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_step.argtypes = [C.c_void_p, C.c_longlong]
        L.orc_get_step.restype = C.c_longlong
        L.orc_get_step.argtypes = [C.c_void_p]
        L.orc_set_state.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_get_state.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp, dp]
        L.orc_set_fields.argtypes = [C.c_void_p, dp, dp]
        L.orc_get_component.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get_fpi.argtypes = [C.c_void_p, dp, dp]
        L.orc_get_history.argtypes = [C.c_void_p, ip, ip, dp]
        L.orc_set_history.argtypes = [C.c_void_p, ip, ip, dp]
        L.orc_neighbors.argtypes = [C.c_void_p]
        L.orc_pairs_brute.restype = C.c_long
        L.orc_pairs_brute.argtypes = [C.POINTER(OrcParams), C.c_int, dp, C.c_long, ip]
        L.orc_get_pairs.restype = C.c_long
        L.orc_get_pairs.argtypes = [C.c_void_p, C.c_long, ip]
        L.orc_density.argtypes = [C.c_void_p]
        L.orc_reinit.argtypes = [C.c_void_p]
        L.orc_filter.argtypes = [C.c_void_p]
        L.orc_forces.argtypes = [C.c_void_p, C.c_int]
        L.orc_update.argtypes = [C.c_void_p, C.c_int]
        L.orc_artvis.argtypes = [C.c_void_p]
        L.orc_substep.argtypes = [C.c_void_p, C.c_int]
        L.orc_run.argtypes = [C.c_void_p, C.c_longlong]
        L.orc_evaluate.argtypes = [C.c_void_p, C.c_int]
        L.orc_profile.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_overflow.argtypes = [C.c_void_p]
        L.orc_set_sample.argtypes = [C.c_void_p, C.POINTER(C.c_ubyte)]
        L.orc_threads.restype = C.c_int
        L.orc_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def make_params(p: dict) -> OrcParams:
    """Fill the oracle's parameter struct from a case parameter dict."""
    s = OrcParams()
    for name, _ in OrcParams._fields_:
        val = p.get(name, 0) if name == "density_reinit" else p[name]
        if name in ("origin", "box", "g"):
            getattr(s, name)[:] = [float(v) for v in val]
        elif name == "periodic":
            getattr(s, name)[:] = [int(v) for v in val]
        elif name == "seed":
            s.seed = int(val)
        elif isinstance(getattr(s, name), int):
            setattr(s, name, int(val))
        else:
            setattr(s, name, float(val))
    return s


def threads(n: int = 0) -> int:
    """Set the number of threads of the oracle's per-particle loops (n > 0)
    and return the number in use (1 when built without OpenMP)."""
    return int(lib().orc_threads(int(n)))


# ---------------------------------------------------------------- pure functions
def W(r, h):
    return lib().orc_W(float(r), float(h))


def Fk(r, h):
    return lib().orc_Fk(float(r), float(h))


def kernel_norm(dx, h):
    return lib().orc_kernel_norm(float(dx), float(h))


def eos(rho, rho0, p0, alpha, beta):
    return lib().orc_eos(float(rho), float(rho0), float(p0), float(alpha), float(beta))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def pair_normals(seed, inst, gi, gj, step):
    z = np.zeros(6)
    lib().orc_pair_normals(int(seed), int(inst), int(gi), int(gj), int(step), _dp(z))
    return z


def noise_vector(z, sa, sb, e):
    z = np.ascontiguousarray(z, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_noise_vector(_dp(z), float(sa), float(sb), _dp(e), _dp(out))
    return out


def drag_force(eps, d, rho, mu, Vs, dv):
    dv = np.ascontiguousarray(dv, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_drag_force(float(eps), float(d), float(rho), float(mu), float(Vs), _dp(dv), _dp(out))
    return out


def dem_coeffs(params: dict, Ri, Rj, mi, mj):
    P = make_params(params)
    out = np.zeros(4)
    lib().orc_dem_coeffs(C.byref(P), float(Ri), float(Rj), float(mi), float(mj), _dp(out))
    return out


def pairs_brute(params: dict, x: np.ndarray, cap: int | None = None) -> np.ndarray:
    P = make_params(params)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    if cap is None:
        cap = n * 400
    ij = np.zeros(2 * cap, dtype=np.int32)
    cnt = lib().orc_pairs_brute(C.byref(P), n, _dp(x), cap, _ip(ij))
    if cnt > cap:
        return pairs_brute(params, x, cnt)
    return ij[: 2 * cnt].reshape(-1, 2)


# ---------------------------------------------------------------- simulation object
class OracleSim:
    """One instance of the FP64 oracle stepper (Algorithm 1)."""

    def __init__(self, case: dict, inst: int = 0, K: int = 16):
        L = lib()
        self.params = case["params"]
        self._P = make_params(self.params)
        self.n = int(case["x"].shape[0])
        self.K = K
        x = np.ascontiguousarray(case["x"], dtype=np.float64)
        v = np.ascontiguousarray(case["v"], dtype=np.float64)
        w = np.ascontiguousarray(case["w"], dtype=np.float64)
        t = np.ascontiguousarray(case["type"], dtype=np.int32)
        R = np.ascontiguousarray(case["radius"], dtype=np.float64)
        m = np.ascontiguousarray(case["mass"], dtype=np.float64)
        self._h = L.orc_create(C.byref(self._P), int(inst), self.n, _dp(x), _dp(v), _dp(w),
                               _ip(t), _dp(R), _dp(m), int(K))
        self.type = t.copy()
        self.mass = m.copy()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def step(self):
        return lib().orc_get_step(self._h)

    @step.setter
    def step(self, k):
        lib().orc_set_step(self._h, int(k))

    def set_state(self, x=None, v=None, w=None):
        keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (x, v, w)]
        lib().orc_set_state(self._h, *[None if a is None else _dp(a) for a in keep])

    def set_fields(self, d=None, p=None):
        """Impose number densities and/or pressures (test hook; the force
        routines then read these instead of those of density())."""
        keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (d, p)]
        lib().orc_set_fields(self._h, *[None if a is None else _dp(a) for a in keep])

    def state(self):
        n = self.n
        out = {k: np.zeros((n, 3)) for k in ("x", "v", "w", "F", "N")}
        out["d"] = np.zeros(n)
        out["p"] = np.zeros(n)
        lib().orc_get_state(self._h, _dp(out["x"]), _dp(out["v"]), _dp(out["w"]), _dp(out["F"]),
                            _dp(out["N"]), _dp(out["d"]), _dp(out["p"]))
        return out

    def component(self, which: str) -> np.ndarray:
        idx = {"sdpd": 0, "pg": 1, "dg": 2, "rxn": 3, "dem": 4, "lub": 5, "ext": 6,
               "N_sdpd": 7, "N_dem": 8, "vf": 9}[which]
        out = np.zeros((self.n, 3))
        lib().orc_get_component(self._h, idx, _dp(out))
        return out

    def fpi(self):
        eps = np.zeros(self.n)
        S = np.zeros(self.n)
        lib().orc_get_fpi(self._h, _dp(eps), _dp(S))
        return eps, S

    def history(self):
        cnt = np.zeros(self.n, dtype=np.int32)
        part = np.zeros(self.n * self.K, dtype=np.int32)
        dl = np.zeros(self.n * self.K * 3)
        lib().orc_get_history(self._h, _ip(cnt), _ip(part), _dp(dl))
        return cnt, part.reshape(self.n, self.K), dl.reshape(self.n, self.K, 3)

    def set_history(self, cnt, part, dl):
        cnt = np.ascontiguousarray(cnt, dtype=np.int32)
        part = np.ascontiguousarray(part, dtype=np.int32)
        dl = np.ascontiguousarray(dl, dtype=np.float64)
        lib().orc_set_history(self._h, _ip(cnt), _ip(part), _dp(dl))

    def neighbors(self):
        lib().orc_neighbors(self._h)

    def pairs(self) -> np.ndarray:
        cap = self.n * 400
        ij = np.zeros(2 * cap, dtype=np.int32)
        cnt = lib().orc_get_pairs(self._h, cap, _ip(ij))
        if cnt > cap:
            ij = np.zeros(2 * cnt, dtype=np.int32)
            cnt = lib().orc_get_pairs(self._h, cnt, _ip(ij))
        return ij[: 2 * cnt].reshape(-1, 2)

    def density(self):
        lib().orc_density(self._h)

    def reinit(self):
        lib().orc_reinit(self._h)

    def filter(self):
        lib().orc_filter(self._h)

    def forces(self, velver: int):
        lib().orc_forces(self._h, int(velver))

    def update(self, velver: int):
        lib().orc_update(self._h, int(velver))

    def artvis(self):
        lib().orc_artvis(self._h)

    def evaluate(self, velver: int = 1) -> int:
        return lib().orc_evaluate(self._h, int(velver))

    def substep(self, velver: int) -> int:
        return lib().orc_substep(self._h, int(velver))

    def run(self, nsteps: int) -> int:
        return lib().orc_run(self._h, int(nsteps))

    def profile(self, nbins: int):
        prof = np.zeros(nbins)
        mu = np.zeros(1)
        lib().orc_profile(self._h, int(nbins), _dp(prof), _dp(mu))
        return prof, float(mu[0])

    def diagnostics(self) -> np.ndarray:
        """Plain sums over the oracle's state (the definitions, no blocking):
        [0..2] total momentum sum m v and [3] kinetic energy 1/2 sum m v^2 of
        the mobile (fluid and rigid) particles, [4] their kinetic temperature
        (sum m v^2 - |P|^2 / M) / (3 n) in energy units (the kBT of the
        fluctuation-dissipation balance of Section 2.1 at equipartition),
        [5] max |v| over them, [6] min and [7] max number density over all
        but the outer walls (valid after density()), [8] the number of
        non-finite components of x, v and w over all particles."""
        st = self.state()
        t = self.type
        mob = (t == T_FLUID) | (t == T_RIGID)
        v = st["v"][mob]
        m = self.mass[mob]
        out = np.zeros(16)
        P = np.array([np.sum(m * v[:, a]) for a in range(3)])
        v2 = np.sum(v * v, axis=1)
        E2 = np.sum(m * v2)
        M = np.sum(m)
        n = int(np.sum(mob))
        out[0:3] = P
        out[3] = 0.5 * E2
        out[4] = (E2 - (P @ P) / M) / (3.0 * n) if n else 0.0
        out[5] = np.sqrt(v2.max()) if n else 0.0
        d = st["d"][t != T_OUTER_WALL]
        if len(d):
            out[6] = d.min()
            out[7] = d.max()
        out[8] = sum(int(np.sum(~np.isfinite(st[k]))) for k in ("x", "v", "w"))
        return out

    def viscosity_fit(self, nbins: int) -> float:
        """Viscosity from the curvature of the steady reverse-Poiseuille profile
        (Section 4.1: the parabola of Eq. poiseuanasol fitted to the convex
        and concave halves; reading B6): fluid particles binned into nbins
        slabs of split_axis; per half, a least-squares parabola (numpy
        polyfit) of the slab mean velocity along body_axis against the slab
        mean position, over the slabs whose mean position lies at least h
        from both ends of the half; steady state mu v'' = -rho0 a with
        a = +body_amp on the lower half and -body_amp on the upper one; the
        mean of the two halves."""
        P = self.params
        ax, fa = int(P["split_axis"]), int(P["body_axis"])
        L, h = float(P["box"][ax]), float(P["r_c"])
        st = self.state()
        fl = self.type == T_FLUID
        rel = st["x"][fl, ax] - float(P["origin"][ax])
        u = st["v"][fl, fa]
        b = np.clip(np.floor(rel / L * nbins).astype(np.int64), 0, nbins - 1)
        cnt = np.bincount(b, minlength=nbins).astype(np.float64)
        has = cnt > 0
        vmean = np.bincount(b, weights=u, minlength=nbins)[has] / cnt[has]
        ymean = np.bincount(b, weights=rel, minlength=nbins)[has] / cnt[has]
        mus = []
        for half in (0, 1):
            y0 = half * 0.5 * L
            y1 = y0 + 0.5 * L
            use = (ymean >= y0 + h) & (ymean <= y1 - h)
            if np.sum(use) < 4:
                raise ValueError("viscosity_fit: fewer than 4 slabs h away from the ends of a half")
            c2 = np.polyfit(ymean[use] - 0.5 * (y0 + y1), vmean[use], 2)[0]
            a = float(P["body_amp"]) if half == 0 else -float(P["body_amp"])
            mus.append(-float(P["rho0"]) * a / (2.0 * c2))
        return 0.5 * (mus[0] + mus[1])

    def set_sample(self, idx=None):
        """Compute forces only for the particles in idx (None: all)."""
        if idx is None:
            lib().orc_set_sample(self._h, None)
            return
        mask = np.zeros(self.n, dtype=np.uint8)
        mask[np.asarray(idx)] = 1
        lib().orc_set_sample(self._h, mask.ctypes.data_as(C.POINTER(C.c_ubyte)))

    def overflow(self) -> bool:
        return bool(lib().orc_overflow(self._h))
