"""Thin ctypes binding of libsdpd (include/sdpd.h): argument marshalling only.

Every step of the SDPD-DEM path runs in the library's CUDA kernels; this module
converts numpy arrays / torch tensors to pointers and status codes to
exceptions.  There is no CPU fallback: if the library is missing, ``load()``
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SDPD_PREC_FP64 = 0
SDPD_PREC_SPLIT = 1

STATUS = {0: "SDPD_OK", 1: "SDPD_E_INVALID", 2: "SDPD_E_CUDA", 3: "SDPD_E_OOM",
          4: "SDPD_E_CAPACITY", 5: "SDPD_E_NONFINITE", 6: "SDPD_E_DOMAIN",
          7: "SDPD_E_TIMEOUT", 8: "SDPD_E_STATE"}
SDPD_E_INVALID = 1
SDPD_MAX_NEIGHBORS = 3072   # include/sdpd.h


class SdpdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class SdpdParams(C.Structure):
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
        ("seed", C.c_ulonglong),
    ]


def make_params(p: dict) -> SdpdParams:
    s = SdpdParams()
    for name, _ in SdpdParams._fields_:
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


_lib = None
EXPORTS = ["sdpd_init", "sdpd_destroy", "sdpd_set_particles", "sdpd_upload_state",
           "sdpd_download_state", "sdpd_set_step", "sdpd_get_step", "sdpd_build_cells",
           "sdpd_compute_density", "sdpd_couple_drag", "sdpd_compute_forces", "sdpd_integrate",
           "sdpd_step", "sdpd_viscosity_probe", "sdpd_get_state", "sdpd_get_drag",
           "sdpd_get_pairs", "sdpd_count_pairs", "sdpd_diagnostics", "sdpd_graph_kernels",
           "sdpd_set_force_mode", "sdpd_set_noise_cache", "sdpd_set_skin", "sdpd_set_block_size", "sdpd_set_threads_per_particle", "sdpd_set_cell_factor", "sdpd_build_count", "sdpd_density_noalloc",
           "sdpd_check",
           "sdpd_last_error", "sdpd_noise_normals", "sdpd_philox4x32_10", "sdpd_alu_peaks", "sdpd_viscosity_fit", "sdpd_checkpoint_size", "sdpd_checkpoint", "sdpd_restore", "mlp_init", "mlp_destroy", "mlp_param_count", "mlp_set_params",
           "mlp_get_params", "mlp_gradients", "mlp_train_step", "mlp_infer", "mlp_check"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsdpd.so (building it with nvcc if absent).  Raises if it cannot
    be built or loaded -- there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libsdpd not built: {path} missing")
        _build.build()
    L = C.CDLL(path)
    vp, dp, ip, llp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_longlong)
    st = C.c_int
    sig = {
        "sdpd_init": (st, [C.POINTER(SdpdParams), C.c_int, llp, C.c_int, C.c_int, C.c_int,
                           C.POINTER(vp)]),
        "sdpd_destroy": (None, [vp]),
        "sdpd_set_particles": (st, [vp, C.c_int, C.c_longlong, dp, dp, dp, ip, dp, dp]),
        "sdpd_upload_state": (st, [vp, vp, vp, vp, vp]),
        "sdpd_download_state": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "sdpd_set_step": (st, [vp, C.c_longlong]),
        "sdpd_get_step": (st, [vp, llp]),
        "sdpd_build_cells": (st, [vp, vp]),
        "sdpd_compute_density": (st, [vp, vp]),
        "sdpd_couple_drag": (st, [vp, vp]),
        "sdpd_compute_forces": (st, [vp, C.c_int, vp]),
        "sdpd_integrate": (st, [vp, C.c_int, vp]),
        "sdpd_step": (st, [vp, C.c_longlong, vp]),
        "sdpd_viscosity_probe": (st, [vp, C.c_int, C.c_int, dp, dp]),
        "sdpd_get_state": (st, [vp, C.c_int, dp, dp, dp, dp, dp, dp, dp]),
        "sdpd_get_drag": (st, [vp, C.c_int, dp, dp]),
        "sdpd_get_pairs": (st, [vp, C.c_int, C.c_longlong, ip, llp]),
        "sdpd_count_pairs": (st, [vp, llp]),
        "sdpd_diagnostics": (st, [vp, C.c_int, dp]),
        "sdpd_graph_kernels": (st, [vp, llp]),
        "sdpd_set_force_mode": (st, [vp, C.c_int]),
        "sdpd_set_noise_cache": (st, [vp, C.c_int]),
        "sdpd_set_skin": (st, [vp, C.c_double]),
        "sdpd_set_block_size": (st, [vp, C.c_int]),
        "sdpd_density_noalloc": (st, [C.POINTER(SdpdParams), C.c_longlong, vp, vp, vp, vp, vp]),
        "sdpd_check": (st, [vp]),
        "sdpd_last_error": (C.c_char_p, []),
        "sdpd_viscosity_fit": (st, [vp, C.c_int, C.c_int, C.POINTER(C.c_double)]),
        "sdpd_checkpoint_size": (st, [vp, C.POINTER(C.c_longlong)]),
        "sdpd_checkpoint": (st, [vp, vp, C.c_longlong]),
        "sdpd_restore": (st, [vp, vp, C.c_longlong]),
        "sdpd_noise_normals": (st, [C.c_int, C.c_ulonglong, C.c_int, C.c_uint, C.c_longlong, vp, vp, vp]),
        "sdpd_philox4x32_10": (st, [C.c_longlong, vp, vp, vp]),
        "sdpd_set_threads_per_particle": (st, [vp, C.c_int]),
        "sdpd_set_cell_factor": (st, [vp, C.c_int]),
        "sdpd_build_count": (st, [vp, C.POINTER(C.c_longlong)]),
        "sdpd_alu_peaks": (st, [vp]),
        "mlp_init": (st, [C.c_int, C.c_int, C.c_int, C.c_ulonglong, C.c_int, C.POINTER(vp)]),
        "mlp_destroy": (None, [vp]),
        "mlp_param_count": (C.c_int, []),
        "mlp_set_params": (st, [vp, vp]),
        "mlp_get_params": (st, [vp, vp, vp]),
        "mlp_gradients": (st, [vp, vp, vp, C.c_int, C.POINTER(C.c_float), vp]),
        "mlp_train_step": (st, [vp, vp, vp, C.c_int, C.c_float, C.POINTER(C.c_float), vp]),
        "mlp_infer": (st, [vp, vp, vp, C.c_longlong, vp]),
        "mlp_check": (st, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code: int):
    if code != 0:
        raise SdpdError(code, load().sdpd_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _stream(stream) -> C.c_void_p:
    if stream is None:
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(int(stream.cuda_stream))  # torch.cuda.Stream


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(int(a.data_ptr()))


NOALLOC_MAX_PARTICLES = 131072
NOALLOC_MAX_CELLS = 65536


def _check_noalloc_args(x, type_, d_out, p_out):
    """The arrays sdpd_density_noalloc reads and writes: CUDA tensors on one
    device, contiguous, x float64 [n, 3], type_ int32 [n], d_out and p_out
    float64 [n].  Raises ValueError otherwise (before any library call)."""
    import torch
    arrs = {"x": x, "type_": type_, "d_out": d_out, "p_out": p_out}
    want = {"x": torch.float64, "type_": torch.int32, "d_out": torch.float64, "p_out": torch.float64}
    for name, a in arrs.items():
        if not isinstance(a, torch.Tensor) or not a.is_cuda:
            raise ValueError(f"density_noalloc: {name} must be a CUDA tensor")
        if a.dtype != want[name]:
            raise ValueError(f"density_noalloc: {name} must be {want[name]}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"density_noalloc: {name} must be contiguous")
    if x.dim() != 2 or x.shape[1] != 3:
        raise ValueError(f"density_noalloc: x must be [n, 3], got {tuple(x.shape)}")
    n = int(x.shape[0])
    for name in ("type_", "d_out", "p_out"):
        if tuple(arrs[name].shape) != (n,):
            raise ValueError(f"density_noalloc: {name} must be [{n}], got {tuple(arrs[name].shape)}")
    devs = {a.device for a in arrs.values()}
    if len(devs) != 1:
        raise ValueError(f"density_noalloc: all arrays must be on one device, got {sorted(map(str, devs))}")
    return n


def density_noalloc(params: dict, x, type_, d_out, p_out, stream=None):
    """Number density and pressure of one particle set with no device
    allocation (sdpd_density_noalloc).  x [n,3] float64, type_ [n] int32,
    d_out / p_out [n] float64: contiguous CUDA tensors on the current device."""
    n = _check_noalloc_args(x, type_, d_out, p_out)
    prm = make_params(params)
    _check(load().sdpd_density_noalloc(C.byref(prm), n, _ptr(x), _ptr(type_), _ptr(d_out),
                                       _ptr(p_out), _stream(stream)))


class Sim:
    """A libsdpd context holding one or more instances (cases)."""

    def __init__(self, cases, precision: int = SDPD_PREC_FP64, max_neighbors: int = 0,
                 max_contacts: int = 0):
        if isinstance(cases, dict):
            cases = [cases]
        L = load()
        self.cases = cases
        self.n_inst = len(cases)
        self.precision = precision
        self.counts = [int(c["x"].shape[0]) for c in cases]
        self.offsets = np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)
        self.N = int(self.offsets[-1])
        params = (SdpdParams * self.n_inst)(*[make_params(c["params"]) for c in cases])
        counts = (C.c_longlong * self.n_inst)(*self.counts)
        h = C.c_void_p()
        _check(L.sdpd_init(params, self.n_inst, counts, int(precision), int(max_neighbors),
                           int(max_contacts), C.byref(h)))
        self._h = h
        for k, c in enumerate(cases):
            self.set_particles(k, c)

    def close(self):
        if getattr(self, "_h", None):
            load().sdpd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ state
    def set_particles(self, k: int, c: dict):
        x = np.ascontiguousarray(c["x"], dtype=np.float64)
        v = np.ascontiguousarray(c["v"], dtype=np.float64)
        w = np.ascontiguousarray(c["w"], dtype=np.float64)
        t = np.ascontiguousarray(c["type"], dtype=np.int32)
        R = np.ascontiguousarray(c["radius"], dtype=np.float64)
        m = np.ascontiguousarray(c["mass"], dtype=np.float64)
        _check(load().sdpd_set_particles(self._h, k, x.shape[0], _dp(x), _dp(v), _dp(w), _ip(t),
                                         _dp(R), _dp(m)))

    def upload_state(self, x=None, v=None, w=None, stream=None):
        _check(load().sdpd_upload_state(self._h, _ptr(x), _ptr(v), _ptr(w), _stream(stream)))

    def download_state(self, x=None, v=None, w=None, F=None, N=None, stream=None):
        _check(load().sdpd_download_state(self._h, _ptr(x), _ptr(v), _ptr(w), _ptr(F), _ptr(N),
                                          _stream(stream)))

    def build_count(self) -> int:
        """Neighbour-list builds run so far (forced and skin-triggered)."""
        n = C.c_longlong()
        _check(load().sdpd_build_count(self._h, C.byref(n)))
        return n.value

    @property
    def step_count(self) -> int:
        s = C.c_longlong()
        _check(load().sdpd_get_step(self._h, C.byref(s)))
        return s.value

    @step_count.setter
    def step_count(self, k: int):
        _check(load().sdpd_set_step(self._h, int(k)))

    def state(self, k: int = 0, density: bool = True) -> dict:
        n = self.counts[k]
        out = {name: np.zeros((n, 3)) for name in ("x", "v", "w", "F", "N")}
        if density:
            out["d"] = np.zeros(n)
            out["p"] = np.zeros(n)
        _check(load().sdpd_get_state(self._h, k, _dp(out["x"]), _dp(out["v"]), _dp(out["w"]),
                                     _dp(out["F"]), _dp(out["N"]),
                                     _dp(out["d"]) if density else None,
                                     _dp(out["p"]) if density else None))
        return out

    def drag(self, k: int = 0):
        nr = int((self.cases[k]["type"] == 1).sum())
        eps = np.zeros(nr)
        F = np.zeros((nr, 3))
        _check(load().sdpd_get_drag(self._h, k, _dp(eps), _dp(F)))
        return eps, F

    def pairs(self, k: int = 0) -> np.ndarray:
        n = C.c_longlong()
        _check(load().sdpd_get_pairs(self._h, k, 0, None, C.byref(n)))
        ij = np.zeros(2 * max(n.value, 1), dtype=np.int32)
        _check(load().sdpd_get_pairs(self._h, k, n.value, _ip(ij), C.byref(n)))
        return ij[: 2 * n.value].reshape(-1, 2)

    def count_pairs(self) -> int:
        n = C.c_longlong()
        _check(load().sdpd_count_pairs(self._h, C.byref(n)))
        return n.value

    def diagnostics(self, k: int = 0) -> np.ndarray:
        out = np.zeros(16)
        _check(load().sdpd_diagnostics(self._h, k, _dp(out)))
        return out

    def viscosity_fit(self, k: int = 0, n_bins: int = 32) -> float:
        """Viscosity from the curvature of the steady profile (sdpd_viscosity_fit)."""
        mu = C.c_double()
        _check(load().sdpd_viscosity_fit(self._h, k, n_bins, C.byref(mu)))
        return mu.value

    def checkpoint(self) -> np.ndarray:
        """The dynamic state as a byte image (sdpd_checkpoint)."""
        n = C.c_longlong()
        _check(load().sdpd_checkpoint_size(self._h, C.byref(n)))
        buf = np.zeros(n.value, dtype=np.uint8)
        _check(load().sdpd_checkpoint(self._h, C.c_void_p(buf.ctypes.data), n.value))
        return buf

    def restore(self, image) -> None:
        buf = np.ascontiguousarray(image, dtype=np.uint8)
        _check(load().sdpd_restore(self._h, C.c_void_p(buf.ctypes.data), buf.size))

    def viscosity_probe(self, k: int = 0, n_bins: int = 32):
        prof = np.zeros(n_bins)
        mu = np.zeros(1)
        _check(load().sdpd_viscosity_probe(self._h, k, n_bins, _dp(prof), _dp(mu)))
        return prof, float(mu[0])

    # ------------------------------------------------------------ stages
    def build_cells(self, stream=None):
        _check(load().sdpd_build_cells(self._h, _stream(stream)))

    def compute_density(self, stream=None):
        _check(load().sdpd_compute_density(self._h, _stream(stream)))

    def couple_drag(self, stream=None):
        _check(load().sdpd_couple_drag(self._h, _stream(stream)))

    def compute_forces(self, velver: int, stream=None):
        _check(load().sdpd_compute_forces(self._h, int(velver), _stream(stream)))

    def integrate(self, velver: int, stream=None):
        _check(load().sdpd_integrate(self._h, int(velver), _stream(stream)))

    def evaluate(self, velver: int = 1, stream=None):
        """Forces of one sub-step at the current state (Algorithm 1 without the
        update): build cells, density, drag, forces."""
        self.build_cells(stream)
        self.compute_density(stream)
        self.couple_drag(stream)
        self.compute_forces(velver, stream)

    def step(self, n: int = 1, stream=None):
        _check(load().sdpd_step(self._h, int(n), _stream(stream)))

    def set_force_mode(self, newton3: int):
        _check(load().sdpd_set_force_mode(self._h, int(newton3)))

    def set_noise_cache(self, on: bool):
        _check(load().sdpd_set_noise_cache(self._h, int(bool(on))))

    def set_block_size(self, threads: int):
        _check(load().sdpd_set_block_size(self._h, int(threads)))

    def set_threads_per_particle(self, tpp: int):
        _check(load().sdpd_set_threads_per_particle(self._h, int(tpp)))

    def set_cell_factor(self, cells: int):
        """Cells per minimum cell width of the neighbour search: 1 or 2."""
        _check(load().sdpd_set_cell_factor(self._h, int(cells)))

    def set_skin(self, skin: float):
        _check(load().sdpd_set_skin(self._h, float(skin)))

    def graph_kernels(self) -> int:
        n = C.c_longlong()
        _check(load().sdpd_graph_kernels(self._h, C.byref(n)))
        return n.value

    def check(self):
        _check(load().sdpd_check(self._h))


def philox4x32_10(ctr, key) -> np.ndarray:
    """Raw Philox4x32-10 blocks computed on the GPU (sdpd_philox4x32_10):
    ctr [n, 4] and key [n, 2] uint32 -> [n, 4] uint32."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    if c.shape[0] != k.shape[0]:
        raise ValueError("philox4x32_10: one key per counter")
    out = np.zeros_like(c)
    _check(load().sdpd_philox4x32_10(c.shape[0], _ptr(c), _ptr(k), _ptr(out)))
    return out


def alu_peaks() -> dict:
    """Measured FP32 / FP64 FMA and INT32 IMAD throughput of the current GPU
    (sdpd_alu_peaks)."""
    out = np.zeros(4)
    _check(load().sdpd_alu_peaks(_ptr(out)))
    return {"fp32_tflops": float(out[0]), "fp64_tflops": float(out[1]), "int32_tops": float(out[2]),
            "sms": int(out[3])}


def noise_normals(precision: int, seed: int, inst: int, step: int, gi, gj) -> np.ndarray:
    """The six normals of the random pair term for pairs (gi, gj) ([n][6])."""
    gi = np.ascontiguousarray(gi, dtype=np.uint32)
    gj = np.ascontiguousarray(gj, dtype=np.uint32)
    z = np.zeros((len(gi), 6))
    _check(load().sdpd_noise_normals(int(precision), int(seed), int(inst), int(step), len(gi),
                                     C.c_void_p(gi.ctypes.data), C.c_void_p(gj.ctypes.data),
                                     C.c_void_p(z.ctypes.data)))
    return z


class Mlp:
    """The tensor-core surrogate network (mlp_* entry points)."""

    def __init__(self, seed: int = 0, batch_max: int = 256):
        h = C.c_void_p()
        _check(load().mlp_init(3, 128, 4, int(seed), int(batch_max), C.byref(h)))
        self._h = h
        self.n_params = int(load().mlp_param_count())

    def close(self):
        if getattr(self, "_h", None):
            load().mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.n_params
        _check(load().mlp_set_params(self._h, C.c_void_p(a.ctypes.data)))

    def params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(load().mlp_get_params(self._h, C.c_void_p(p.ctypes.data), None))
        return p

    def grads(self):
        g = np.zeros(self.n_params, dtype=np.float32)
        _check(load().mlp_get_params(self._h, None, C.c_void_p(g.ctypes.data)))
        return g

    def gradients(self, X, T, stream=None) -> float:
        loss = C.c_float()
        _check(load().mlp_gradients(self._h, _ptr(X), _ptr(T), int(X.shape[0]), C.byref(loss),
                                    _stream(stream)))
        return loss.value

    def train_step(self, X, T, lr=1e-3, stream=None, want_loss=True):
        loss = C.c_float()
        _check(load().mlp_train_step(self._h, _ptr(X), _ptr(T), int(X.shape[0]), float(lr),
                                     C.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None

    def infer(self, X, Y, stream=None):
        _check(load().mlp_infer(self._h, _ptr(X), _ptr(Y), int(X.shape[0]), _stream(stream)))

    def check(self):
        _check(load().mlp_check(self._h))
