"""The C-ABI library builds (nvcc, sm_103a) and exports every function that
include/sdpd.h declares.  No compute call: this runs without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2002_03120_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:sdpd|mlp)_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared("sdpd.h")
    for must in ("sdpd_init", "sdpd_build_cells", "sdpd_compute_forces", "sdpd_couple_drag", "mlp_train_step", "mlp_infer",
                 "sdpd_integrate", "sdpd_viscosity_probe"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for header in sorted(os.listdir(os.path.join(ROOT, "include"))):
        for name in _declared(header):
            assert hasattr(lib, name), f"{name} declared in {header} but not exported"
    assert set(binding.EXPORTS) <= set(_declared("sdpd.h"))


def test_last_error_callable_without_gpu():
    lib = binding.load()
    assert isinstance(lib.sdpd_last_error(), bytes)


def test_neighbour_capacity_is_bounded_without_gpu():
    # validated before the device is touched: SDPD_E_INVALID, not a launch failure
    from paper_2002_03120_gb300 import cases
    case = cases.poiseuille_si(nx=4, ny=8, nz=4)
    for bad in (-1, binding.SDPD_MAX_NEIGHBORS + 1):
        with pytest.raises(binding.SdpdError) as ei:
            binding.Sim(case, max_neighbors=bad)
        assert ei.value.code == binding.SDPD_E_INVALID


def test_noalloc_binding_checks_its_arrays_without_gpu():
    # host arrays, wrong dtypes or shapes are refused before the library is
    # called (a host pointer handed to a kernel would be an illegal address)
    import numpy as np
    import torch
    from paper_2002_03120_gb300 import cases
    case = cases.poiseuille_si(nx=4, ny=8, nz=4)
    n = len(case["x"])
    x = np.zeros((n, 3))
    t = np.zeros(n, dtype=np.int32)
    d = np.zeros(n)
    with pytest.raises(ValueError, match="CUDA tensor"):
        binding.density_noalloc(case["params"], x, t, d, d)
    xt = torch.zeros((n, 3), dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        binding.density_noalloc(case["params"], xt, torch.zeros(n, dtype=torch.int32),
                                torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64))
