"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def pair_set(ij):
    ij = np.sort(np.asarray(ij), axis=1)
    return set(map(tuple, ij.tolist()))


# tolerances (relative L2 over all particles) fixed by the accuracy targets:
# FP64 pair arithmetic <= 1e-5 (summation order is the only difference, so
# ~1e-12 is expected); split precision <= 2e-4.
TOL_FORCE = {0: 1e-5, 1: 2e-4}


def philox_kat():
    """The published Philox4x32-10 known-answer vectors of tests/golden/
    (counter [n,4], key [n,2], expected output [n,4], uint32)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([int(t, 16) for t in line.split()])
    a = np.array(rows, dtype=np.uint64).astype(np.uint32)
    return a[:, 0:4], a[:, 4:6], a[:, 6:10]


def per_type_errors(g, o, types, idx=None):
    """Relative L2 errors of the force and the torque separately over the
    fluid particles (type 0) and the rigid particles (type 1), so that an
    error on the few spheres is not hidden under the fluid's norm.  g, o:
    state dicts with "F" and "N"; idx: restrict to these particles."""
    types = np.asarray(types)
    sel = np.arange(len(types)) if idx is None else np.asarray(idx)
    out = {}
    for name, t in (("fluid", 0), ("rigid", 1)):
        k = sel[types[sel] == t]
        if len(k) == 0:
            continue
        out[name] = {q: rel_l2(g[q][k], o[q][k]) for q in ("F", "N")}
    return out


def check_per_type(g, o, types, tol, idx=None):
    errs = per_type_errors(g, o, types, idx)
    for name, e in errs.items():
        for q, v in e.items():
            assert v < tol, (name, q, v, errs)
    return errs
