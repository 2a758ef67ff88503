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
