"""The random stream of the pair kernels (Eq. FijT noise: Philox4x32-10 and
Box-Muller, through sdpd_noise_normals) against the oracle's draw of the same
pairs.  The FP64 transform on the GPU is table-driven (Tang's logarithm,
angle addition), the oracle's uses the C library's log, cos and sin: they
agree to a few units in the last place."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import binding as B

from _gpu_common import need_gpu, philox_kat

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    gi = rng.integers(0, 1 << 22, size=n, dtype=np.uint32)
    gj = rng.integers(0, 1 << 22, size=n, dtype=np.uint32)
    gj[gj == gi] += 1
    return gi, gj


# FP64 bound: the oracle forms the angle 2 pi U in double (up to half an ulp
# of 2 pi, 4.4e-16, absolute) and the radius reaches 5.8, so its own draws
# carry up to ~2.6e-15; the GPU reduces the angle exactly from the integer.
# FP32 bound: hardware sine and cosine (absolute error below 2^-21.4), the
# FP32 angle (half an ulp of pi) and the radius to a few ulp, times a radius
# up to 5.8: about 5e-6 at worst, far inside the split path's force error.
@pytest.mark.parametrize("prec,tol", [(B.SDPD_PREC_FP64, 1e-14), (B.SDPD_PREC_SPLIT, 1e-5)])
def test_normals_match_oracle(prec, tol):
    gi, gj = _pairs(20000, 1)
    seed, inst, step = 0x1234_5678_9ABC_DEF0, 3, 77
    z = B.noise_normals(prec, seed, inst, step, gi, gj)
    ref = np.array([oracle.pair_normals(seed, inst, a, b, step) for a, b in zip(gi, gj)])
    err = np.abs(z - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < tol, err.max()
    # the tails reach beyond 4 sigma: the logarithm was exercised far from 1
    assert np.abs(ref).max() > 4.0


def test_normals_symmetric_and_keyed():
    gi, gj = _pairs(4096, 2)
    a = B.noise_normals(B.SDPD_PREC_FP64, 9, 0, 5, gi, gj)
    b = B.noise_normals(B.SDPD_PREC_FP64, 9, 0, 5, gj, gi)
    assert np.array_equal(a, b)
    c = B.noise_normals(B.SDPD_PREC_FP64, 9, 1, 5, gi, gj)   # another instance
    d = B.noise_normals(B.SDPD_PREC_FP64, 9, 0, 6, gi, gj)   # another step
    assert np.mean(a == c) < 1e-3 and np.mean(a == d) < 1e-3


def test_gpu_philox_known_answer_vectors():
    # the generator the pair kernels run, against the published vectors
    ctr, key, want = philox_kat()
    got = B.philox4x32_10(ctr, key)
    assert np.array_equal(got, want)
    # and bit for bit with the oracle over many counters and keys
    rng = np.random.default_rng(4)
    c = rng.integers(0, 1 << 32, size=(5000, 4), dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 1 << 32, size=(5000, 2), dtype=np.uint64).astype(np.uint32)
    g = B.philox4x32_10(c, k)
    ref = np.array([oracle.philox(a.tolist(), b.tolist()) for a, b in zip(c, k)], dtype=np.uint32)
    assert np.array_equal(g, ref)
