"""Sobol low-discrepancy points in up to 3 dimensions (Bratley & Fox
construction, Gray-code order).

Direction numbers: dimension 1 is the van der Corput sequence in base 2
(v_k = 2^-k); dimensions 2 and 3 come from the primitive polynomials x + 1
(degree 1, initial m = 1) and x^2 + x + 1 (degree 2, initial m = 1, 3) through
the recurrence  m_k = 2 a_1 m_{k-1} ^ ... ^ 2^(s-1) a_{s-1} m_{k-s+1}
^ 2^s m_{k-s} ^ m_{k-s}.
"""
from __future__ import annotations

import numpy as np

BITS = 32
# (degree s, coefficients a_1..a_{s-1} packed as bits, initial m_1..m_s)
_POLYS = [(1, 0, [1]), (2, 1, [1, 3])]


def _directions(dim: int) -> np.ndarray:
    v = np.zeros((dim, BITS), dtype=np.uint64)
    for k in range(BITS):
        v[0, k] = 1 << (BITS - 1 - k)
    for d in range(1, dim):
        s, a, m0 = _POLYS[d - 1]
        m = list(m0)
        for k in range(s, BITS):
            new = m[k - s] ^ (m[k - s] << s)
            for i in range(1, s):
                if (a >> (s - 1 - i)) & 1:
                    new ^= m[k - i] << i
            m.append(new)
        for k in range(BITS):
            v[d, k] = m[k] << (BITS - 1 - k)
    return v


def sobol(n: int, dim: int = 3, skip: int = 0) -> np.ndarray:
    """n points in [0, 1)^dim (the first point is the origin unless skipped)."""
    if not 1 <= dim <= 3:
        raise ValueError("dim must be 1..3")
    v = _directions(dim)
    x = np.zeros(dim, dtype=np.uint64)
    out = np.empty((n + skip, dim))
    for i in range(n + skip):
        out[i] = x / float(1 << BITS)
        c = (~i & (i + 1)).bit_length() - 1  # index of the lowest zero bit of i
        x = x ^ v[:, c]
    return out[skip:]
