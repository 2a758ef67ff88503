"""Pin of the oracle's background-grid neighbour search (Section 3.2) against
brute force on tiny boxes: the pair sets must be identical."""
import numpy as np
import pytest

import oracle
from paper_2002_03120_gb300 import cases


def _set(ij):
    return set(map(tuple, np.sort(ij, axis=1).tolist()))


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 1, 0), (0, 0, 0), (0, 1, 1)])
@pytest.mark.parametrize("n,rcdx", [(6, 1.6), (7, 2.2), (9, 3.9)])
def test_cell_search_equals_brute_force(periodic, n, rcdx):
    c = cases.tiny_box(n=n, periodic=periodic, r_c_dx=rcdx, jitter=0.3, seed=n)
    s = oracle.OracleSim(c)
    s.neighbors()
    got = _set(s.pairs())
    ref = _set(oracle.pairs_brute(c["params"], c["x"]))
    assert got == ref
    assert len(ref) > 0


def test_empty_and_single():
    c = cases.tiny_box(n=6)
    c1 = {k: (v[:1] if isinstance(v, np.ndarray) else v) for k, v in c.items()}
    s = oracle.OracleSim(c1)
    s.neighbors()
    assert len(s.pairs()) == 0
