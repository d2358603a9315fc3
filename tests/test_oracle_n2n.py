"""Table 1 as message passing (oracle/n2n.py, one thread per subgraph): the iterates equal the
synchronous iteration bit for bit, also with late and reordered messages; a dropped message ends
the run with a timeout instead of a hang (host-side failure detection; no GPU involved)."""
import time

import numpy as np
import pytest

from oracle import evs, n2n
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs


def _setup():
    A = inputs.grid_poisson((20, 17), sigma=0.7, seed=71)
    split = evs.split_grid(A, (20, 17), (7, 6))       # 3 x 3 subgraphs, 2-cube corners
    b = inputs.rhs_uniform(A.n, 2, seed=71)
    Z = np.random.default_rng(2).uniform(0.5, 2.0, len(split.vtl))
    return A, split, b, Z


def _sync(split, Z, b, k):
    m = ovtm.VTM(split, Z)
    st = m.initial_state(2)
    for _ in range(k):
        st = m.sweep(st, b)
    return st


def _same(a, b):
    assert np.array_equal(a.u, b.u) and np.array_equal(a.omega, b.omega)
    for xa, xb in zip(a.x_local, b.x_local):
        assert np.array_equal(xa, xb)


def test_message_passing_equals_synchronous_iteration():
    A, split, b, Z = _setup()
    _same(n2n.N2N(split, Z).run(b, 12), _sync(split, Z, b, 12))


def test_late_and_reordered_messages():
    A, split, b, Z = _setup()
    rng = np.random.default_rng(3)
    E = 2 * len(split.vtl)
    delay = {(int(k), int(e)): 0.002 for k, e in zip(rng.integers(1, 8, 40), rng.integers(0, E, 40))}
    st = n2n.N2N(split, Z, delay=delay, reverse=True).run(b, 8)
    _same(st, _sync(split, Z, b, 8))


def test_dropped_message_times_out():
    A, split, b, Z = _setup()
    t0 = time.perf_counter()
    with pytest.raises(n2n.N2NTimeout):
        n2n.N2N(split, Z, timeout=0.3, drop={(4, 7)}).run(b, 10)
    assert time.perf_counter() - t0 < 10.0
