"""The global residual from port data alone (oracle/vtm.py residual_from_ports) equals the plain
b - A x̄ of the assembled iterate: KCL plus the local equation of eq. 5.8, uncoupled and coupled
lines, multilevel corners, several right-hand sides."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coupled, evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs


@pytest.mark.parametrize("dims,block,k", [((24, 21), (8, 7), 5), ((9, 8, 7), (4, 4, 3), 9)])
def test_port_residual_equals_plain_residual(dims, block, k):
    A = inputs.grid_poisson(dims, sigma=0.8, seed=61)
    split = evs.split_grid(A, dims, block)
    b = inputs.rhs_uniform(A.n, 2, seed=61)
    Z = np.random.default_rng(1).uniform(0.5, 3.0, len(split.vtl))
    m = ovtm.VTM(split, Z)
    st = m.initial_state(2)
    for _ in range(k):
        st = m.sweep(st, b)
    plain = b - (A.to_scipy() @ m.assemble(st).T).T
    got = ovtm.residual_from_ports(split, st)
    assert np.max(np.abs(got - plain)) <= 1e-12 * np.max(np.abs(b))
    # nonzero only at boundary vertices and their first interior neighbours
    ncopy = np.zeros(A.n, dtype=int)
    for g in split.subgraphs:
        np.add.at(ncopy, g.vertices, 1)
    near = (abs(A.to_scipy()) @ (ncopy > 1).astype(float)) > 0
    assert np.all(got[:, ~near] == 0)


def test_port_residual_coupled_lines():
    dims, block = (20, 18), (7, 6)
    A = inputs.grid_poisson(dims, sigma=0.5, seed=62)
    split = evs.split_grid(A, dims, block)
    pairs, w = coupled.adjacent_line_pairs(split, A)
    m = coupled.CoupledVTM(split, coupled.laplacian_admittance(split, 3.0, pairs, 0.7 * w))
    b = inputs.rhs_uniform(A.n, 1, seed=62)
    st = m.initial_state()
    for _ in range(6):
        st = m.sweep(st, b)
    plain = b - (A.to_scipy() @ m.assemble(st).T).T
    assert np.max(np.abs(ovtm.residual_from_ports(split, st) - plain)) <= 1e-12 * np.max(np.abs(b))
