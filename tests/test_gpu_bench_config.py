"""The benchmarked configurations, element by element against the coupled FP64 oracle (§7.2).

The timed runs use 17^3 subgraphs (cut planes every 16 nodes), learned impedances scaled by the
model's z_scale and every candidate pair of lines of a bundle coupled by gamma |a_ik| (the rule
stored with the model), FP32 sweeps in port form:
  * 128^3, one right-hand side: the port responses S_j stored in FP16 (per-tile scale);
  * 256^3, 32 right-hand sides: the tensor-core port sweep (three TF32 products per term).
Here the same subgraph shape (34^3 in 16^3 blocks: eight 17^3 / 17^2 x 16 / ... subgraphs, up to
817 ports each, 26 tile rows) runs the same kernels with the same impedance and coupling rule, and
the copies and waves after 7 and 10 sweeps (6 + 2 port sweeps and one band sweep per batch) are
compared with oracle/coupled.py iterating the paper's (u, omega) pair with the same admittance.
Tolerances: TOL_FP16 for FP16 storage, TOL_FP32 for FP32 storage and the tensor-core form.
"""
import json
import os

import numpy as np
import pytest

from oracle import coupled, evs
from paper_0807_1949_gb300 import inputs
from test_gpu_parity import _line_map, _rel
from test_precision_bounds import TOL_FP16, TOL_FP32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _model(vtmlib, family):
    from paper_0807_1949_gb300 import learned_z
    path = os.path.join(learned_z.MODELS, "z_" + family + ".json")
    with open(path) as f:
        rule = json.load(f)["coupling"]
    return learned_z.load(path), rule


def _case(vtmlib, family, sigma, seed):
    dims, block = (34, 34, 34), (16, 16, 16)
    A = inputs.grid_poisson(dims, sigma=sigma, seed=seed)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    mdl, rule = _model(vtmlib, family)
    z = vtmlib.Solver(part, z=mdl, precision="fp32", form="band").impedances() * rule["z_scale"]
    pr, w = part.line_pairs()
    y = rule["gamma"] * w
    idx = {tuple(int(v) for v in q): t for t, q in enumerate(osplit.vtl)}
    lib_to_or = np.array([idx[tuple(int(v) for v in q)] for q in part.lines()])
    zo = np.empty_like(z)
    zo[lib_to_or] = z
    Y = coupled.laplacian_admittance(osplit, zo, lib_to_or[pr], y)
    return A, part, osplit, z, (pr, y), Y


def _oracle(osplit, Y, b, ks):
    m = coupled.CoupledVTM(osplit, Y)
    st = m.initial_state(np.atleast_2d(b).shape[0])
    out = {}
    for k in range(1, max(ks) + 1):
        st = m.sweep(st, b)
        if k in ks:
            out[k] = (np.concatenate(st.x_local, axis=1), m.waves_out(st))
    return out


@pytest.mark.parametrize("storage,tol", [("fp16", TOL_FP16), ("native", TOL_FP32)])
def test_poisson3d_128_configuration(vtmlib, storage, tol):
    A, part, osplit, z, cpl, Y = _case(vtmlib, "poisson3d", 1.0, 0)
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    ref = _oracle(osplit, Y, b, (7, 10))
    s = vtmlib.Solver(part, z=z, precision="fp32", nrhs=1, form="port", port_storage=storage, coupling=cpl)
    info = s.info()
    assert info.sweep_form == 2 and info.ncouplings == len(cpl[1]) > 0
    assert info.port_storage_bits == (16 if storage == "fp16" else 32)
    lm = _line_map(part, osplit)
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    assert _rel(s.copies(), ref[7][0]) <= tol
    assert _rel(s.get_state(), ref[7][1][:, lm]) <= tol
    s.iterate(3)
    assert _rel(s.copies(), ref[10][0]) <= tol
    assert _rel(s.get_state(), ref[10][1][:, lm]) <= tol


def test_poisson3d_256_r32_configuration(vtmlib):
    """The multi-RHS run's rule (the sigma 0.75-1.75 model, sigma = 1.5) on the tensor cores."""
    A, part, osplit, z, cpl, Y = _case(vtmlib, "poisson3d-wide", 1.5, 0)
    b = inputs.rhs_uniform(A.n, 32, seed=0)
    ref = _oracle(osplit, Y, b, (7, 10))
    s = vtmlib.Solver(part, z=z, precision="fp32", nrhs=32, form="port", coupling=cpl)
    assert s.info().sweep_form == 2
    lm = _line_map(part, osplit)
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    assert _rel(s.copies(), ref[7][0]) <= TOL_FP32
    assert _rel(s.get_state(), ref[7][1][:, lm]) <= TOL_FP32
    s.iterate(3)
    assert _rel(s.copies(), ref[10][0]) <= TOL_FP32
    assert _rel(s.get_state(), ref[10][1][:, lm]) <= TOL_FP32


@pytest.mark.parametrize("nrhs", [16, 32])
def test_tensor_core_fp16_storage(vtmlib, nrhs):
    """FP16 storage on the tensor cores (the hi half of S_j / sigma_j only): within TOL_FP16 of the
    coupled oracle after 7 and 10 sweeps."""
    A, part, osplit, z, cpl, Y = _case(vtmlib, "poisson3d-wide", 1.5, 0)
    b = inputs.rhs_uniform(A.n, nrhs, seed=1)
    ref = _oracle(osplit, Y, b, (7, 10))
    s = vtmlib.Solver(part, z=z, precision="fp32", nrhs=nrhs, form="port", port_storage="fp16", coupling=cpl)
    assert s.info().port_storage_bits == 16
    lm = _line_map(part, osplit)
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    assert _rel(s.copies(), ref[7][0]) <= TOL_FP16
    assert _rel(s.get_state(), ref[7][1][:, lm]) <= TOL_FP16
    s.iterate(3)
    assert _rel(s.copies(), ref[10][0]) <= TOL_FP16
    assert _rel(s.get_state(), ref[10][1][:, lm]) <= TOL_FP16
