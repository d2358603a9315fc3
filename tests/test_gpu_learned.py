"""What the trained impedance network gains over the method without it (GPU).

The committed 2D model (paper_0807_1949_gb300/models/z_poisson2d-256.json, trained on searched
impedances of 800 seeded problems) is applied to problems it has not seen; the learned impedances
must reach the tolerance in far fewer sweeps than Z = 1 and than the paper's matching rule (§7.1).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0807_1949_gb300 import learned_z  # noqa: E402  (loads the library; GPU runs only)


@pytest.mark.parametrize("seed", [200_001, 200_002])
def test_learned_impedances_beat_z1_and_matching(vtmlib, seed):
    import os
    model = learned_z.load(os.path.join(learned_z.MODELS, "z_poisson2d-256.json"))
    A, dims, block, sigma, b = learned_z.problem("poisson2d-256", seed)
    ev = learned_z.Evaluator(A, dims, block, b)
    z1 = ev.to_tolerance(1.0)
    lz = ev.to_tolerance(model)
    mz = ev.to_tolerance("matched")
    assert z1["converged"] and lz["converged"] and mz["converged"]
    assert lz["sweeps"] < 0.4 * z1["sweeps"], (lz, z1)
    assert lz["sweeps"] < 0.4 * mz["sweeps"], (lz, mz)
    x = ev.x.cpu().numpy()  # the last solve was the matched one; residual of the returned iterate
    r = np.linalg.norm(b - (A.to_scipy() @ x.T).T) / np.linalg.norm(b)
    assert r <= 1e-8
