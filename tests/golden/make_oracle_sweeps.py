"""Write tests/golden/oracle_sweeps.json: sweeps the plain FP64 method needs to reach a relative
residual of 1e-8 on the benchmark workloads, computed by the oracle alone (oracle/, inputs).

Plain method: Z = 1 on every line, zero initial boundary variables (Table 1 step 2), relative
residual checked every 10 sweeps.  Run: python tests/golden/make_oracle_sweeps.py [workload ...]
(the 128^3 workload takes tens of minutes on one CPU core).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import evs  # noqa: E402
from oracle import vtm as ovtm  # noqa: E402
from paper_0807_1949_gb300 import inputs  # noqa: E402

WORKLOADS = {
    "poisson3d-128": dict(dims=(128, 128, 128), block=(16, 16, 16), sigma=1.0),
    "laplace2d-32": dict(dims=(32, 32), block=(16, 16), sigma=0.0),
    "poisson2d-256": dict(dims=(256, 256), block=(32, 32), sigma=1.25),
}


def main(names):
    path = os.path.join(HERE, "oracle_sweeps.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        w = WORKLOADS[name]
        t0 = time.time()
        A = inputs.grid_poisson(w["dims"], sigma=w["sigma"], seed=0)
        b = inputs.rhs_uniform(A.n, 1, seed=0)
        split = evs.split_grid(A, w["dims"], w["block"])
        t1 = time.time()
        res = ovtm.solve(split, A, b, 1.0, rtol=1e-8, maxit=100000, check_every=10)
        t2 = time.time()
        out[name] = dict(sweeps=res.sweeps, rel_residual=res.history[-1][1], z=1.0, check_every=10, rtol=1e-8,
                         seed=0, history=res.history[::10], split_seconds=round(t1 - t0, 1),
                         solve_seconds=round(t2 - t1, 1),
                         source="oracle.vtm.solve on the seeded workload (inputs.grid_poisson seed 0, "
                                "inputs.rhs_uniform seed 0), written by tests/golden/make_oracle_sweeps.py")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(name, out[name]["sweeps"], out[name]["rel_residual"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
