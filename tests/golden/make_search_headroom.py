"""Write tests/golden/search_headroom.json: how much a richer impedance search gains over the
learned part's three-parameter search family, with the FP64 oracle as the solver.

The learned impedances are trained on targets from a search over the family
log Z_t = th0 + th1 (g_t - median g) + th2 (m_t - 1) (learned_z.search).  Here, on small 2D 5-point
problems of the learned family's kind (log-normal coefficients, sigma ~ U[0.5, 2]), that search is
followed by coordinate descent with far more freedom, on the same objective (the relative residual
after K sweeps):
  face  one factor per subgraph interface (all lines joining the same two subgraphs), 24 on a
        4 x 4 split;
  line  one factor per line (per-port impedances), from the face result; only with --line.
Each descent multiplies one group's impedances by 2 or 1/2, keeps a change that lowers the
objective and repeats until nothing improves, then does the same with sqrt(2).  Every impedance set
is then judged by what the method is for: sweeps to a relative residual of 1e-8 (checked every 5
sweeps), next to Z = 1 and the best uniform Z (a scan of 22 values).  On the 64 x 64 problems both
searches are repeated on that quantity itself (family_tol, face_tol): the objective is the sweep
count to 1e-8 with the residual checked after every sweep, interpolated in log residual between
the two sweeps around 1e-8 so that it varies smoothly with Z.  §7 makes Z the preconditioner and
leaves its choice open; this measures what per-interface and per-port freedom would add to the
training targets.

With --profiled the 64 x 64 rows also get the search with its profiled walk (learned_z.search with
profile=True: th0 re-refined at every step of the th1 / th2 walks) and per-interface descent from
that result (family_profiled, face_profiled), and one fixed parameter set for all problems: the
component-wise median of the other problems' profiled parameters (global_profiled, leave one out).
With --three-d the plain and the profiled walk are compared the same way on eight 3D problems of the
kind of the 256^3 run's family (33^3 in 8^3 blocks, sigma ~ U[0.75, 1.75], horizon 60 sweeps).
With --networks the two trained 2D networks (plain-walk and profiled-walk targets) and one parameter
set of each walk are compared on eight held-out 256^2 problems of their family; with --refined as
well, the solves run FP32 factors and sweeps inside FP64 defect correction (oracle.mixed, the
structure of the library's FP32 solve) instead of the FP64 iteration.

Run: python tests/golden/make_search_headroom.py            (8 problems of 64 x 64, faces; about
                                                             30 min on 8 cores)
     python tests/golden/make_search_headroom.py --line     (5 problems of 32 x 32, faces and lines)
     python tests/golden/make_search_headroom.py --profiled (after the first; about 10 min)
     python tests/golden/make_search_headroom.py --three-d  (about 30 min on 8 cores)
     python tests/golden/make_search_headroom.py --networks (about 5 min on 8 cores)
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def problem(n: int, blk: int, seed: int, dim: int = 2):
    """The seeded problem: 2D with sigma drawn as in the learned 2D family, or 3D (n^3, blocks of
    blk^3) with sigma ~ U[0.75, 1.75] as in the family of the 256^3 run; coefficients and b from
    inputs."""
    from oracle import evs
    from paper_0807_1949_gb300 import inputs

    lo, hi = (0.5, 2.0) if dim == 2 else (0.75, 1.75)
    sigma = float(np.random.default_rng(10_000 + seed).uniform(lo, hi))
    A = inputs.grid_poisson((n,) * dim, sigma=sigma, seed=seed)
    b = inputs.rhs_uniform(A.n, 1, seed=seed)
    return A, evs.split_grid(A, (n,) * dim, (blk,) * dim), b, sigma


def run_3d(args) -> dict:
    """3D: the plain and the profiled walk of the family search, judged by sweeps to 1e-8."""
    n, blk, seed, K = args
    from paper_0807_1949_gb300 import learned_z

    A, split, b, sigma = problem(n, blk, seed, dim=3)
    ev = OracleSolves(A, split, b, K)
    L = ev.lines
    th, log = learned_z.search(ev, sweeps=K)
    tp, logp = learned_z.search(ev, sweeps=K, profile=True)
    return dict(n=n, block=blk, seed=seed, sigma=round(sigma, 4), horizon=K, lines=L,
                theta=[round(v, 4) for v in th], theta_profiled=[round(v, 4) for v in tp],
                evals=len(log), profiled_evals=len(logp),
                objective=dict(family=ev.residual_after(learned_z.family_z(ev.feats, th)),
                               family_profiled=ev.residual_after(learned_z.family_z(ev.feats, tp))),
                sweeps=dict(z1=ev.to_tolerance(np.ones(L)), family=ev.to_tolerance(learned_z.family_z(ev.feats, th)),
                            family_profiled=ev.to_tolerance(learned_z.family_z(ev.feats, tp))))


def run_global3(args) -> int:
    n, blk, seed, theta = args
    from paper_0807_1949_gb300 import learned_z

    A, split, b, _ = problem(n, blk, seed, dim=3)
    ev = OracleSolves(A, split, b, 0)
    return ev.to_tolerance(learned_z.family_z(ev.feats, theta))


class OracleSolves:
    """The FP64 oracle iterated for a per-line impedance vector (objective cached by its value)."""

    def __init__(self, A, split, b, horizon: int):
        from oracle import features

        self.A, self.split, self.b, self.K = A, split, b, horizon
        self.feats = features.line_features(split, A).astype(np.float32)
        self.lines = len(split.vtl)
        self.cache = {}

    def residual_after(self, z, sweeps: int | None = None) -> float:
        from oracle import vtm as ovtm

        z = np.broadcast_to(np.asarray(z, dtype=np.float64), (self.lines,)).copy()
        K = self.K if sweeps is None else sweeps
        key = (K, np.round(np.log(z), 6).tobytes())
        if key not in self.cache:
            m = ovtm.VTM(self.split, z)
            st = m.initial_state()
            for _ in range(K):
                st = m.sweep(st, self.b)
            r = float(ovtm.relative_residual(self.A, self.b, m.assemble(st))[0])
            self.cache[key] = r if math.isfinite(r) else 1e30
        return self.cache[key]

    def fractional_sweeps(self, z, rtol: float = 1e-8, maxit: int = 6000) -> float:
        """Sweeps to reach rtol, interpolated in log residual between the two sweeps around it
        (the residual is checked after every sweep), so that the count varies smoothly with z."""
        from oracle import vtm as ovtm

        z = np.broadcast_to(np.asarray(z, dtype=np.float64), (self.lines,)).copy()
        key = ("tol", np.round(np.log(z), 6).tobytes())
        if key not in self.cache:
            m = ovtm.VTM(self.split, z)
            st = m.initial_state()
            prev, val = 1.0, float(maxit)
            for k in range(1, maxit + 1):
                st = m.sweep(st, self.b)
                r = float(ovtm.relative_residual(self.A, self.b, m.assemble(st))[0])
                if not math.isfinite(r):
                    break
                if r <= rtol:
                    val = k - 1 + (math.log(prev / rtol) / math.log(prev / r) if prev > r else 1.0)
                    break
                prev = r
            self.cache[key] = val
        return self.cache[key]

    def to_tolerance(self, z, rtol: float = 1e-8, maxit: int = 6000, every: int = 5) -> int:
        from oracle import vtm as ovtm

        m = ovtm.VTM(self.split, np.broadcast_to(np.asarray(z, dtype=np.float64), (self.lines,)).copy())
        st = m.initial_state()
        for k in range(1, maxit + 1):
            st = m.sweep(st, self.b)
            if k % every == 0 and ovtm.relative_residual(self.A, self.b, m.assemble(st))[0] <= rtol:
                return k
        return maxit


def interfaces(split) -> list[list[int]]:
    """Lines grouped by the unordered pair of subgraphs they join."""
    groups = {}
    for t, (ja, _, jb, _) in enumerate(split.vtl):
        groups.setdefault((min(int(ja), int(jb)), max(int(ja), int(jb))), []).append(t)
    return [groups[k] for k in sorted(groups)]


def descend(objective, z: np.ndarray, groups, steps=(2.0, math.sqrt(2.0))):
    """Coordinate descent of objective(z) over multiplicative factors of the groups' impedances."""
    z = z.copy()
    best = objective(z)
    evals = 0
    for step in steps:
        improved = True
        while improved:
            improved = False
            for idx in groups:
                for f in (step, 1.0 / step):
                    zt = z.copy()
                    zt[idx] *= f
                    r = objective(zt)
                    evals += 1
                    if r < best:
                        best, z, improved = r, zt, True
                        break
    return z, best, evals


def run(args) -> dict:
    n, blk, seed, K, per_line, true_objective = args
    from paper_0807_1949_gb300 import learned_z

    A, split, b, sigma = problem(n, blk, seed)
    ev = OracleSolves(A, split, b, K)
    L = ev.lines
    zs = np.exp(np.linspace(np.log(0.25), np.log(32.0), 22))
    ru = [ev.residual_after(np.full(L, z)) for z in zs]
    z_uni = float(zs[int(np.argmin(ru))])
    theta, _ = learned_z.search(ev, sweeps=K)
    z_fam = learned_z.family_z(ev.feats, theta)
    groups = interfaces(split)
    z_face, r_face, n_face = descend(ev.residual_after, z_fam, groups)
    out = dict(n=n, block=blk, seed=seed, sigma=round(sigma, 4), horizon=K, lines=L, interfaces=len(groups),
               z_uniform=round(z_uni, 4), theta=[round(v, 4) for v in theta],
               objective=dict(uniform=min(ru), family=ev.residual_after(z_fam), face=r_face),
               face_evals=n_face,
               sweeps=dict(z1=ev.to_tolerance(np.ones(L)), uniform=ev.to_tolerance(np.full(L, z_uni)),
                           family=ev.to_tolerance(z_fam), face=ev.to_tolerance(z_face)))
    if true_objective:
        # the same two searches on the quantity the impedances are for: sweeps to 1e-8
        class _Tol:
            feats = ev.feats

            @staticmethod
            def residual_after(z, sweeps):
                return ev.fractional_sweeps(z)

        theta_t, _ = learned_z.search(_Tol, sweeps=K)
        z_ft = learned_z.family_z(ev.feats, theta_t)
        z_gt, s_gt, n_gt = descend(ev.fractional_sweeps, z_ft, groups)
        out["theta_tol"] = [round(v, 4) for v in theta_t]
        out["fractional_sweeps"] = dict(family=ev.fractional_sweeps(z_fam), face=ev.fractional_sweeps(z_face),
                                        family_tol=ev.fractional_sweeps(z_ft), face_tol=s_gt)
        out["face_tol_evals"] = n_gt
        out["sweeps"].update(family_tol=ev.to_tolerance(z_ft), face_tol=ev.to_tolerance(z_gt))
    if per_line:
        z_line, r_line, n_line = descend(ev.residual_after, z_face, [[t] for t in range(L)])
        out["objective"]["line"] = r_line
        out["line_evals"] = n_line
        out["sweeps"]["line"] = ev.to_tolerance(z_line)
        out["line_log_spread"] = round(float(np.std(np.log(z_line / z_face))), 4)
    return out


def run_profiled(args) -> dict:
    """The profiled search (th0 re-refined at every walk step) and per-interface descent from it."""
    n, blk, seed, K = args
    from paper_0807_1949_gb300 import learned_z

    A, split, b, _ = problem(n, blk, seed)
    ev = OracleSolves(A, split, b, K)
    theta, log = learned_z.search(ev, sweeps=K, profile=True)
    z_p = learned_z.family_z(ev.feats, theta)
    z_pf, r_pf, n_pf = descend(ev.residual_after, z_p, interfaces(split))
    return dict(seed=seed, theta_profiled=[round(v, 4) for v in theta], profiled_evals=len(log),
                profiled_face_evals=n_pf, objective=dict(family_profiled=ev.residual_after(z_p), face_profiled=r_pf),
                sweeps=dict(family_profiled=ev.to_tolerance(z_p), face_profiled=ev.to_tolerance(z_pf)))


def run_global(args) -> int:
    """Sweeps to 1e-8 of one fixed parameter set of the family on one problem."""
    n, blk, seed, theta = args
    from paper_0807_1949_gb300 import learned_z

    A, split, b, _ = problem(n, blk, seed)
    ev = OracleSolves(A, split, b, 0)
    return ev.to_tolerance(learned_z.family_z(ev.feats, theta))


def run_networks(args) -> dict:
    """256^2 (the 2D family's own size): sweeps to 1e-8 of the two trained networks (their forward
    pass taken by the oracle's FP64 perceptron on the BF16-rounded weights; both ends of a line
    agree on the geometric mean) and of one parameter set of each walk (the median of the model
    file's training-set parameters), all with the FP64 oracle as the solver."""
    seed, models, refined = args
    from oracle import evs, mixed, mlp
    from paper_0807_1949_gb300 import learned_z

    A, dims, block, sigma, b = learned_z.problem("poisson2d-256", seed)
    split = evs.split_grid(A, dims, block)
    ev = OracleSolves(A, split, b, 0)
    if refined:
        # FP32 factors and sweeps inside FP64 defect correction (oracle.mixed), checked every 10
        def sweeps(z):
            return mixed.solve_refined(split, A, b, z, kind="fp32", rtol=1e-8, maxit=6000, check_every=10).sweeps
    else:
        sweeps = ev.to_tolerance
    row = dict(seed=seed, sigma=round(sigma, 4), lines=ev.lines, sweeps={})
    for name, (params, theta) in models.items():
        y, _ = mlp.forward(mlp.bf16_round(params), ev.feats.astype(np.float64))
        z_net = np.exp(np.clip(0.5 * (y[0::2] + y[1::2]), -30.0, 30.0))
        row["sweeps"][name + "_network"] = sweeps(z_net)
        row["sweeps"][name + "_one_theta"] = sweeps(learned_z.family_z(ev.feats, theta))
    return row


def summary(rows, keys) -> dict:
    fam = np.array([r["sweeps"]["family"] for r in rows], dtype=float)
    s = {"median_sweeps": {k: float(np.median([r["sweeps"][k] for r in rows])) for k in keys}}
    s["median_sweep_ratio_to_family"] = {k: round(float(np.median(np.array([r["sweeps"][k] for r in rows]) / fam)), 4)
                                         for k in keys if k != "family"}
    s["min_sweep_ratio_to_family"] = {k: round(float(np.min(np.array([r["sweeps"][k] for r in rows]) / fam)), 4)
                                      for k in keys if k != "family"}
    s["median_objective_gain_over_family"] = {
        k: round(float(np.median([r["objective"]["family"] / r["objective"][k] for r in rows])), 3)
        for k in keys if k in rows[0]["objective"] and k != "family"}
    return s


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--line", action="store_true", help="also descend per line (32 x 32, 8^2 blocks)")
    ap.add_argument("--profiled", action="store_true",
                    help="add the profiled search and per-interface descent from it to the stored 64 x 64 rows")
    ap.add_argument("--networks", action="store_true",
                    help="the two trained 2D networks against one parameter set of each walk, on 8 held-out "
                         "256^2 problems")
    ap.add_argument("--refined", action="store_true",
                    help="with --networks: FP32 sweeps inside FP64 defect correction (oracle.mixed) instead of FP64")
    ap.add_argument("--three-d", action="store_true",
                    help="plain against profiled walk on eight 3D problems (33^3 in 8^3 blocks, 64 subgraphs)")
    ap.add_argument("--procs", type=int, default=min(8, os.cpu_count() or 1))
    a = ap.parse_args()
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    path = os.path.join(HERE, "search_headroom.json")
    if a.networks:
        from paper_0807_1949_gb300 import learned_z

        models = {}
        for name, fname in (("plain", "z_poisson2d-256.json"), ("profiled", "z_poisson2d-256-profiled.json")):
            with open(os.path.join(learned_z.MODELS, fname)) as f:
                m = json.load(f)
            th = np.median(np.array([list(r["theta"]) + [0.0] * (4 - len(r["theta"])) for r in m["search"]]), axis=0)
            models[name] = (np.asarray(m["params"], dtype=np.float64), tuple(float(v) for v in th))
        jobs = [(sd, models, a.refined) for sd in range(100_000, 100_008)]
        with mp.get_context("spawn").Pool(min(a.procs, len(jobs))) as pool:
            rows = pool.map(run_networks, jobs)
        keys = ("plain_network", "plain_one_theta", "profiled_network", "profiled_one_theta")
        med = {k: float(np.median([r["sweeps"][k] for r in rows])) for k in keys}
        out = json.load(open(path)) if os.path.exists(path) else {}
        out["networks256_fp32" if a.refined else "networks256"] = dict(rows=rows, theta={k: [round(v, 4) for v in t] for k, (_, t) in models.items()},
                                  median_sweeps=med)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(json.dumps(med, indent=1))
        return
    if a.three_d:
        jobs = [(33, 8, s, 60) for s in range(1, 9)]
        with mp.get_context("spawn").Pool(min(a.procs, len(jobs))) as pool:
            rows = sorted(pool.map(run_3d, jobs), key=lambda r: r["seed"])
            th = np.array([r["theta_profiled"] for r in rows])
            glob = [tuple(float(v) for v in np.median(np.delete(th, i, axis=0), axis=0)) for i in range(len(rows))]
            sw = pool.map(run_global3, [(r["n"], r["block"], r["seed"], g) for r, g in zip(rows, glob)])
        for r, g, k in zip(rows, glob, sw):
            r["theta_global_profiled"] = [round(v, 4) for v in g]
            r["sweeps"]["global_profiled"] = k
        out = json.load(open(path)) if os.path.exists(path) else {}
        out["profiled3d"] = dict(rows=rows, summary=summary(rows, ("z1", "family", "family_profiled", "global_profiled")))
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(json.dumps(out["profiled3d"]["summary"], indent=1))
        return
    if a.profiled:
        out = json.load(open(path))
        rows = out["face64"]["rows"]
        with mp.get_context("spawn").Pool(min(a.procs, len(rows))) as pool:
            extra = pool.map(run_profiled, [(r["n"], r["block"], r["seed"], r["horizon"]) for r in rows])
            for r, e in zip(rows, extra):
                assert r["seed"] == e["seed"]
                r["theta_profiled"], r["profiled_evals"] = e["theta_profiled"], e["profiled_evals"]
                r["profiled_face_evals"] = e["profiled_face_evals"]
                r["objective"].update(e["objective"])
                r["sweeps"].update(e["sweeps"])
            # one fixed parameter set for every problem: the component-wise median of the other
            # problems' profiled parameters (leave one out), i.e. the method without a network
            th = np.array([r["theta_profiled"] for r in rows])
            glob = [tuple(float(v) for v in np.median(np.delete(th, i, axis=0), axis=0)) for i in range(len(rows))]
            sw = pool.map(run_global, [(r["n"], r["block"], r["seed"], g) for r, g in zip(rows, glob)])
        for r, g, k in zip(rows, glob, sw):
            r["theta_global_profiled"] = [round(v, 4) for v in g]
            r["sweeps"]["global_profiled"] = k
        keys = ("z1", "uniform", "family", "face", "family_tol", "face_tol", "family_profiled", "face_profiled",
                "global_profiled")
        out["face64"]["summary"] = summary(rows, keys)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(json.dumps(out["face64"]["summary"], indent=1))
        return
    if a.line:
        name, jobs, keys = "line32", [(32, 8, s, 50, True, False) for s in range(1, 6)], \
            ("z1", "uniform", "family", "face", "line")
    else:
        name, jobs, keys = "face64", [(64, 16, s, 100, False, True) for s in range(1, 9)], \
            ("z1", "uniform", "family", "face", "family_tol", "face_tol")
    with mp.get_context("spawn").Pool(min(a.procs, len(jobs))) as pool:
        rows = sorted(pool.map(run, jobs), key=lambda r: r["seed"])
    out = json.load(open(path)) if os.path.exists(path) else {}
    out[name] = dict(rows=rows, summary=summary(rows, keys))
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out[name]["summary"], indent=1))


if __name__ == "__main__":
    main()
