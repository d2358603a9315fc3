#!/usr/bin/env python
"""Benchmark: time to relative residual 1e-8 of the Virtual Transmission Method on one GB300.

Workload (default "poisson3d-256-r32"): 3D 7-point variable-coefficient Poisson operator on a 256^3
vertex grid (16,777,216 unknowns), node coefficients log-normal (sigma = 1.5, seed 0), Dirichlet
boundary; Electric Vertex Splitting into 16x16x16 = 4096 cubic subgraphs (cut planes every 16
nodes, shared); 32 right-hand sides i.i.d. uniform[-1, 1] solved together.  Line impedances from
the learned model (models/z_poisson3d-wide.json) with coupled lines (§7.2): every line scaled by the
model's z_scale and every candidate pair of lines of a bundle joined by the conductance
gamma |a_ik| (rule selected on held-out seeds, stored with the model).  The product path uses FP32
factors and FP32 sweeps inside FP64 defect correction (residual b - A x in FP64 on the device), in
port-response form: the port responses S_j (lower block triangle, fp16 hi/lo pairs) multiply the
32 port vectors on the tensor cores.  The plain method (FP64 factors and band sweeps every sweep,
Z = 1, no coupling, no correction, one right-hand side) is timed beside it on the same GPU.

One step = one vtm_solve from zero waves to max relative residual <= 1e-8 over all right-hand sides
(every sweep gathers the twins' waves, forms the port right-hand sides including the coupling
currents, updates the ports through S_j (the last sweep of each batch through the band factors)
and emits the outgoing waves; the FP64 residual is checked every 20 sweeps or as the observed rate
predicts).  vtm_setup (factorisation, port responses) happens once, before the timed region; it is
reported as setup_ms and added in value_with_setup.  The port responses (19 GB) and factors
(24 GB) are far larger than L2, so no flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vtm|reference] [--workload W]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the benchmarked configuration: 3D 128^3, sigma = 1, 512 subgraphs, one right-hand side
    "poisson3d-128": dict(kind="grid", dims=(128, 128, 128), block=(16, 16, 16), sigma=1.0, nrhs=1,
                          z="learned:poisson3d", coupling="model", rtol=1e-8),
    # large multi-RHS run: 256^3, sigma = 1.5, 4096 subgraphs, 32 right-hand sides per sweep
    "poisson3d-256-r32": dict(kind="grid", dims=(256, 256, 256), block=(16, 16, 16), sigma=1.5, nrhs=32,
                              z="learned:poisson3d-wide", coupling="model", rtol=1e-8),
    # mid-size multi-RHS case of the same family (512 subgraphs)
    "poisson3d-128-r32": dict(kind="grid", dims=(128, 128, 128), block=(16, 16, 16), sigma=1.5, nrhs=32,
                              z="learned:poisson3d-wide", coupling="model", rtol=1e-8),
    # small case of the multi-RHS kernel for profiler captures: 96^3 in 12^3 blocks (512 subgraphs of
    # 866 ports, 0.9 GB of port responses > L2, about 3.5 GB on the device)
    "poisson3d-96b12-r32": dict(kind="grid", dims=(96, 96, 96), block=(12, 12, 12), sigma=1.5, nrhs=32,
                                z="learned:poisson3d-wide", coupling="model", rtol=1e-8),
    # uneven batching: P1 FEM on the Delaunay triangulation of 1M points, 2000 RCB subgraphs, 16 RHS.
    # The one-level method does not reach 1e-8 here in any practical number of sweeps (contrast 1e6),
    # so a step is a fixed number of sweeps and the line reports the residual it reaches.
    "fem2d-1m-r16": dict(kind="fem", npoints=1_000_000, pieces=2000, nrhs=16, z="scaled:2", plain_z="scaled:2",
                         rtol=1e-8, sweeps=1000),
    # learned-impedance family: 2D 256^2, 64 subgraphs
    "poisson2d-256": dict(kind="grid", dims=(256, 256), block=(32, 32), sigma=1.25, nrhs=1,
                          z="learned:poisson2d-256", coupling="model", rtol=1e-8),
    "laplace2d-32": dict(kind="grid", dims=(32, 32), block=(16, 16), sigma=0.0, nrhs=1, z=1.0, rtol=1e-8),
    # small case of the 3D subgraph shape (64 subgraphs, 0.37 GB factor > L2) for ncu captures
    "poisson3d-64": dict(kind="grid", dims=(64, 64, 64), block=(16, 16, 16), sigma=1.0, nrhs=1, z=1.0, rtol=1e-8),
    # the same with 32 right-hand sides (tensor-core port form; 0.5 GB of port responses > L2)
    "poisson3d-64-r32": dict(kind="grid", dims=(64, 64, 64), block=(16, 16, 16), sigma=1.0, nrhs=32, z=1.0,
                             rtol=1e-8),
}
METRIC = "time to rel. residual 1e-8 (learned-Z batched vs plain VTM) on 1 GB300; HBM GB/s"
FP64_TFLOPS = 1.25  # nominal FP64 rate of a GB300 (non-tensor), the bound of the plain FP64 band sweep


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="vtm", choices=["vtm", "reference"])
    p.add_argument("--workload", default="poisson3d-256-r32", choices=list(WORKLOADS))
    p.add_argument("--check-every", type=int, default=20,
                   help="sweeps between FP64 residual checks (a port-form batch ends with one band sweep)")
    p.add_argument("--inner-reduction", type=float, default=0.0,
                   help="FP32 defect correction: restart once the inner residual has dropped by this factor "
                        "(0: the library's default)")
    p.add_argument("--form", default="auto", choices=["auto", "band", "port"])
    p.add_argument("--port-storage", default="fp16-auto", choices=["native", "fp16", "fp16-auto"],
                   help="port form, nrhs <= 8: storage of the port responses")
    p.add_argument("--z", default=None, help="impedance rule overriding the workload's (a number, "
                   "learned:<family> or scaled:<c>)")
    p.add_argument("--coupling", default=None,
                   help="coupled lines (§7.2): 'none', 'model' (the rule stored with the learned model) or a "
                        "conductance factor gamma (y_p = gamma |a_ik|); default: the workload's")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--record-plain", action="store_true",
                   help="write the plain method's sweep count to profiles/plain_sweeps.json")
    return p.parse_args()


# ----------------------------------------------------------------------------- CPU oracle timing
#
# The FP64 oracle (oracle.vtm, as it stands) runs on a bounded sample of the workload: a grid of
# nb^d blocks of exactly the workload's block shape (every subgraph has the workload's size and
# bandwidth), with the workload's number of right-hand sides.  Its subgraphs are spread over one
# worker process per host core (spawned; BLAS limited to one thread each), which call the oracle's
# own Table 1 step (VTM.piece_step) on their subgraphs and exchange the boundary pairs (u, omega)
# through shared memory, so that the time per sweep is the oracle's on all cores.  The sample also
# times the oracle's residual check (assembly and FP64 b - A x, every 10 sweeps as in the plain
# method).  Time to tolerance = (sweep + check / 10) x sweeps to tolerance, scaled from the sample's
# subgraphs to the workload's; the factorisation is excluded (paid once, like vtm_setup).

_OW = {}


def _ow_main(conn, dims, block, sigma, nrhs, pieces, shm_names, shapes, coff):
    """Worker: the oracle's split of the sample, factors of its own subgraphs, then sweeps on request."""
    import numpy as np
    from multiprocessing import shared_memory

    from oracle import evs
    from oracle import vtm as ovtm
    from paper_0807_1949_gb300 import inputs

    A = inputs.grid_poisson(dims, sigma=sigma, seed=0)
    split = evs.split_grid(A, dims, block)
    m = ovtm.VTM(split, 1.0, pieces=pieces)
    b = inputs.rhs_uniform(A.n, nrhs, seed=0)
    shm = {k: shared_memory.SharedMemory(name=n) for k, n in shm_names.items()}
    arr = {k: np.ndarray(shapes[k], dtype=np.float64, buffer=shm[k].buf) for k in shm}
    import time as _time
    spent = {j: [] for j in pieces}   # seconds of each subgraph's step, one entry per sweep since the last report
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            break
        if msg == "times":
            # median of single steps: a stall of the host during one sweep moves no subgraph's time
            conn.send({j: (float(np.median(v)) if v else 0.0) for j, v in spent.items()})
            spent = {j: [] for j in pieces}
            continue
        cur = msg
        u, om = arr["u%d" % cur], arr["o%d" % cur]
        nu, no = arr["u%d" % (cur ^ 1)], arr["o%d" % (cur ^ 1)]
        for j in pieces:
            t0 = _time.perf_counter()
            x = m.piece_step(j, u, om, b, nu, no)
            spent[j].append(_time.perf_counter() - t0)
            arr["x"][:, coff[j]:coff[j + 1]] = x
        conn.send("done")
    for v in shm.values():
        v.close()


class OracleSampler:
    """The FP64 oracle on all host cores over a bounded sample of a workload (see above): the
    workers, the sample's split and its factors are made once; each time() call times sweeps and
    one residual check of the running iteration."""

    def __init__(self, workload: str, cores: int | None = None, nb: int | None = None):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        import numpy as np

        from oracle import evs
        from paper_0807_1949_gb300 import inputs

        self.workload = workload
        w = self.w = WORKLOADS[workload]
        d = len(w["dims"])
        if nb is None:
            nb = 4 if d == 3 else 8                 # 64 subgraphs
        dims = self.dims = tuple(min(n, nb * s + 1) for n, s in zip(w["dims"], w["block"]))
        R = self.R = w["nrhs"]
        self.A = inputs.grid_poisson(dims, sigma=w["sigma"], seed=0)
        self.b = inputs.rhs_uniform(self.A.n, R, seed=0)
        split = self.split = evs.split_grid(self.A, dims, w["block"])
        P = self.P = len(split.subgraphs)
        E = 2 * len(split.vtl)
        sizes = [len(g.vertices) for g in split.subgraphs]
        self.coff = coff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        if cores is None:
            cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        self.cores = cores = max(1, min(cores, P))
        shapes = {"u0": (R, E), "o0": (R, E), "u1": (R, E), "o1": (R, E), "x": (R, int(coff[-1]))}
        self.shm, self.procs, self.conns = {}, [], []
        self.cur, self.warm = 0, False
        env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env_keep:
            os.environ[k] = "1"
        try:
            for k, v in shapes.items():              # one at a time, so that close() frees every one made
                self.shm[k] = shared_memory.SharedMemory(create=True, size=max(8, int(np.prod(v)) * 8))
            self.arr = {k: np.ndarray(shapes[k], dtype=np.float64, buffer=self.shm[k].buf) for k in self.shm}
            for v in self.arr.values():
                v[...] = 0.0
            ctx = mp.get_context("spawn")
            for c in range(cores):
                mine = list(range(c, P, cores))
                pa, pb = ctx.Pipe()
                pr = ctx.Process(target=_ow_main, args=(pb, dims, w["block"], w["sigma"], R, mine,
                                                        {k: v.name for k, v in self.shm.items()}, shapes, coff))
                pr.start()
                self.procs.append(pr)
                self.conns.append(pa)
            for cn in self.conns:
                assert cn.recv() == "ready"
        except BaseException:
            self.close()
            raise
        finally:
            for k, v in env_keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def _sweep(self):
        for cn in self.conns:
            cn.send(self.cur)
        for cn in self.conns:
            assert cn.recv() == "done"
        self.cur ^= 1

    def time(self, sweeps: int) -> dict:
        """Seconds per sweep (median of single sweeps) and per residual check, and the work ratio of
        the workload to the sample (by class of subgraph)."""
        import numpy as np

        from oracle import vtm as ovtm

        if not self.warm:
            self._sweep()                            # warm-up
            self.warm = True
        for cn in self.conns:                        # reset the per-subgraph clocks
            cn.send("times")
            cn.recv()
        per = []
        for _ in range(sweeps):                      # median of single sweeps: robust to a stray stall
            t0 = time.perf_counter()
            self._sweep()
            per.append(time.perf_counter() - t0)
        t_sweep = float(np.median(per))
        spent = {}
        for cn in self.conns:
            cn.send("times")
            spent.update(cn.recv())
        t0 = time.perf_counter()
        arr, coff, cur = self.arr, self.coff, self.cur
        st = ovtm.State(u=arr["u%d" % cur], omega=arr["o%d" % cur],
                        x_local=[arr["x"][:, coff[j]:coff[j + 1]] for j in range(self.P)])
        x = ovtm.assemble(self.split, st)
        rr = ovtm.relative_residual(self.A, self.b, x)
        t_check = time.perf_counter() - t0
        assert np.all(np.isfinite(rr))
        w, dims = self.w, self.dims
        nbw = [max(1, -(-(n - 1) // s)) if n > 1 else 1 for n, s in zip(w["dims"], w["block"])]
        nbs = [max(1, -(-(n - 1) // s)) if n > 1 else 1 for n, s in zip(dims, w["block"])]
        total = int(np.prod(nbw))

        # The work of a subgraph grows with its ports, i.e. with the number of block faces it shares
        # with neighbours; a small sample has more boundary subgraphs than the workload.  Scale the
        # sample's time by the workload's work over the sample's, with the step time of each class
        # measured in the sample (classes by neighbour count; a missing class from a linear fit in
        # that count).
        def faces(idx, nb):
            return sum((i > 0) + (i < m - 1) for i, m in zip(idx, nb))

        def class_counts(nb):
            cnt = {}
            for idx in np.ndindex(*nb):
                k = faces(idx, nb)
                cnt[k] = cnt.get(k, 0) + 1
            return cnt

        blk = np.array(w["block"])
        per_class = {}
        for j, g in enumerate(self.split.subgraphs):
            coord = np.array(np.unravel_index(int(np.min(g.vertices)), dims))
            idx = tuple(int(v) for v in np.minimum(coord // blk, np.array(nbs) - 1))
            per_class.setdefault(faces(idx, nbs), []).append(spent.get(j, 0.0))
        mean = {k: float(np.mean(v)) for k, v in per_class.items()}
        ks = sorted(mean)
        if len(ks) >= 2:
            slope, icpt = np.polyfit(ks, [mean[k] for k in ks], 1)
        else:
            slope, icpt = 0.0, (mean[ks[0]] if ks else 1.0)

        def cost(k):
            return mean[k] if k in mean else max(icpt + slope * k, 1e-12)

        work = lambda cnt: sum(c * cost(k) for k, c in cnt.items())
        ratio = work(class_counts(nbw)) / max(work(class_counts(nbs)), 1e-30)
        return dict(t_sweep=t_sweep, t_check=t_check, sample_pieces=self.P, total_pieces=total, sample_dims=dims,
                    sweeps=sweeps, cores=self.cores, nrhs=self.R, work_ratio=ratio,
                    n_ratio=float(np.prod(w["dims"])) / float(np.prod(dims)))

    def close(self):
        for cn in self.conns:
            try:
                cn.send(None)
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
        for v in self.shm.values():
            v.close()
            v.unlink()
        self.conns, self.procs, self.shm = [], [], {}


def oracle_timing(workload: str, sweeps: int = 4, cores: int | None = None, nb: int | None = None) -> dict:
    """Seconds per sweep and per residual check of the FP64 oracle on all host cores (see above),
    from a sampler made for this one measurement."""
    smp = OracleSampler(workload, cores, nb)
    try:
        return smp.time(sweeps)
    finally:
        smp.close()


def oracle_time_to_tol(t: dict, sweeps_to_tol: int, check_every: int = 10) -> float:
    """Milliseconds the oracle needs for sweeps_to_tol sweeps with a check every check_every, scaled
    from the sample to the workload: sweeps by the work ratio of the subgraph classes, checks
    (assembly and residual, linear in the unknowns) by the ratio of unknowns."""
    per = t["t_sweep"] * t["work_ratio"] + t["t_check"] * t["n_ratio"] / check_every
    return per * sweeps_to_tol * 1e3


def cpu_baseline(workload: str, sweeps_to_tol: int, count_source: str, sweeps: int = 4) -> dict:
    try:
        t = oracle_timing(workload, sweeps)
    except Exception as e:  # noqa: BLE001 - reported, not fatal to the GPU measurement
        return dict(value=None, unit="ms", cores=None, kind="oracle", error=str(e)[-300:])
    v = oracle_time_to_tol(t, sweeps_to_tol)
    return dict(value=round(v, 1), unit="ms", cores=t["cores"], kind="oracle",
                per_sweep_ms=round((t["t_sweep"] * t["work_ratio"] + t["t_check"] * t["n_ratio"] / 10) * 1e3, 1),
                sample=(f"FP64 oracle (oracle.vtm, Table 1 step per subgraph) on {t['cores']} host cores: "
                        f"{t['sweeps']} sweeps and one residual check of a {list(t['sample_dims'])} grid = "
                        f"{t['sample_pieces']} subgraphs of the workload's block shape, {t['nrhs']} right-hand "
                        f"sides ({t['t_sweep']:.2f} s per sweep, {t['t_check']:.2f} s per check), scaled to "
                        f"{t['total_pieces']} subgraphs (by the measured step time of each class of subgraph: "
                        f"work ratio {t['work_ratio']:.1f}) and {sweeps_to_tol} sweeps ({count_source}), a "
                        f"check every 10 sweeps (scaled by the unknowns); factorisation excluded"))


# ----------------------------------------------------------------------------- clocks


class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_traffic(kernel_src: str, workload: str, kname: str):
    """Measured DRAM bytes per sweep launch from a committed ncu summary, if it is current (same
    kernel source, same kernel variant)."""
    path = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        with open(kernel_src, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
        for e in d.get(workload, []):
            if e.get("kernel_sha") == h and e.get("kernel") == kname:
                return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl == "vtm" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    """Largest value over the ranks (the slowest replica sets the time)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- arms


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    ksweeps, ksrc = reference_sweeps(args.workload)
    if ksweeps <= 0:
        print(json.dumps({"impl": "reference", "unavailable": "no recorded sweep count of the plain method for "
                          + args.workload}))
        return 0
    t0 = time.perf_counter()
    smp = OracleSampler(args.workload)      # workers, split and factors once (factorisation excluded)
    t_make = time.perf_counter() - t0
    vals, t = [], None
    try:
        for _ in range(args.warmup):
            smp.time(1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            t = smp.time(2)
            vals.append(oracle_time_to_tol(t, ksweeps))
        dt = time.perf_counter() - t0
    finally:
        smp.close()
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "dims": w["dims"], "block": w["block"], "sigma": w["sigma"],
                   "nrhs": w["nrhs"], "rtol": w["rtol"], "z": 1.0, "sweeps_to_tol": ksweeps,
                   "sweeps_source": ksrc},
        "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": t["cores"], "kind": "oracle",
                         "sample": (f"each step: FP64 oracle on {t['cores']} host cores, {t['sweeps']} sweeps and one "
                                    f"residual check of a {list(t['sample_dims'])} grid ({t['sample_pieces']} "
                                    f"subgraphs of the workload's block shape, {t['nrhs']} right-hand sides), scaled "
                                    f"to {t['total_pieces']} subgraphs and {ksweeps} sweeps ({ksrc}); wall "
                                    f"{dt:.1f} s for {args.steps} steps, after {t_make:.1f} s to split and "
                                    f"factor the sample once")},
        "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def reference_sweeps(workload: str):
    """Sweeps the plain FP64 method (Z = 1, FP64 band sweeps, one right-hand side) needs to reach
    1e-8: the oracle's own count where it has run to tolerance (tests/golden/oracle_sweeps.json),
    else the count this bench's plain arm recorded on the GPU (profiles/plain_sweeps.json)."""
    for path, src in ((os.path.join(ROOT, "tests", "golden", "oracle_sweeps.json"), "the FP64 oracle's own run"),
                      (os.path.join(ROOT, "profiles", "plain_sweeps.json"), "the plain FP64 method on the GPU")):
        try:
            with open(path) as f:
                return int(json.load(f)[workload]["sweeps"]), src
        except Exception:
            continue
    return -1, ""


def build_problem(w, vtm, inputs):
    """(A, partition, b) of a workload; b has shape (nrhs, n)."""
    if w["kind"] == "grid":
        A = inputs.grid_poisson(w["dims"], sigma=w["sigma"], seed=0)
        t0 = time.perf_counter()
        part = vtm.partition_evs(A, "grid", dims=w["dims"], block=w["block"])
    else:
        fem = inputs.fem_delaunay(w["npoints"], seed=0)
        A = fem.A
        t0 = time.perf_counter()
        part = vtm.partition_evs(A, "elements", elements=dict(elem_nodes=fem.elem_nodes, elem_mats=fem.elem_mats,
                                                            node_unknown=fem.node_unknown,
                                                            elem_coords=fem.centroids), npieces=w["pieces"])
    t_part = time.perf_counter() - t0
    b = inputs.rhs_uniform(A.n, w["nrhs"], seed=0)
    return A, part, b, t_part


def impedance_arg(z, vtm, part):
    """Solver impedance argument and its description for a workload's impedance rule:
    a number (uniform), "learned:<family>" (a trained model) or "scaled:<c>" (fixed per-line rule
    Z_t = c / (d_a + d_b), d the split diagonal weights of the line's two copies)."""
    if isinstance(z, str) and z.startswith("scaled:"):
        import numpy as np

        f = part.line_features()
        d = np.exp(f[:, 1].astype(np.float64))
        return float(z.split(":", 1)[1]) / (d[0::2] + d[1::2]), z
    if isinstance(z, str) and z.startswith("learned:"):
        from paper_0807_1949_gb300 import learned_z

        path = os.path.join(learned_z.MODELS, "z_" + z.split(":", 1)[1] + ".json")
        return learned_z.load(path), z
    if isinstance(z, str):
        return float(z), z
    return z, z


def coupling_arg(rule, z, zarg, zdesc, vtm, part):
    """(impedance argument, coupling argument, description) for a coupled-line rule: None / "none",
    "model" (the learned model's stored rule: Z = z_scale Z_model, y_p = gamma |a_ik|) or a number
    gamma (conductance factor on the workload's own impedances)."""
    if rule is None or rule == "none":
        return zarg, None, None
    if rule == "model":
        if not (isinstance(z, str) and z.startswith("learned:")):
            raise SystemExit("--coupling model needs a learned impedance model")
        import json

        from paper_0807_1949_gb300 import learned_z

        with open(os.path.join(learned_z.MODELS, "z_" + z.split(":", 1)[1] + ".json")) as f:
            c = json.load(f).get("coupling")
        if c is None:
            raise SystemExit("the model file has no coupling rule (learned_z --couple)")
        zl = vtm.Solver(part, z=zarg, precision="fp32", form="band").impedances()
        return c["z_scale"] * zl, float(c["gamma"]), {"rule": "model", "z_scale": c["z_scale"], "gamma": c["gamma"]}
    g = float(rule)
    return zarg, g, {"rule": "gamma", "gamma": g}


def run_vtm(args):
    import numpy as np
    import torch

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_0807_1949_gb300 import inputs, vtm

    w = WORKLOADS[args.workload]
    A, part, b, t_part = build_problem(w, vtm, inputs)
    R = w["nrhs"]
    stream = torch.cuda.Stream()
    zrule = args.z if args.z is not None else w["z"]
    zarg, zdesc = impedance_arg(zrule, vtm, part)
    zarg, carg, cdesc = coupling_arg(args.coupling if args.coupling is not None else w.get("coupling"),
                                     zrule, zarg, zdesc, vtm, part)
    solver = vtm.Solver(part, z=zarg, precision="fp32", nrhs=R, stream=stream, check_every=args.check_every,
                        inner_reduction=args.inner_reduction,
                        form=args.form, port_storage=args.port_storage, z_init=w.get("z_init", 1.0), coupling=carg)
    sinfo = solver.info()
    bd = torch.tensor(b, device="cuda")
    xd = torch.zeros_like(bd)
    torch.cuda.synchronize()

    # ---- warm-up and timed steps (device timing on the solver's stream)
    maxit = w.get("sweeps", 100000)
    fixed = "sweeps" in w
    for _ in range(args.warmup):
        solver.solve(bd, xd, rtol=w["rtol"], maxit=maxit, raise_on_fail=not fixed)
    torch.cuda.synchronize()
    barrier(ws)
    clk = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        stats.append(solver.solve(bd, xd, rtol=w["rtol"], maxit=maxit, raise_on_fail=not fixed))
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier(ws)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ws, ms)
    x = xd.cpu().numpy()
    As = A.to_scipy()
    rel = float(np.max(np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)))
    sweeps = stats[-1].sweeps
    # port form: every batch ends with a band sweep (interior unknowns for the FP64 check) and every
    # defect-correction phase starts with one (u_base from zero waves)
    band_sweeps = (stats[-1].checks + stats[-1].restarts + 1) if solver.info().sweep_form == 2 else sweeps
    launches = sum(s_.launches for s_ in stats)
    hs, hr, hi = solver.history()   # the FP64 checks of the last timed solve: [sweeps, rel, inner]
    check_history = [[int(a_), float("%.3g" % b_), float("%.3g" % c_)] for a_, b_, c_ in zip(hs, hr, hi)]
    bits_now = solver.info().port_storage_bits
    dtype_desc = ("f32 (f16-stored port responses, f64 residual + defect correction)"
                  if sinfo.sweep_form == 2 and bits_now == 16 else "f32 (f64 residual + defect correction)")

    # ---- dominant kernel, timed with CUDA events on the solver's stream.  Band form: back-to-back
    # band sweeps.  Port form: a batch of k sweeps is k - 1 port sweeps and one band sweep, so the
    # port sweep is (t(k batch) - t(one band sweep)) / (k - 1).
    solver.set_rhs(bd)
    solver.reset()
    solver.iterate(1)          # computes u_base (port form) outside the timed region
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)

    def timed(k, reps):
        k0.record(stream)
        for _ in range(reps):
            solver.iterate(k)
        k1.record(stream)
        torch.cuda.synchronize()
        return k0.elapsed_time(k1) / reps

    elem = 4
    port = sinfo.sweep_form == 2
    band_ms = timed(1, 20)
    vec_passes = 4 if R >= 16 else 1   # wide kernel: b̃ read, y written and read back, x written
    band_bytes = (2 * sinfo.band_entries * elem + vec_passes * sinfo.ncopies * R * elem
                  + 2 * sinfo.nends * R * elem + sinfo.nends * 8)
    if sinfo.ncouplings:
        band_bytes += 4 * sinfo.ncouplings * (8 + R * elem) + sinfo.nports * 4
    if port:
        nsw = 41
        sweep_ms = (timed(nsw, 3) - band_ms) / (nsw - 1)
        # S_j once; waves in (through twin) and out; twin and 1/Z per end; u_base and the end
        # pointers per port
        alg_bytes = (sinfo.port_bytes + 2 * sinfo.nends * R * elem + sinfo.nends * 8
                     + sinfo.nports * (R * elem + 4))
        if sinfo.ncouplings:
            # per coupling 4 list entries (two ports on each side): wave index, -y and one gathered wave
            alg_bytes += 4 * sinfo.ncouplings * (8 + R * elem) + sinfo.nports * 4
        if R >= 16:
            kname, ksrc = "k_port_sweep_tc<%d>" % R, "port_tc.cu"
        else:
            kname = "k_port_sweep<float,%s,%d>" % ("__half" if bits_now == 16 else "float", R)
            ksrc = "port.cu"
    else:
        sweep_ms = band_ms
        alg_bytes = band_bytes
        if R >= 16:
            kname = "k_sweep_wide<float,float,%d>" % R
        elif sinfo.sweep_variant == 1:
            kname = "k_sweep_pipe<float,float,%d>" % R
        else:
            kname = "k_sweep<float,float,%d>" % R
        ksrc = "sweep_wide.cu" if R >= 16 else "sweep.cu"
    pk = peaks()
    achieved = alg_bytes / (sweep_ms * 1e-3) / 1e9
    traffic = kernel_traffic(os.path.join(ROOT, "paper_0807_1949_gb300", "csrc", ksrc), args.workload, kname)

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region);
    # at most 3 repetitions (each is a whole solve), the median reported
    bh = torch.tensor(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    e2e = []
    e2e_reps = max(1, min(args.steps, 3))
    for _ in range(e2e_reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.solve(bh, xh, rtol=w["rtol"], maxit=maxit, raise_on_fail=not fixed)
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = max_over_ranks(ws, statistics.median(e2e))
    del solver

    # ---- plain method (the paper's VTM as stated: FP64 factors and band sweeps every sweep, Z = 1,
    # uncoupled lines, no correction), same workload, first right-hand side, same GPU
    plain = None
    if not args.no_plain:
        torch.cuda.empty_cache()
        pz, pzdesc = impedance_arg(w.get("plain_z", 1.0), vtm, part)
        ps = vtm.Solver(part, z=pz, precision="fp64", nrhs=1, stream=stream, check_every=10, form="band")
        pinfo = ps.info()
        b1, x1 = bd[:1].contiguous(), torch.zeros_like(bd[:1])
        # one band sweep, timed on the solver's stream (the plain method's only kernel per sweep)
        ps.set_rhs(b1)
        ps.reset()
        ps.iterate(1)
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        ps.iterate(10)
        q1.record(stream)
        torch.cuda.synchronize()
        psweep = q0.elapsed_time(q1) / 10
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        pst = ps.solve(b1, x1, rtol=w["rtol"], maxit=maxit, raise_on_fail=False)
        p1.record(stream)
        torch.cuda.synchronize()
        pk0 = peaks()
        pflop = 4.0 * pinfo.band_entries           # 2 flops per band entry, forward and backward
        pbytes = 2.0 * pinfo.band_entries * 8      # FP64 factor read forward and backward
        plain = {"ms": round(p0.elapsed_time(p1), 3), "nrhs": 1, "sweeps": pst.sweeps, "converged": pst.status == 0,
                 "setup_ms": round(pinfo.setup_ms, 1), "precision": "fp64", "z": pzdesc,
                 "sweep_ms": round(psweep, 3),
                 "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": round(pflop / psweep / 1e9, 3),
                              "peak": FP64_TFLOPS, "peak_source": "nominal FP64 rate (no measured FP64 peak)",
                              "frac": round(pflop / psweep / 1e9 / FP64_TFLOPS, 4),
                              "hbm_frac": round(pbytes / psweep / 1e6 / pk0["hbm_gbs"], 4)}}
        if R > 1:
            plain["ms_for_all_rhs"] = round(plain["ms"] * R, 3)
            plain["all_rhs"] = f"{R} x the measured one-right-hand-side solve"
        plain["ms_with_setup"] = round(plain.get("ms_for_all_rhs", plain["ms"]) + pinfo.setup_ms, 1)
        if args.record_plain:
            path = os.path.join(ROOT, "profiles", "plain_sweeps.json")
            rec = {}
            if os.path.exists(path):
                with open(path) as f:
                    rec = json.load(f)
            rec[args.workload] = {"sweeps": pst.sweeps, "rtol": w["rtol"], "z": pzdesc, "check_every": 10,
                                  "source": "bench.py plain arm (FP64 band sweeps, one right-hand side) on a GB300"}
            with open(path, "w") as f:
                json.dump(rec, f, indent=1)
        del ps

    if rank != 0:
        return 0
    cpu = None
    if ws > 1:
        cpu = {"value": None, "unit": "ms", "kind": "oracle", "note": "the oracle is timed at one GPU (N = 1) only"}
    elif not args.no_cpu_baseline and w["kind"] == "grid":
        ks, src = reference_sweeps(args.workload)
        if ks <= 0 and plain:
            ks, src = plain["sweeps"], "the plain FP64 method's count on this GPU"
        elif ks <= 0:
            ks, src = sweeps, "this run's sweep count; the plain method was not run"
        cpu = cpu_baseline(args.workload, ks, src)
    if cdesc is not None:
        cdesc["pairs"] = int(sinfo.ncouplings)
    cfg = {"workload": args.workload, "nrhs": R, "rtol": w["rtol"], "z": zdesc, "coupling": cdesc,
           "pieces": sinfo.npieces,
           "parallelism": "replicas" if ws > 1 else "single",
           "l2": "inputs larger than L2 (FP32 factor %.2f GB, port responses %.2f GB)"
                 % (sinfo.factor_bytes / 1e9, (sinfo.port_bytes if port else 0) / 1e9),
           "sweeps": sweeps, "restarts": stats[-1].restarts, "final_rel_residual": rel,
           "value_with_setup_ms": round(ms + sinfo.setup_ms, 1),
           "setup_ms": round(sinfo.setup_ms, 1), "factor_ms": round(sinfo.factor_ms, 1),
           "partition_ms": round(t_part * 1e3, 1), "sweep_stages": sinfo.sweep_stages,
           "sweep_variant": "pipelined" if sinfo.sweep_variant == 1 else "single-block",
           "form": "port" if port else "band", "check_every": args.check_every,
           "port_storage_bits": int(bits_now) if port else None,
           "band_sweep_ms": round(band_ms, 4), "port_sweep_ms": round(sweep_ms, 4) if port else None,
           "band_sweeps": int(band_sweeps), "port_sweeps": int(sweeps - band_sweeps) if port else 0,
           "port_setup_ms": round(sinfo.port_setup_ms, 1) if port else None,
           "port_bytes": int(sinfo.port_bytes) if port else None,
           "sweep_ctas_per_sm": sinfo.sweep_ctas_per_sm, "e2e_reps": e2e_reps,
           "check_history": check_history, "plain": plain}
    cfg.update({k: w[k] for k in ("dims", "block", "sigma", "npoints") if k in w})
    line = {
        "metric": METRIC if not fixed else ("time for %d VTM sweeps x %d right-hand sides on 1 GB300 "
                                            "(relative residual reached: config.final_rel_residual)" % (maxit, R)),
        "value": round(ms, 3), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_desc, "data": "synthetic",
        "value_with_setup": round(ms + sinfo.setup_ms, 1),
        "config": cfg,
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                     "peak": pk["hbm_gbs"], "peak_source": pk["source"], "unit": "GB/s",
                     "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": traffic,
                     "alg_bytes_per_launch": int(alg_bytes), "launch_ms": round(sweep_ms, 4)},
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": int(A.n * 8 * R),
                "d2h_bytes_per_step": int(A.n * 8 * R)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_vtm(args)


if __name__ == "__main__":
    sys.exit(main())
