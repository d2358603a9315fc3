"""How much a richer impedance search could add to the learned part's training targets.

The targets come from a three-parameter search family (learned_z.search).  Freeing one impedance
factor per subgraph interface, or per line (port), and descending on the same objective (the FP64
residual after a fixed number of sweeps) lowers that objective further, but the sweeps to 1e-8 --
what the impedances are for (§7: Z is the preconditioner) -- move much less: most of the gain at
the search horizon is a transient that the asymptotic contraction does not keep, and what remains
comes from problems where the search's plain coordinate walk stalled (a step in th1 or th2 needed a
new th0).  The profiled walk (th0 re-refined at every step) removes those stalls, and per-interface
freedom then adds next to nothing.  One parameter set of the profiled walk for all problems does
about as well as the per-problem search, and at 256^2 it beats both trained 2D networks.  One small
case runs live with the FP64 oracle as the solver; the stored experiment
(tests/golden/make_search_headroom.py, oracle only) covers 8 problems of 64 x 64 with per-interface
freedom, 5 of 32 x 32 with per-line freedom, 8 of 33^3 in 3D, and the networks on 8 held-out
256^2 problems (FP64, and FP32 sweeps inside FP64 defect correction).
"""
import json
import math
import os
import sys

import numpy as np

from conftest import ROOT

GOLDEN = os.path.join(ROOT, "tests", "golden", "search_headroom.json")


def _headroom_module():
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    try:
        import make_search_headroom as m
    finally:
        sys.path.pop(0)
    return m


def test_interface_descent_lowers_the_objective_but_not_the_sweeps(vtmlib):
    from paper_0807_1949_gb300 import learned_z   # loads the library (built by the vtmlib fixture)

    h = _headroom_module()
    A, split, b, _ = h.problem(32, 8, seed=3)
    ev = h.OracleSolves(A, split, b, horizon=50)
    theta, _ = learned_z.search(ev, sweeps=50)
    z_fam = learned_z.family_z(ev.feats, theta)
    groups = h.interfaces(split)
    assert len(groups) == 24 and sorted(t for g in groups for t in g) == list(range(ev.lines))
    z_face, r_face, _ = h.descend(ev.residual_after, z_fam, groups, steps=(2.0,))
    r_fam = ev.residual_after(z_fam)
    assert r_face < r_fam                                  # the family is not a per-interface optimum
    k1 = ev.to_tolerance(np.ones(ev.lines))
    k_fam = ev.to_tolerance(z_fam)
    k_face = ev.to_tolerance(z_face)
    assert k_fam <= 0.7 * k1                               # the family search itself pays
    assert k_face >= 0.8 * k_fam, (k1, k_fam, k_face, r_fam / r_face)
    # the profiled walk (th0 re-refined at every th1 / th2 step) gets past the plain walk's stall
    theta_p, _ = learned_z.search(ev, sweeps=50, profile=True)
    z_p = learned_z.family_z(ev.feats, theta_p)
    assert ev.residual_after(z_p) <= r_fam
    assert ev.to_tolerance(z_p) <= 0.8 * k_fam            # recorded: 100 against 160


def test_stored_experiment_shows_little_headroom():
    g = json.load(open(GOLDEN))
    face = g["face64"]
    assert len(face["rows"]) == 8 and all(r["lines"] == 402 and r["interfaces"] == 24 for r in face["rows"])
    s = face["summary"]
    # per-interface freedom: the objective drops several-fold, sweeps to 1e-8 by well under 20 %
    assert s["median_objective_gain_over_family"]["face"] >= 2.0
    assert 0.85 <= s["median_sweep_ratio_to_family"]["face"] <= 1.05
    assert s["median_sweep_ratio_to_family"]["z1"] >= 2.0
    # descending on sweeps to 1e-8 itself: per-interface freedom buys a few per cent (median); the
    # family searched on that rugged objective settles worse than on the residual after K sweeps
    assert 0.8 <= s["median_sweep_ratio_to_family"]["face_tol"] <= 1.0
    assert s["median_sweep_ratio_to_family"]["family_tol"] >= 1.0
    # the profiled walk (th0 re-refined at every th1 / th2 step) removes the plain walk's stalls, and
    # per-interface freedom then adds next to nothing
    assert s["median_sweep_ratio_to_family"]["family_profiled"] <= 0.7
    assert s["median_sweeps"]["family_profiled"] < s["median_sweeps"]["face_tol"]
    extra = [r["sweeps"]["face_profiled"] / r["sweeps"]["family_profiled"] for r in face["rows"]]
    assert np.median(extra) >= 0.95 and min(extra) >= 0.8
    # and one parameter set for all problems (leave one out) does nearly as well as the per-problem one
    assert s["median_sweeps"]["global_profiled"] <= 1.1 * s["median_sweeps"]["family_profiled"]
    line = g["line32"]
    assert len(line["rows"]) == 5 and all(r["interfaces"] == 24 for r in line["rows"])
    s = line["summary"]
    # per-line freedom: the objective drops far more than per interface, the sweeps much less
    assert s["median_objective_gain_over_family"]["line"] >= 4 * s["median_objective_gain_over_family"]["face"]
    assert 0.75 <= s["median_sweep_ratio_to_family"]["line"] <= 1.0
    # 3D (the family of the 256^3 run, 33^3 in 8^3 blocks): the same stall and the same one-theta rule
    d3 = g["profiled3d"]
    assert len(d3["rows"]) == 8 and all(r["theta_profiled"][1] == -1.0 for r in d3["rows"])
    s = d3["summary"]
    assert s["median_sweep_ratio_to_family"]["family_profiled"] <= 0.75
    assert s["median_sweeps"]["global_profiled"] <= 1.1 * s["median_sweeps"]["family_profiled"]
    # 256^2, held-out seeds of the 2D family, FP64 oracle: the one-theta rule of the profiled walk
    # needs fewer sweeps than either trained network
    net = g["networks256"]
    assert len(net["rows"]) == 8 and net["theta"]["profiled"][1] == -1.0
    m = net["median_sweeps"]
    assert m["profiled_one_theta"] < min(m["plain_network"], m["profiled_network"], m["plain_one_theta"])
    # the same with FP32 sweeps inside FP64 defect correction (the structure of the library's solve),
    # where the network of profiled targets beats the shipped one but not the one-theta rule
    net = g["networks256_fp32"]
    m = net["median_sweeps"]
    assert m["profiled_network"] < 0.8 * m["plain_network"]
    assert m["profiled_one_theta"] < min(m["plain_network"], m["profiled_network"], m["plain_one_theta"])
    for r in face["rows"] + line["rows"] + d3["rows"]:
        assert all(math.isfinite(v) for v in r["objective"].values())
