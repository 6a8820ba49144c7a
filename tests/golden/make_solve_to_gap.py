"""Writes tests/golden/solve_to_gap.json: the FP64 oracle's solves of two mid-size instances to
relative duality gap 1e-4 (and 1e-8), the references the reduced-precision GPU modes are held to.

Calls only ``oracle/`` (and the seeded generators of ``cr_synth``).  Iterates start from
theta^0 = 0 (K = N, Step 1 in closed form) and are checked every ``check`` iterations with the
relative gap of the library,
    rel_gap = max(|theta^T C eta| / r_gamma(eta), ||(C eta)_-||_2 / (sqrt(N^2 - N) rms(ybar))),
eta = eta(theta^k) (Section 5.1's duality gap and normalised infeasibility, made scale-free).
Recorded per instance, besides the step constant L (oracle.lipschitz):
  * "constant" (log-sum-exp instance): Figure "papg" with the constant step 1/L up to the first
    checked K with rel_gap <= 1e-4; at K the dual objective g_gamma(theta^K), r_gamma, theta^T C eta,
    the infeasibility, rel_gap, the fitted values y of eta(theta^K) and the subgradients xi of a
    sample of rows, and the run's g and rel_gap at every check;
  * "adaptive_restart": Section 4's adaptive step with momentum restart until rel_gap <= 1e-8;
    its dual value there (the optimum p*_gamma to about 1e-8) and where it first met 1e-4.

Run:  python tests/golden/make_solve_to_gap.py   (a few minutes on 8-16 host cores)
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import cr_synth  # noqa: E402
import oracle  # noqa: E402

GAMMA = 1e-4
TOL = 1e-4
TIGHT = 1e-8
CASES = [
    # the N = 20000 log-sum-exp workload's family at N = 1500 (mixed precision on the GPU)
    dict(name="lse_N1500_n20", N=1500, n=20, family="lse", noise=0.1, seed=0, check=100, cap=60000),
    # the N = 5000 max-affine workload's family at N = 1000 (FP32 on the GPU)
    dict(name="maxaff_N1000_n10", N=1000, n=10, family="maxaff", noise=0.05, seed=0, check=100, cap=60000),
]


def rel_gap(X, ybar, o):
    d = o.dual()
    cert = oracle.certify(X, ybar, GAMMA, d["y"], d["xi"])
    N = X.shape[0]
    infeas = math.sqrt(cert["infeas_sq"] / (N * N - N))
    rms = math.sqrt(float(np.mean(ybar * ybar)))
    return max(abs(d["lg"]) / d["r"], infeas / rms), d, infeas


def constant_step_to_gap(c, X, ybar, L):
    """Figure "papg" with the constant step 1/L from theta^0 = 0 to the first checked rel_gap <= TOL."""
    o = oracle.PAPG(X, ybar, GAMMA, L)
    trace = []
    K = None
    while o.k < c["cap"]:
        o.step(c["check"], log=False)
        rg, d, infeas = rel_gap(X, ybar, o)
        trace.append([o.k, d["g"], rg])
        if rg <= TOL:
            K = o.k
            break
    N = c["N"]
    rows = sorted({0, 1, 2, 31, 32, 127, 128, 129, N // 3, N // 2, 2 * N // 3, N - 129, N - 33, N - 2, N - 1}
                  | set(range(0, N, max(1, N // 48))))
    return dict(K=K, g=d["g"], r=d["r"], lg=d["lg"], infeas=infeas, rel_gap=rg, y=[float(v) for v in d["y"]],
                xi_rows=rows, xi=[[float(v) for v in d["xi"][i]] for i in rows], trace=trace)


def adaptive_to_tight_gap(c, X, ybar, L):
    """Section 4's adaptive step with momentum restart from theta^0 = 0: the dual value at the first
    checked rel_gap <= TOL and at the first checked rel_gap <= TIGHT (the optimum to about 1e-8)."""
    o = oracle.PAPG(X, ybar, GAMMA, L, adaptive=True, restart=True)
    first = None
    trace = []
    while o.k < c["cap"]:
        o.step(c["check"], log=False)
        rg, d, _ = rel_gap(X, ybar, o)
        trace.append([o.k, d["g"], rg])
        if first is None and rg <= TOL:
            first = dict(k=o.k, g=d["g"], rel_gap=rg)
        if rg <= TIGHT:
            return dict(at_tol=first, k=o.k, g=d["g"], rel_gap=rg, trace=trace)
    return dict(at_tol=first, k=None, g=d["g"], rel_gap=rg, trace=trace)


def main():
    out = {"_source": "FP64 oracle (oracle/cr_oracle.c), K = N; written by tests/golden/make_solve_to_gap.py",
           "gamma": GAMMA, "tol": TOL, "tight": TIGHT, "cases": []}
    for c in CASES:
        inst = cr_synth.make_instance(c["N"], c["n"], c["family"], c["noise"], c["seed"])
        X, ybar = inst.X, inst.ybar
        L = oracle.lipschitz(X, GAMMA)
        t0 = time.time()
        rec = dict(name=c["name"], N=c["N"], n=c["n"], family=c["family"], noise=c["noise"], seed=c["seed"],
                   L=L, check=c["check"])
        if c["family"] == "lse":
            rec["constant"] = constant_step_to_gap(c, X, ybar, L)
        rec["adaptive_restart"] = adaptive_to_tight_gap(c, X, ybar, L)
        rec["oracle_seconds"] = time.time() - t0
        out["cases"].append(rec)
        print(c["name"], "constant K =", rec.get("constant", {}).get("K"), "adaptive: tol at",
              rec["adaptive_restart"]["at_tol"], "tight at k =", rec["adaptive_restart"]["k"],
              "g* = %.12f" % rec["adaptive_restart"]["g"], "%.0f s" % rec["oracle_seconds"], flush=True)
    with open(os.path.join(HERE, "solve_to_gap.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
