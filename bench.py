"""Benchmark of the dual-smoothing hot path (one P-APG iteration = one step).

Default workload: the log-sum-exp instance with N = 20000 points in 20 dimensions
(x ~ U[-1,1]^20, y = log sum_k exp(a_k.x) + N(0, 0.1^2), 8 terms, seed 0), FP32 multipliers
(2 x 1.6 GB, larger than L2, so no flush is needed between steps), gamma = 1e-4.

A step is one iteration: the fused Lambda sweep (every one of the N(N-1) pairs read and
written once) plus the O(N n) finalize/recovery kernel.  ``value`` is lambda-pair updates
per second over the timed steps (inputs already resident in HBM), timed with CUDA events on
the library's stream; ``e2e`` is the same metric through the public API from host buffers
(create from host X and ybar, the K iterations, and the copy of (y, xi) back to the host
inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Under torchrun (N > 1) every rank solves its own instance (seed + rank, weak scaling); the
timed region is bracketed by barriers and the slowest rank's time is reported.
``--impl reference`` times the FP64 CPU oracle instead (on a bounded row sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import cr_synth  # noqa: E402

METRIC = "lambda_pair_updates_per_s"
UNIT = "pairs/s"
GAMMA = 1e-4
CPU_SAMPLE_S = 12.0           # host seconds of the oracle sample beside the GPU line
L2_BYTES = 126 * 2**20        # GB300 L2
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5: SMs x FP32 lanes x FMA x max SM clock
FP64_PEAK_TFLOPS = 1.25       # nominal GB300 FP64
CPU_SAMPLE_N = 8000  # oracle sample: the first 8000 points of the same instance
REF_BUDGET_S = 90.0  # --impl reference: target seconds of oracle work for warm-up + steps


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()  # the timed region starts once samples are flowing
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_instance(workload, rank, N=0):
    """The instance a rank solves: the named workload drawn with seed + rank (replicas: each
    rank holds its own independent instance of the same shape)."""
    spec = dict(cr_synth.WORKLOADS[workload])
    spec["seed"] = spec.get("seed", 0) + rank
    if N:
        spec["N"] = N
    return cr_synth.make_instance(**spec)


def max_over_ranks(x, ws, device="cuda"):
    """The largest value of x over all ranks (x itself when there is one rank)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(pairs_per_rank, steps, ws, t_max_ms):
    """Whole-job rate: the pairs all ranks updated in `steps` iterations over the slowest
    rank's time."""
    return pairs_per_rank * steps * ws / (t_max_ms / 1e3)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    inst = cr_synth.workload(args.workload)
    # bounded sample: the oracle's cost per iteration grows as N^2, so the sample size is
    # chosen from a one-iteration calibration to keep warm-up + steps near REF_BUDGET_S
    n0 = min(1000, inst.N)
    oc = oracle.PAPG(inst.X[:n0], inst.ybar[:n0], GAMMA, oracle.lipschitz(inst.X[:n0], GAMMA))
    t0 = time.perf_counter()
    oc.step(1, log=False)
    t1 = max(time.perf_counter() - t0, 1e-6)
    scale = (REF_BUDGET_S / (args.steps + args.warmup) / t1) ** 0.5
    Ns = int(max(200, min(CPU_SAMPLE_N, inst.N, n0 * scale)) // 100 * 100)
    X, yb = inst.X[:Ns], inst.ybar[:Ns]
    L = oracle.lipschitz(X, GAMMA)
    o = oracle.PAPG(X, yb, GAMMA, L)
    o.step(args.warmup, log=False)
    t0 = time.perf_counter()
    o.step(args.steps, log=False)
    dt = time.perf_counter() - t0
    pairs = Ns * (Ns - 1) * args.steps
    v = pairs / dt
    sample = (f"first {Ns} of the {inst.N} points of {args.workload}; {args.steps} oracle iterations "
              f"(FP64 C, OpenMP)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "N": Ns, "n": inst.n, "gamma": GAMMA},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def solve_record(crgb, inst, prec, tol=1e-4, max_sweeps=20000):
    """The solve half of the metric on the timed instance: cr_solve to rel_gap <= tol with the
    adaptive step of Section 4 and momentum restart, through the public API from host buffers
    (creation, the step constant and the copies included)."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, precision=prec, step_rule=crgb.CR_STEP_ADAPTIVE,
                     restart=1, upsilon=2.0, check_every=100) as s:
        t1 = time.perf_counter()
        ok, g = s.solve(tol, max_sweeps)
        y, xi = s.primal()
    t2 = time.perf_counter()
    return {"converged": bool(ok), "tol": tol, "wall_s": t2 - t0, "create_s": t1 - t0, "sweeps": g["sweeps"],
            "iterations": g["k"], "rel_gap": g["rel_gap"], "dual_g": g["dual_g"], "solves_per_s": 1.0 / (t2 - t0),
            "rule": "adaptive + restart", "max_sweeps": max_sweeps}


def batch_record(crgb, count=64, tol=1e-4, max_iter=20000):
    """Batched solves against the plain single-instance path on the same instances: `count`
    instances of the batched workload (N log-uniform in [100, 4000], n in {2..16},
    ||x||^2 + N(0, 0.1^2)), mixed precision, adaptive step + restart, each to rel_gap <= tol.
    Completion times count from the moment all instances are handed over (t = 0)."""
    import torch

    insts = cr_synth.batch_workload(count, seed=0)
    ropt = dict(step_rule=crgb.CR_STEP_ADAPTIVE, upsilon=2.0, restart=1)
    check = 100

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(q * len(v)))]

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done_at = {}
    with crgb.Batch(gamma=GAMMA, graph_iters=20, check_every=check, precision=crgb.CR_MIXED_TF32, **ropt) as b:
        ids = [b.add(i.X, i.ybar, tol=tol, max_iter=max_iter) for i in insts]
        active = len(ids)
        while active:
            active = b.step(check)
            now = time.perf_counter() - t0
            for i in ids:
                if i not in done_at and b.poll(i)[0]:
                    done_at[i] = now
        conv = sum(1 for i in ids if b.poll(i)[1] == 0)
    wall = time.perf_counter() - t0
    t1 = time.perf_counter()
    plain_at, plain_conv = [], 0
    for inst in insts:
        with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, check_every=check, graph_iters=20,
                         precision=_prec(crgb, "tf32", inst.n), **ropt) as s:
            ok, _ = s.solve(tol, max_iter)
        plain_conv += int(ok)
        plain_at.append(time.perf_counter() - t1)
    plain_wall = time.perf_counter() - t1
    lat = list(done_at.values())
    return {"workload": f"batch{count}_sqnorm_N100-4000_n2-16", "precision": "tf32", "tol": tol,
            "batched": {"solves_per_s": count / wall, "p50_s": pct(lat, 0.5), "p99_s": pct(lat, 0.99),
                        "converged": conv, "wall_s": wall},
            "plain_single_instance": {"solves_per_s": count / plain_wall, "p50_s": pct(plain_at, 0.5),
                                      "p99_s": pct(plain_at, 0.99), "converged": plain_conv, "wall_s": plain_wall}}


def cpu_one_core(workload, seconds=6.0):
    """The oracle on one host core (OMP_NUM_THREADS=1 in a fresh process): pairs/s."""
    code = ("import json, time, sys; sys.path.insert(0, %r); import cr_synth, oracle; "
            "inst = cr_synth.workload(%r); Ns = 2000; X, yb = inst.X[:Ns], inst.ybar[:Ns]; "
            "o = oracle.PAPG(X, yb, %r, oracle.lipschitz(X, %r)); t0 = time.perf_counter(); o.step(1, log=False); "
            "t1 = time.perf_counter() - t0; it = int(max(2, min(200, %r / max(t1, 1e-3)))); "
            "t0 = time.perf_counter(); o.step(it, log=False); dt = time.perf_counter() - t0; "
            "print(json.dumps({'value': Ns * (Ns - 1) * it / dt, 'cores': oracle.threads(), "
            "'sample': 'first %%d points, %%d iterations (%%.1f s)' %% (Ns, it, dt)}))"
            % (ROOT, workload, GAMMA, GAMMA, seconds))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1:] or ["failed"]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    d["unit"] = UNIT
    return d


def cpu_baseline(workload):
    import oracle

    inst = cr_synth.workload(workload)
    Ns = min(CPU_SAMPLE_N, inst.N)
    X, yb = inst.X[:Ns], inst.ybar[:Ns]
    o = oracle.PAPG(X, yb, GAMMA, oracle.lipschitz(X, GAMMA))
    t0 = time.perf_counter()
    o.step(1, log=False)  # warm-up, also the calibration of the sample length
    t1 = time.perf_counter() - t0
    iters = int(min(500, max(3, round(CPU_SAMPLE_S / max(t1, 1e-3)))))  # about CPU_SAMPLE_S of host work
    t0 = time.perf_counter()
    o.step(iters, log=False)
    dt = time.perf_counter() - t0
    return {"value": Ns * (Ns - 1) * iters / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"first {Ns} points of {workload}, {iters} FP64 oracle iterations ({dt:.1f} s)"}


def _prec(crgb, name, n=None):
    """Library precision for a --precision name; n = 32 points run the FP32 sweep under tf32
    (the tensor-core operand carries a row of ones, so it holds n <= 31), as batches do."""
    if name == "tf32" and n is not None and n > crgb.CR_MAX_N_TF32:
        name = "fp32"
    return {"fp32": crgb.CR_FP32, "fp64": crgb.CR_FP64, "tf32": crgb.CR_MIXED_TF32}[name]


def _rule_options(crgb, rule):
    if rule == "adaptive":
        return dict(step_rule=crgb.CR_STEP_ADAPTIVE, upsilon=2.0, restart=1)
    return dict(step_rule=crgb.CR_STEP_CONSTANT)


def run_batch(args):
    """Batched solves: `count` instances (N log-uniform in [100, 4000], n in {2..16},
    f0 = ||x||^2 + N(0, 0.1^2)), all submitted at t = 0 into one cr_batch, each retired at
    rel_gap <= tol.  Reports solves/s, lambda-pair updates/s and completion-time p50/p99,
    against the same instances solved one after another with the single-instance path and the
    same step rule (within --plain-budget seconds; the rate is over the instances it finished)."""
    import torch

    import paper_1608_02227_gb300 as crgb

    torch.cuda.set_device(0)
    insts = cr_synth.batch_workload(args.count, seed=0)
    check = 100
    max_iter = 200000
    ropt = _rule_options(crgb, args.rule)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done_at = {}
    pairs = 0.0
    with crgb.Batch(gamma=GAMMA, graph_iters=20, check_every=check, precision=_prec(crgb, args.precision),
                    **ropt) as b:
        ids = [b.add(i.X, i.ybar, tol=args.tol, max_iter=max_iter) for i in insts]
        t_setup = time.perf_counter() - t0
        width = b.autotune(2)
        active = len(ids)
        while active:
            active = b.step(check)
            now = time.perf_counter() - t0
            for i in ids:
                if i not in done_at and b.poll(i)[0]:
                    done_at[i] = now
        infos = [b.poll(i) for i in ids]
    wall = time.perf_counter() - t0
    for inst, (done, st, info) in zip(insts, infos):
        pairs += inst.N * (inst.N - 1) * info["sweeps"]
    lat = sorted(done_at.values())
    conv = sum(1 for d, st, _ in infos if st == 0)
    # the plain single-instance path: one cr_solve after another, same options
    t1 = time.perf_counter()
    plain_done, plain_conv = 0, 0
    for inst in insts:
        with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, check_every=check, graph_iters=20,
                         precision=_prec(crgb, args.precision, inst.n), **ropt) as s:
            ok, _ = s.solve(args.tol, max_iter)
        plain_done += 1
        plain_conv += int(ok)
        if time.perf_counter() - t1 > args.plain_budget:
            break
    plain_wall = time.perf_counter() - t1
    line = {"metric": "solves_per_s", "value": len(insts) / wall, "unit": "solves/s", "n_gpus": 1,
            "steps": None, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch{len(insts)}_sqnorm_N100-4000_n2-16", "gamma": GAMMA, "tol": args.tol,
                       "check_every": check, "tile_cols": width, "step_rule": args.rule,
                       "precision": args.precision},
            "converged": conv, "lambda_pairs_per_s": pairs / wall, "setup_s": t_setup, "wall_s": wall,
            "latency_s": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                          "max": lat[-1]},
            "sweeps": {"min": min(i[2]["sweeps"] for i in infos), "max": max(i[2]["sweeps"] for i in infos)},
            "plain_single_instance": {"solves_per_s": plain_done / plain_wall, "instances": plain_done,
                                      "converged": plain_conv, "wall_s": plain_wall}}
    print(json.dumps(line), flush=True)
    return 0


def run_solve(args):
    """Time to a relative gap `tol` on one instance of the workload: the adaptive step size of
    Section 4 with and without momentum restart against the constant step 1/L (each capped at
    --max-sweeps sweeps), mixed precision by default; `value` is the adaptive run with restart.  Reports the solve time through the public API (creation included and
    separately), sweeps, accepted iterations and the final certificate."""
    import torch

    import paper_1608_02227_gb300 as crgb

    torch.cuda.set_device(0)
    prec = {"fp32": crgb.CR_FP32, "fp64": crgb.CR_FP64, "tf32": crgb.CR_MIXED_TF32}[args.precision]
    spec = dict(cr_synth.WORKLOADS[args.workload])
    if args.N:
        spec["N"] = args.N
    inst = cr_synth.make_instance(**spec)
    runs = {}
    for name, rule, restart in (("adaptive_restart", crgb.CR_STEP_ADAPTIVE, 1), ("adaptive", crgb.CR_STEP_ADAPTIVE, 0),
                                ("constant", crgb.CR_STEP_CONSTANT, 0)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, precision=prec, step_rule=rule, restart=restart,
                         check_every=args.check_every) as s:
            t1 = time.perf_counter()
            ok, g = s.solve(args.tol, args.max_sweeps)
            t2 = time.perf_counter()
        runs[name] = {"converged": bool(ok), "solve_s": t2 - t1, "create_s": t1 - t0, "sweeps": g["sweeps"],
                      "iterations": g["k"], "rel_gap": g["rel_gap"], "dual_g": g["dual_g"],
                      "cert_gap_rel": g["cert_gap_rel"], "ms_per_sweep": 1e3 * (t2 - t1) / max(1, g["sweeps"])}
    best = runs.get("adaptive_restart", runs["constant"])
    line = {"metric": "solves_per_s", "value": 1.0 / (best["solve_s"] + best["create_s"]), "unit": "solves/s",
            "n_gpus": 1, "steps": None, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec != crgb.CR_FP64 else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": inst.N, "n": inst.n, "gamma": GAMMA, "tol": args.tol,
                       "precision": args.precision, "check_every": args.check_every,
                       "max_sweeps": args.max_sweeps},
            "runs": runs}
    print(json.dumps(line), flush=True)
    return 0


def run_paper(args):
    """Section 5's experiment shapes on this K = N path: f0 in {1/2 x^T Q x (condition number
    15), exp(p^T x)}, n in {20, 80}, N in {200, 400, 800, 1600, 2400}, x ~ N(0, 4 I), noise
    N(0, 100), 30% of the observations scaled by 1.3, gamma = 1e-4.  PAPG_C (constant step),
    PAPG_A (Section 4's adaptive step) and PAPG_A with momentum restart each run to Section 5's
    stopping rule -- normalised infeasibility <= 1e-1 and |lambda^T C eta| / (N^2 - N) <= 5e-7 --
    checked every --check-every sweeps (at most --max-sweeps).  Wall time includes creation
    (Section 5's "Preprocess": the step constant; here also the transfers and transposes).
    SubOpt_Reg = |r_gamma(eta) - p*| / p*, with p* taken as the dual value of a long adaptive
    restart run (its certified bracket is reported).  One JSON line per configuration."""
    import torch

    import paper_1608_02227_gb300 as crgb

    torch.cuda.set_device(0)
    Ns = [200, 400] if args.paper_set == "small" else [200, 400, 800, 1600, 2400]
    rows = []
    for fam in (("exp",) if args.paper_set == "exp20" else ("quad", "exp")):
        for n in ((20,) if args.paper_set == "exp20" else (20, 80)):
            for N in Ns:
                inst = cr_synth.make_instance(N, n, fam, 10.0, 0, x_dist="normal4", interior_frac=0.3)
                pname = args.precision if not (args.precision == "tf32" and n > crgb.CR_MAX_N_TF32) else "fp32"
                prec = {"fp32": crgb.CR_FP32, "fp64": crgb.CR_FP64, "tf32": crgb.CR_MIXED_TF32}[pname]
                pairs = float(N) * (N - 1)
                runs = {}
                for name, rule, restart in (("PAPG_C", crgb.CR_STEP_CONSTANT, 0), ("PAPG_A", crgb.CR_STEP_ADAPTIVE, 0),
                                            ("PAPG_A_restart", crgb.CR_STEP_ADAPTIVE, 1)):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, precision=prec, step_rule=rule,
                                     restart=restart) as sv:
                        t1 = time.perf_counter()
                        sweeps, ok, g = 0, False, None
                        while sweeps < args.max_sweeps:
                            step = min(args.check_every, args.max_sweeps - sweeps)
                            sv.step(step)
                            sweeps += step
                            g = sv.gap()
                            if g["infeas_norm"] <= 1e-1 and abs(g["lagr_gap"]) / pairs <= 5e-7:
                                ok = True
                                break
                        t2 = time.perf_counter()
                    runs[name] = {"converged": ok, "wall_s": t2 - t0, "preprocess_s": t1 - t0, "sweeps": g["sweeps"],
                                  "iterations": g["k"], "infeasibility": g["infeas_norm"],
                                  "dual_gap": abs(g["lagr_gap"]) / pairs, "primal_r": g["primal_r"],
                                  "dual_g": g["dual_g"]}
                # p* of Eq. (regularize): a long adaptive restart run (FP64 where the working
                # precision cannot resolve the gap: p* of the exp workloads is ~1e-2 of r at eta = 0)
                ref_prec = "fp32"
                with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, precision=crgb.CR_FP32,
                                 step_rule=crgb.CR_STEP_ADAPTIVE, restart=1, check_every=200) as sv:
                    ok_r, gr = sv.solve(1e-7, args.max_sweeps * 4)
                if not ok_r:
                    ref_prec = "fp64"
                    with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, precision=crgb.CR_FP64,
                                     step_rule=crgb.CR_STEP_ADAPTIVE, restart=1, check_every=500) as sv:
                        ok_r, gr = sv.solve(1e-9, args.max_sweeps)
                pstar = gr["dual_g"]
                for r in runs.values():
                    r["subopt_reg"] = abs(r["primal_r"] - pstar) / abs(pstar)
                line = {"config": {"f0": fam, "n": n, "N": N, "gamma": GAMMA, "precision": pname,
                                   "check_every": args.check_every, "max_sweeps": args.max_sweeps},
                        "pstar": {"dual_g": pstar, "cert_primal": gr["cert_primal"], "rel_gap": gr["rel_gap"],
                                  "converged": bool(ok_r), "precision": ref_prec},
                        "runs": runs}
                rows.append(line)
                print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson stream (rate args.rate) of `count` requests: N log-uniform in [200, N_max], n in
    {2..32}, f0 drawn from {||x||^2, max of 10 affine, log-sum-exp of 8}, noise 0.1; each to
    rel_gap <= tol (cap 20000 sweeps).  Served with continuous batching (60 GB cap), then
    the same stream on the plain single-instance path (one solve at a time, FIFO, same
    arrival times, cr_solve with the same check interval and step rule)."""
    import torch

    import paper_1608_02227_gb300 as crgb

    torch.cuda.set_device(0)
    reqs = cr_synth.serving_stream(args.count, rate=args.rate, seed=0, N_lo=200, N_hi=args.N_max)
    max_iter, check = 20000, 100
    # continuous batching
    t0 = time.perf_counter()
    ropt = _rule_options(crgb, args.rule)
    with crgb.Server(mem_cap_bytes=60 << 30, max_active=256, gamma=GAMMA, check_every=check,
                     graph_iters=20, precision=_prec(crgb, args.precision), **ropt) as srv:
        ids = []
        for t_arr, inst in reqs:
            delay = t_arr - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(inst.X, inst.ybar, tol=args.tol, max_iter=max_iter))
        for r in ids:
            srv.wait(r, 3600)
        polls = [srv.poll(r) for r in ids]
        stats = srv.stats()
    wall = time.perf_counter() - t0
    lat = sorted(p[3] for p in polls)
    served = {"solves_per_s": len(ids) / wall, "p50_s": lat[len(lat) // 2],
              "p99_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "converged": sum(p[1] == 0 for p in polls),
              "wall_s": wall, "busy_s": stats["busy_s"]}
    # plain single-instance path, FIFO over the same arrival times
    clock = 0.0
    lat_plain, conv_plain = [], 0
    for t_arr, inst in reqs:
        start = max(clock, t_arr)
        s0 = time.perf_counter()
        with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, check_every=check, graph_iters=20,
                         precision=_prec(crgb, args.precision, inst.n), **ropt) as s:
            ok, rec = s.solve(args.tol, max_iter)
        clock = start + (time.perf_counter() - s0)
        lat_plain.append(clock - t_arr)
        conv_plain += int(ok)
    lat_plain.sort()
    plain = {"solves_per_s": len(reqs) / clock, "p50_s": lat_plain[len(lat_plain) // 2],
             "p99_s": lat_plain[min(len(lat_plain) - 1, int(0.99 * len(lat_plain)))], "converged": conv_plain,
             "wall_s": clock}
    line = {"metric": "solves_per_s", "value": served["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": None, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serve_poisson{args.rate:g}_{len(reqs)}req_N200-{args.N_max}_n2-32",
                       "gamma": GAMMA, "tol": args.tol, "max_iter": max_iter, "mem_cap_GB": 60,
                       "step_rule": args.rule, "precision": args.precision},
            "served": served, "plain_single_instance": plain,
            "offered_rate": args.rate, "achieved_rate": served["solves_per_s"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="lse_N20000_n20")
    ap.add_argument("--N", type=int, default=0, help="shrink the workload to its first N points (profiling)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32", choices=["fp32", "fp64", "tf32"],
                    help="tf32: FP32 multipliers with hi+lo TF32 tensor-core contractions (the mixed-precision "
                         "configuration of the N = 20000 workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paper-set", default="all", choices=["all", "small", "exp20"],
                    help="--mode paper: all of Section 5's N, N in {200, 400}, or exp(p^T x) at n = 20 only")
    ap.add_argument("--mode", default="sweep", choices=["sweep", "batch", "serve", "solve", "paper"],
                    help="sweep: lambda-pair rate of one instance; batch: solves/s of 256 instances; "
                         "serve: Poisson request stream through the serving runtime; solve: time to the "
                         "gap on one instance, adaptive vs constant step")
    ap.add_argument("--max-sweeps", type=int, default=40000, help="sweep cap of each run in --mode solve")
    ap.add_argument("--check-every", type=int, default=100, help="sweeps between gap checks in --mode solve")
    ap.add_argument("--rule", default="adaptive", choices=["adaptive", "constant"],
                    help="step rule of --mode batch / serve: adaptive (Section 4, with momentum restart) or "
                         "constant 1/L")
    ap.add_argument("--plain-budget", type=float, default=120.0,
                    help="seconds for the one-after-another single-instance comparison in --mode batch")
    ap.add_argument("--rate", type=float, default=20.0, help="requests/s in --mode serve")
    ap.add_argument("--N-max", type=int, default=4000, help="largest N of a request in --mode serve")
    ap.add_argument("--count", type=int, default=256, help="instances in --mode batch")
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--quick", action="store_true",
                    help="default mode: skip the solve and batch records (profiling runs)")
    ap.add_argument("--batch-count", type=int, default=64, help="instances of the batch record")
    ap.add_argument("--refresh", type=int, default=64,
                    help="iterations between exact FP64 re-evaluations of C^T lambda (0: C^T from FP32 partials "
                         "every iteration, no delta form)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "solve":
        return run_solve(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "paper":
        return run_paper(args)

    import torch

    import paper_1608_02227_gb300 as crgb

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    prec = {"fp32": crgb.CR_FP32, "fp64": crgb.CR_FP64, "tf32": crgb.CR_MIXED_TF32}[args.precision]
    inst = rank_instance(args.workload, rank, args.N)
    N, n = inst.N, inst.n
    pairs = N * (N - 1)

    s = crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, precision=prec, refresh_every=args.refresh)
    desc = s.describe()
    s.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # clock samples cover the whole measured block (the timed sweeps, the end-to-end run and
    # the solve and batch records): the timed region alone can be shorter than one sample
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    sweep_ms, total_ms = crgb.cr_dual_step_timed(s.ctx, args.steps)
    barrier()
    gap = s.gap()
    s.close()
    t_max = max_over_ranks(total_ms, ws)
    value = job_rate(pairs, args.steps, ws, t_max)

    # end to end through the public API from host buffers
    barrier()
    t0 = time.perf_counter()
    with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, precision=prec, refresh_every=args.refresh) as s2:
        s2.step(args.steps)
        y, xi = s2.primal()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": job_rate(pairs, args.steps, ws, 1e3 * e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": (inst.X.nbytes + inst.ybar.nbytes) / args.steps,
           "d2h_bytes_per_step": (y.nbytes + xi.nbytes) / args.steps}
    extras = {}
    if not args.quick and ws == 1:
        extras["solve"] = solve_record(crgb, inst, prec, tol=args.tol)
        extras["batch"] = batch_record(crgb, count=args.batch_count, tol=args.tol)
    clk = clocks.stop()

    if rank == 0:
        peak, src = _peaks()
        tsz = 8 if prec == crgb.CR_FP64 else 4
        alg_bytes = 3 * tsz * pairs  # read lambda^{k-1}, lambda^{k-2}; write lambda^k
        sweep_avg_s = sweep_ms / 1e3 / args.steps
        achieved = alg_bytes / sweep_avg_s / 1e9
        traffic = None
        tpath = os.path.join(ROOT, "profiles", "sweep_traffic.json")
        if os.path.exists(tpath):
            with open(tpath) as fh:
                td = json.load(fh)
            if td.get("workload") == args.workload and td.get("precision") == args.precision:
                traffic = td.get("bytes_per_launch")
        # Lambda state that fits in L2 (the Section 5 sizes, N <= 2400) stays there between
        # sweeps, as it does in a real solve: the sweep is then bound by the FP32 (or FP64) ALU,
        # 4n + 7 flop per pair, not by HBM
        l2_resident = 2 * tsz * float(N) * N <= L2_BYTES and prec != crgb.CR_MIXED_TF32
        if l2_resident:
            alu_peak = FP64_PEAK_TFLOPS if prec == crgb.CR_FP64 else FP32_PEAK_TFLOPS
            flops = float(4 * n + 7) * pairs
            roof = {"bound": "alu", "achieved": flops / sweep_avg_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": flops / sweep_avg_s / 1e12 / alu_peak, "traffic": None,
                    "peak_source": "derived (152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz)"
                    if prec != crgb.CR_FP64 else "nominal FP64", "kernel": "sweep",
                    "algorithmic_flops_per_launch": flops, "avg_launch_ms": sweep_avg_s * 1e3,
                    "hbm_equivalent_gbs": achieved}
            l2_note = "Lambda resident in L2 (2 N x N arrays below 126 MB), no flush: ALU-bound"
        else:
            roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic, "peak_source": src,
                    "kernel": "sweep", "algorithmic_bytes_per_launch": alg_bytes,
                    "avg_launch_ms": sweep_avg_s * 1e3}
            l2_note = "inputs larger than L2 (two N x N FP32 multiplier arrays)"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "tf32": "f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "n": n, "gamma": GAMMA, "precision": args.precision,
                       "l2": l2_note,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "grid": desc["grid"], "rows_per_item": desc["rows_per_item"],
                       "col_splits": desc["col_splits"], "ct_delta_form": bool(desc.get("delta")),
                       "refresh_every": desc.get("refresh_every", 0)},
            "roofline": roof,
            "e2e": e2e,
            # per iteration: sweep + finalize (+ the three gated kernels of the exact C^T refresh)
            "gpu_launches": (2 + (3 if desc.get("delta") else 0)) * args.steps,
            "clocks": clk,
            "gap_at_end": {"k": gap["k"], "rel_gap": gap["rel_gap"], "dual_g": gap["dual_g"]},
        }
        line.update(extras)
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload)
            line["cpu_baseline"]["one_core"] = cpu_one_core(args.workload)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
