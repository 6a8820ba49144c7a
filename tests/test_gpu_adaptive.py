"""Adaptive step size (Section 4, Eq. (adaptive-check)), with and without function-value
restart of the momentum, on the GPU against the FP64 oracle's adaptive iteration.

FP64 mode: the accept/reject decisions (candidate steps per iteration) are identical and the
iterates agree to 1e-10 relative.  CR_MIXED_TF32: the solve reaches the relative gap with far
fewer sweeps than the constant step 1/L, and its dual objective agrees with the oracle's at the
same gap (both within the gap of the same optimum).
"""
import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gpu_trials(s, iters, max_sweeps=1000):
    """Runs candidate steps one at a time until `iters` iterations are accepted; returns the
    candidate count of every accepted iteration (read from the device-side counter)."""
    trials, last_k, since = [], s.gap()["k"], 0
    for _ in range(max_sweeps):
        s.step(1)
        since += 1
        k = s.gap()["k"]
        if k != last_k:
            assert k == last_k + 1
            trials.append(since)
            since, last_k = 0, k
            if k == iters:
                break
    return trials, last_k


# The adaptive steps grow to hundreds of times 1/L along the trajectory, so rounding
# differences between any two FP64 implementations are amplified by a factor of ~2-3 per
# iteration (measured: 1e-12 at k = 30, 1e-3 at k = 59 on the first case).  Decision-for-
# decision and 1e-10 agreement is checked over the first 30 iterations; beyond that the
# comparison is in outcome (the TF32 solve below).
@pytest.mark.parametrize("N,n,fam,gamma,seed,restart", [(200, 2, "sqnorm", 1e-3, 0, 0), (150, 5, "maxaff", 1e-4, 1, 0),
                                                          (200, 10, "lse", 1e-4, 2, 1)])
def test_fp64_adaptive_matches_oracle_decision_for_decision(N, n, fam, gamma, seed, restart):
    inst = cr_synth.make_instance(N, n, fam, 0.1, seed)
    L = oracle.lipschitz(inst.X, gamma)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_FP64,
                     step_rule=crgb.CR_STEP_ADAPTIVE, upsilon=2.0, restart=restart, graph_iters=0) as s:
        trials, k = _gpu_trials(s, 30)
        assert k == 30
        y, xi = s.primal()
        lam = s.lam()
        g = s.gap()
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L, adaptive=True, upsilon=2.0, restart=bool(restart))
    ref.step(k, log=False)
    assert trials == ref.trials
    y_r, xi_r = ref.primal()
    assert rel(y, y_r) <= 1e-10 and rel(xi, xi_r) <= 1e-10
    assert rel(lam, ref.theta) <= 1e-10
    # the next candidate tries s_k / upsilon unless rejections of iteration k + 1 are pending
    assert g["step"] * ref.s[0] / 2.0 <= 1.0 + 1e-12


def test_fp64_adaptive_graph_replay_equals_single_steps():
    inst = cr_synth.make_instance(180, 3, "sqnorm", 0.1, 3)
    L = oracle.lipschitz(inst.X, 1e-3)
    out = []
    for gi in (0, 16):
        with crgb.Solver(inst.X, inst.ybar, gamma=1e-3, lipschitz=L, precision=crgb.CR_FP64,
                         step_rule=crgb.CR_STEP_ADAPTIVE, graph_iters=gi) as s:
            s.step(3)
            s.step(45)
            y, xi = s.primal()
            out.append((y, xi, s.gap()["k"]))
    assert out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def _oracle_optimum(inst, gamma, L, tol):
    """The oracle's adaptive iteration with restart run to rel gap <= tol (checked every 100
    iterations, at most 40000)."""
    o = oracle.PAPG(inst.X, inst.ybar, gamma, L, adaptive=True, upsilon=2.0, restart=True)
    rms = float(np.sqrt(np.mean(inst.ybar ** 2)))
    N = inst.N
    for _ in range(400):
        o.step(100, log=False)
        d = o.dual()
        y, xi = o.primal()
        c = oracle.c_apply(inst.X, y, xi)
        inf = float(np.sqrt(np.sum(np.minimum(c, 0.0) ** 2) / (N * N - N)))
        if max(abs(d["r"] - d["g"]) / d["r"], inf / rms) <= tol:
            return d["g"], y
    raise AssertionError("oracle did not reach the reference gap")


@pytest.mark.parametrize("N,n,fam,seed", [(300, 8, "maxaff", 5), (400, 20, "lse", 4)])
def test_tf32_adaptive_solve_needs_fewer_sweeps_and_finds_the_optimum(N, n, fam, seed):
    inst = cr_synth.make_instance(N, n, fam, 0.1, seed)
    gamma, tol, cap = 1e-4, 1e-4, 80000
    L = oracle.lipschitz(inst.X, gamma)
    res = {}
    for rule in (crgb.CR_STEP_CONSTANT, crgb.CR_STEP_ADAPTIVE):
        with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_MIXED_TF32,
                         step_rule=rule, restart=int(rule == crgb.CR_STEP_ADAPTIVE), check_every=50) as s:
            ok, g = s.solve(tol, cap)
            y, _ = s.primal()
            res[rule] = (ok, g, y)
    ok_a, g_a, y_a = res[crgb.CR_STEP_ADAPTIVE]
    ok_c, g_c, _ = res[crgb.CR_STEP_CONSTANT]
    assert ok_a
    assert g_a["sweeps"] < (g_c["sweeps"] if ok_c else cap)
    # the adaptive trajectory is not followed iterate for iterate (see above).  The oracle
    # pins p* to 1e-5 (its own gap); the GPU's dual objective and its certified feasible
    # upper bound bracket it (weak duality: g(lambda) <= p* <= r(repair)), and the objective
    # sits within a few gap tolerances of it (rel_gap bounds r - g, and the infeasibility of
    # eta separately, so p* - g is not bounded by tol alone)
    g_ref, y_ref = _oracle_optimum(inst, gamma, L, 1e-5)
    assert g_a["dual_g"] <= g_ref * (1.0 + 1e-5)
    assert g_ref <= g_a["cert_primal"] * (1.0 + 1e-5)
    assert abs(g_a["dual_g"] - g_ref) <= 5 * tol * abs(g_ref)
    assert rel(y_a, y_ref) <= 1e-2


def test_adaptive_rejects_bad_options():
    inst = cr_synth.make_instance(50, 2, "sqnorm", 0.1, 6)
    with pytest.raises(crgb.CRError):
        crgb.Solver(inst.X, inst.ybar, precision=crgb.CR_FP64, step_rule=crgb.CR_STEP_ADAPTIVE, upsilon=1.0)
    with pytest.raises(crgb.CRError):
        crgb.Solver(inst.X, inst.ybar, precision=crgb.CR_FP32, step_rule=7)
