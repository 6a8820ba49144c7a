"""Wide points, 32 < n <= CR_MAX_N (the paper's Section 5 workloads have n = 80): the wide
sweep, certificate pass and eigen solve of the step constant, against the FP64 oracle.

Tolerances as for narrow points: FP64 1e-10 on y, xi, g and Lambda iterate for iterate
(padded widths NP = 48, 80, 128 and ragged N); FP32 1e-4 on y and g, 1e-3 on xi.  The
adaptive step (Section 4) decides candidate for candidate like the oracle in FP64.
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


def _paper_instance(N, n, fam, seed):
    # Section 5's shape: x ~ N(0, 4 I), noise N(0, 100), 30% of the observations scaled by 1.3
    return cr_synth.make_instance(N, n, fam, 10.0, seed, x_dist="normal4", interior_frac=0.3)


@pytest.mark.parametrize("N,n,fam,seed", [(300, 80, "exp", 0), (161, 33, "quad", 1), (130, 128, "quad", 2),
                                          (257, 48, "sqnorm", 3)])
def test_fp64_wide_iterate_for_iterate(N, n, fam, seed):
    inst = _paper_instance(N, n, fam, seed) if fam != "sqnorm" else cr_synth.make_instance(N, n, fam, 0.1, seed)
    gamma = 1e-4
    L = oracle.lipschitz(inst.X, gamma)
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_FP64) as s:
        assert s.describe()["sweep"] == "wide-fp64"
        k = 0
        for it in (1, 5, 30):
            log = ref.step(it - k)
            s.step(it - k)
            k = it
            y, xi = s.primal()
            y_r, xi_r = ref.primal()
            g = s.gap()
            lam = s.lam()
            assert rel(y, y_r) <= 1e-10 and rel(xi, xi_r) <= 1e-10, (it, rel(y, y_r), rel(xi, xi_r))
            assert abs(g["dual_g"] - log["g"][-1]) <= 1e-10 * abs(log["g"][-1])
            assert rel(lam, ref.theta) <= 1e-10
            assert lam.min() >= 0.0 and np.abs(np.diag(lam)).max() == 0.0


@pytest.mark.parametrize("N,n,fam,seed", [(400, 80, "exp", 4), (333, 40, "quad", 5), (260, 128, "sqnorm", 6)])
def test_fp32_wide_iterate_for_iterate(N, n, fam, seed):
    inst = _paper_instance(N, n, fam, seed) if fam != "sqnorm" else cr_synth.make_instance(N, n, fam, 0.1, seed)
    gamma = 1e-4
    L = oracle.lipschitz(inst.X, gamma)
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_FP32) as s:
        assert s.describe()["sweep"] == "wide-fp32"
        k = 0
        for it in (1, 10, 100):
            log = ref.step(it - k)
            s.step(it - k)
            k = it
            y, xi = s.primal()
            y_r, xi_r = ref.primal()
            g = s.gap()
            assert rel(y, y_r) <= 1e-4 and rel(xi, xi_r) <= 1e-3, (it, rel(y, y_r), rel(xi, xi_r))
            assert abs(g["dual_g"] - log["g"][-1]) <= 1e-4 * abs(log["g"][-1])
            lam = s.lam()
            assert lam.min() >= 0.0 and np.abs(np.diag(lam)).max() == 0.0


def test_fp64_wide_adaptive_matches_oracle_decision_for_decision():
    inst = _paper_instance(180, 80, "quad", 7)
    gamma = 1e-4
    L = oracle.lipschitz(inst.X, gamma)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_FP64,
                     step_rule=crgb.CR_STEP_ADAPTIVE, upsilon=2.0, restart=1, graph_iters=0) as s:
        trials, last_k, since = [], 0, 0
        for _ in range(400):
            s.step(1)
            since += 1
            k = s.gap()["k"]
            if k != last_k:
                trials.append(since)
                since, last_k = 0, k
                if k == 30:
                    break
        y, xi = s.primal()
        lam = s.lam()
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L, adaptive=True, upsilon=2.0, restart=True)
    ref.step(30, log=False)
    assert trials == ref.trials
    y_r, xi_r = ref.primal()
    assert rel(y, y_r) <= 1e-10 and rel(xi, xi_r) <= 1e-10 and rel(lam, ref.theta) <= 1e-10


def test_fp32_wide_adaptive_reaches_the_oracle_optimum():
    inst = cr_synth.make_instance(220, 40, "lse", 0.1, 8)
    gamma = 1e-3
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, precision=crgb.CR_FP32, step_rule=crgb.CR_STEP_ADAPTIVE,
                     upsilon=2.0, restart=1, check_every=50) as s:
        ok, g = s.solve(1e-5, 60000)
    assert ok
    o = oracle.PAPG(inst.X, inst.ybar, gamma, oracle.lipschitz(inst.X, gamma), adaptive=True, upsilon=2.0,
                    restart=True)
    for _ in range(100):
        o.step(200, log=False)
        d = o.dual()
        if abs(d["r"] - d["g"]) <= 1e-7 * d["r"]:
            break
    # both dual objectives sit below p* and the GPU's certified repair above it
    assert g["dual_g"] <= d["g"] * (1.0 + 1e-5)
    assert d["g"] <= g["cert_primal"] * (1.0 + 1e-5)
    assert abs(g["dual_g"] - d["g"]) <= 1e-3 * d["g"]


@pytest.mark.parametrize("N,n", [(500, 33), (800, 80), (300, 128)])
@pytest.mark.parametrize("rule", ["hessian", "paper"])
def test_wide_lipschitz_matches_oracle(N, n, rule):
    inst = _paper_instance(N, n, "exp", 9)
    gamma = 1e-4
    Lr = oracle.lipschitz(inst.X, gamma, rule=rule)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma,
                     lipschitz_rule=crgb.CR_L_PAPER if rule == "paper" else crgb.CR_L_HESSIAN) as s:
        assert abs(s.L - Lr) <= 1e-10 * Lr
        assert s.L >= Lr * (1 - 1e-13)


@pytest.mark.parametrize("prec,tol", [(crgb.CR_FP64, 1e-9), (crgb.CR_FP32, 1e-4)])
def test_wide_certificate_and_infeasibility_match_oracle(prec, tol):
    inst = _paper_instance(350, 80, "quad", 10)
    gamma = 1e-4
    L = oracle.lipschitz(inst.X, gamma)
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=prec) as s:
        for it in (5, 100):
            ref.step(it - ref.k, log=False)
            s.step(it - s.k)
            y, xi = ref.primal()
            c = oracle.certify(inst.X, inst.ybar, gamma, y, xi)
            gap = s.gap()
            N = inst.N
            inf_ref = np.sqrt(c["infeas_sq"] / (N * N - N))
            assert abs(gap["infeas_norm"] - inf_ref) <= tol * max(inf_ref, 1e-12) + 1e-12
            assert abs(gap["cert_primal"] - c["P"]) <= tol * abs(c["P"])
            assert gap["cert_primal"] >= gap["dual_g"]


def test_wide_limits():
    inst = cr_synth.make_instance(64, 40, "sqnorm", 0.1, 11)
    with pytest.raises(crgb.CRError):
        crgb.Solver(inst.X, inst.ybar, precision=crgb.CR_MIXED_TF32)
    wide = cr_synth.make_instance(64, crgb.CR_MAX_N + 1, "sqnorm", 0.1, 12)
    with pytest.raises(crgb.CRError):
        crgb.Solver(wide.X, wide.ybar, precision=crgb.CR_FP64)
    b = crgb.Batch(precision=crgb.CR_FP32)
    try:
        with pytest.raises(crgb.CRError):
            b.add(inst.X, inst.ybar, 1e-4, 100)
    finally:
        b.close()
