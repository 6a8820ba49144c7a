"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative 2-norm errors against the oracle, written per test):
  FP64 mode      1e-10 on y, xi, g and on Lambda (iterate for iterate)
  FP32 modes     1e-4 on y, 1e-3 on xi, 1e-4 on g (Lambda stored in FP32: ~6e-8 per
                 element; the residual u_i - y_j + xi_i.x_j is formed with hi+lo y and u)
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


def _run_pair(inst, gamma, iters_list, precision, accelerate=True, graph_iters=32, tile_cols=0,
              check_lambda=True):
    L = oracle.lipschitz(inst.X, gamma)
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L, accel=accelerate)
    out = []
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=precision,
                     accelerate=int(accelerate), graph_iters=graph_iters, tile_cols=tile_cols) as s:
        k = 0
        for it in iters_list:
            log = ref.step(it - k)
            s.step(it - k)
            k = it
            y_r, xi_r = ref.primal()
            y, xi = s.primal()
            gap = s.gap()
            rec = dict(k=it, ey=rel(y, y_r), exi=rel(xi, xi_r),
                       eg=abs(gap["dual_g"] - log["g"][-1]) / max(abs(log["g"][-1]), 1e-300),
                       gap=gap, g_ref=log["g"][-1], r_ref=log["r"][-1])
            if check_lambda:
                lam = s.lam()
                rec["elam"] = rel(lam, ref.theta)
                rec["lam_min"] = float(lam.min())
                rec["lam_diag"] = float(np.abs(np.diag(lam)).max())
            out.append(rec)
    return out


@pytest.mark.parametrize("N,n,seed", [(200, 2, 0), (333, 3, 1), (129, 7, 2), (517, 10, 3), (64, 20, 4),
                                      (300, 32, 5), (2, 1, 6), (3, 2, 7)])
def test_fp64_iterate_for_iterate(N, n, seed):
    inst = cr_synth.make_instance(N, n, "sqnorm", 0.1, seed)
    for rec in _run_pair(inst, 1e-3, [1, 2, 5, 20, 60], crgb.CR_FP64):
        assert rec["ey"] <= 1e-10, rec
        assert rec["exi"] <= 1e-10, rec
        assert rec["eg"] <= 1e-10, rec
        assert rec["elam"] <= 1e-10, rec
        assert rec["lam_min"] >= 0.0 and rec["lam_diag"] == 0.0


def test_fp64_sqnorm_N200_500_iterations():
    inst = cr_synth.workload("sqnorm_N200_n2")
    for rec in _run_pair(inst, 1e-4, [100, 500], crgb.CR_FP64):
        assert rec["ey"] <= 1e-10 and rec["exi"] <= 1e-10 and rec["eg"] <= 1e-10, rec
        assert rec["elam"] <= 1e-10, rec


@pytest.mark.parametrize("N,n,fam,seed", [(1000, 10, "maxaff", 0), (777, 20, "lse", 1), (450, 2, "sqnorm", 2),
                                          (300, 16, "sqnorm", 3)])
def test_fp32_iterate_for_iterate(N, n, fam, seed):
    inst = cr_synth.make_instance(N, n, fam, 0.05, seed)
    for rec in _run_pair(inst, 1e-4, [1, 10, 100], crgb.CR_FP32):
        assert rec["ey"] <= 1e-4, rec
        assert rec["exi"] <= 1e-3, rec
        assert rec["eg"] <= 1e-4, rec
        assert rec["lam_min"] >= 0.0 and rec["lam_diag"] == 0.0


def test_dual_gradient_ascent_mode():
    inst = cr_synth.make_instance(150, 3, "sqnorm", 0.1, 9)
    for rec in _run_pair(inst, 1e-3, [10, 50], crgb.CR_FP64, accelerate=False):
        assert rec["ey"] <= 1e-10 and rec["elam"] <= 1e-10, rec


@pytest.mark.parametrize("tile_cols", [128, 256, 384])
def test_column_splits_do_not_change_results(tile_cols):
    inst = cr_synth.make_instance(700, 5, "sqnorm", 0.1, 11)
    for rec in _run_pair(inst, 1e-3, [7, 30], crgb.CR_FP64, tile_cols=tile_cols):
        assert rec["ey"] <= 1e-10 and rec["elam"] <= 1e-10, rec


def test_graph_replay_is_bitwise_identical():
    inst = cr_synth.make_instance(900, 6, "maxaff", 0.05, 12)
    L = oracle.lipschitz(inst.X, 1e-4)
    res = []
    for g in (0, 8, 32):
        with crgb.Solver(inst.X, inst.ybar, gamma=1e-4, lipschitz=L, graph_iters=g) as s:
            s.step(3)
            s.step(70)
            y, xi = s.primal()
            res.append((y, xi, s.lam(0, 50)))
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            assert np.array_equal(a, b)


def test_runs_are_deterministic():
    inst = cr_synth.make_instance(1500, 10, "maxaff", 0.05, 13)
    outs = []
    for _ in range(2):
        with crgb.Solver(inst.X, inst.ybar, gamma=1e-4) as s:
            s.step(25)
            outs.append(s.primal())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("N,n", [(200, 2), (1000, 10), (333, 31), (5000, 20)])
@pytest.mark.parametrize("rule", ["hessian", "paper"])
def test_lipschitz_matches_oracle(N, n, rule):
    inst = cr_synth.make_instance(N, n, "lse", 0.1, 14)
    gamma = 1e-4
    Lr = oracle.lipschitz(inst.X, gamma, rule=rule)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma,
                     lipschitz_rule=crgb.CR_L_PAPER if rule == "paper" else crgb.CR_L_HESSIAN) as s:
        assert abs(s.L - Lr) / Lr <= 1e-10
        assert s.L >= Lr * (1 - 1e-13)


@pytest.mark.parametrize("prec,tol", [(crgb.CR_FP64, 1e-9), (crgb.CR_FP32, 1e-4)])
def test_certificate_and_infeasibility_match_oracle(prec, tol):
    inst = cr_synth.make_instance(420, 4, "sqnorm", 0.1, 15)
    gamma = 1e-3
    L = oracle.lipschitz(inst.X, gamma)
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=prec) as s:
        for it in (5, 200):
            ref.step(it - ref.k, log=False)
            s.step(it - s.k)
            y, xi = ref.primal()
            c = oracle.certify(inst.X, inst.ybar, gamma, y, xi)
            d = ref.dual()
            gap = s.gap()
            N = inst.N
            inf_ref = np.sqrt(c["infeas_sq"] / (N * N - N))
            assert abs(gap["infeas_norm"] - inf_ref) <= tol * max(inf_ref, 1e-12) + 1e-12
            assert abs(gap["cert_primal"] - c["P"]) <= tol * abs(c["P"])
            assert abs(gap["lagr_gap"] - d["lg"]) <= tol * max(abs(d["lg"]), abs(d["r"]))
            assert gap["cert_primal"] >= gap["dual_g"]


def test_solve_reaches_tolerance_like_oracle():
    inst = cr_synth.workload("sqnorm_N200_n2")
    gamma = 1e-2
    L = oracle.lipschitz(inst.X, gamma)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_FP64,
                     check_every=50) as s:
        ok, rec = s.solve(1e-4, 200000)
        assert ok, rec
        k = s.k
        y, _ = s.primal()
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L)
    log = ref.step(k)
    y_r, _ = ref.primal()
    assert rel(y, y_r) <= 1e-9
    assert abs(rec["dual_g"] - log["g"][-1]) <= 1e-9 * abs(log["g"][-1])
    assert abs(rec["primal_r"] - log["r"][-1]) <= 1e-9 * abs(log["r"][-1])


@pytest.mark.parametrize("bad", ["N1", "n_over", "gamma0", "nanX", "infy", "odd_graph"])
def test_invalid_inputs_are_rejected(bad):
    inst = cr_synth.make_instance(10, 2, "sqnorm", 0.1, 0)
    X, y, kw = inst.X.copy(), inst.ybar.copy(), {}
    if bad == "N1":
        X, y = X[:1], y[:1]
    elif bad == "n_over":
        X = np.zeros((10, crgb.CR_MAX_N + 1))
    elif bad == "gamma0":
        kw["gamma"] = 0.0
    elif bad == "nanX":
        X[3, 1] = np.nan
    elif bad == "infy":
        y[2] = np.inf
    elif bad == "odd_graph":
        kw["graph_iters"] = 3
    with pytest.raises(crgb.CRError) as e:
        crgb.Solver(X, y, **kw)
    assert e.value.status == 1


def test_device_inputs_and_outputs():
    import torch
    inst = cr_synth.make_instance(256, 8, "maxaff", 0.05, 16)
    Xd = torch.tensor(inst.X, device="cuda")
    yd = torch.tensor(inst.ybar, device="cuda")
    gamma = 1e-3
    with crgb.Solver(Xd, yd, gamma=gamma) as s1, crgb.Solver(inst.X, inst.ybar, gamma=gamma) as s2:
        s1.step(30)
        s2.step(30)
        y1, xi1 = s1.primal(device=True)
        y2, xi2 = s2.primal()
        assert np.array_equal(y1.cpu().numpy(), y2) and np.array_equal(xi1.cpu().numpy(), xi2)
        lam = s1.lam(10, 20, device=True)
        assert np.array_equal(lam.cpu().numpy(), s2.lam(10, 20))
