"""Continuation in gamma (Section 6) and checkpoint / resume.

* Checkpoint then resume in a fresh context continues bitwise like the uninterrupted run, in
  every precision and step rule (graphs on).
* A continuation stage is a warm start: FP64 iterates after gamma 1e-2 -> 1e-3 match the
  oracle's two P-APG runs (the second started from the first's theta) to 1e-10, and the step
  constant follows gamma.
* cr_solve_path reaches the final gamma's optimum (bracketed by the oracle's p*).
* cr_solve_continuation (Section 6's schedule, Section 5's stopping test per stage) ends
  delta_T-optimal and meets Eq. (delta-bound) against the oracle's optimum.
"""
import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb

pytestmark = pytest.mark.gpu

ADAPT = dict(step_rule=crgb.CR_STEP_ADAPTIVE, upsilon=2.0, restart=1)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision,extra", [(crgb.CR_FP64, {}), (crgb.CR_FP32, {}), (crgb.CR_MIXED_TF32, {}),
                                             (crgb.CR_MIXED_TF32, ADAPT), (crgb.CR_FP32, ADAPT),
                                             (crgb.CR_FP64, ADAPT)])
def test_checkpoint_resume_is_bitwise(precision, extra):
    inst = cr_synth.make_instance(700, 6, "maxaff", 0.1, 31)
    opts = dict(gamma=1e-4, precision=precision, graph_iters=8, **extra)
    with crgb.Solver(inst.X, inst.ybar, **opts) as a:
        a.step(23)
        buf = a.checkpoint()
        a.step(41)
        ya, xia = a.primal()
        la = a.lam(0, 64)
        ga = a.gap()
    with crgb.Solver(inst.X, inst.ybar, **opts) as b:
        b.step(5)  # state that the restore overwrites
        b.restore(buf)
        b.step(41)
        yb, xib = b.primal()
        lb = b.lam(0, 64)
        gb = b.gap()
    assert np.array_equal(ya, yb) and np.array_equal(xia, xib) and np.array_equal(la, lb)
    assert ga["k"] == gb["k"] and ga["sweeps"] == gb["sweeps"] and ga["dual_g"] == gb["dual_g"]


def test_restore_rejects_another_shape():
    a_inst = cr_synth.make_instance(300, 4, "sqnorm", 0.1, 32)
    b_inst = cr_synth.make_instance(301, 4, "sqnorm", 0.1, 33)
    with crgb.Solver(a_inst.X, a_inst.ybar, precision=crgb.CR_FP32) as a:
        a.step(3)
        buf = a.checkpoint()
    with crgb.Solver(b_inst.X, b_inst.ybar, precision=crgb.CR_FP32) as b:
        with pytest.raises(crgb.CRError):
            b.restore(buf)
    with crgb.Solver(a_inst.X, a_inst.ybar, precision=crgb.CR_FP32, **ADAPT) as c:
        with pytest.raises(crgb.CRError):
            c.restore(buf)
    # same shape and options, other data
    other = cr_synth.make_instance(300, 4, "sqnorm", 0.1, 99)
    with crgb.Solver(other.X, other.ybar, precision=crgb.CR_FP32) as d:
        with pytest.raises(crgb.CRError):
            d.restore(buf)
    # and the block restores into a fresh context on the same data
    with crgb.Solver(a_inst.X, a_inst.ybar, precision=crgb.CR_FP32) as e:
        e.restore(buf)
        assert e.k == 3


def test_continuation_stage_is_a_warm_start_fp64():
    inst = cr_synth.make_instance(150, 3, "sqnorm", 0.1, 34)
    g0, g1 = 1e-2, 1e-3
    o_mid = oracle.PAPG(inst.X, inst.ybar, g0, oracle.lipschitz(inst.X, g0))
    o_mid.step(60, log=False)
    d_mid = oracle.dual_obj(inst.X, inst.ybar, g1, o_mid.theta)  # theta^60 under the new gamma
    with crgb.Solver(inst.X, inst.ybar, gamma=g0, precision=crgb.CR_FP64) as s:
        s.step(60)
        s.set_gamma(g1)
        assert abs(s.L - oracle.lipschitz(inst.X, g1)) <= 1e-12 * s.L
        # the record describes lambda^k at the new gamma (the stop tests of a stage compare it)
        gm = s.gap()
        assert abs(gm["dual_g"] - d_mid["g"]) <= 1e-10 * abs(d_mid["g"])
        assert abs(gm["primal_r"] - d_mid["r"]) <= 1e-10 * abs(d_mid["r"])
        s.step(60)
        y, xi = s.primal()
        lam = s.lam()
    o0 = oracle.PAPG(inst.X, inst.ybar, g0, oracle.lipschitz(inst.X, g0))
    o0.step(60, log=False)
    o1 = oracle.PAPG(inst.X, inst.ybar, g1, oracle.lipschitz(inst.X, g1), theta0=o0.theta)
    o1.step(60, log=False)
    y_r, xi_r = o1.primal()
    assert rel(y, y_r) <= 1e-10 and rel(xi, xi_r) <= 1e-10 and rel(lam, o1.theta) <= 1e-10


def test_solve_path_reaches_the_final_optimum():
    inst = cr_synth.make_instance(500, 10, "lse", 0.1, 35)
    gammas, tols = [1e-2, 1e-3, 1e-4], [1e-3, 1e-3, 1e-4]
    with crgb.Solver(inst.X, inst.ybar, gamma=gammas[0], precision=crgb.CR_MIXED_TF32, check_every=50,
                     **ADAPT) as s:
        ok, g = s.solve_path(gammas, tols, 40000)
    assert ok
    L = oracle.lipschitz(inst.X, 1e-4)
    o = oracle.PAPG(inst.X, inst.ybar, 1e-4, L, adaptive=True, upsilon=2.0, restart=True)
    for _ in range(400):
        o.step(100, log=False)
        d = o.dual()
        if abs(d["r"] - d["g"]) / d["r"] <= 1e-6:
            break
    assert g["dual_g"] <= d["g"] * (1.0 + 1e-5)
    assert d["g"] <= g["cert_primal"] * (1.0 + 1e-5)


@pytest.fixture(scope="module")
def continuation_case():
    """Section 6's schedule on a 200-point instance: eps_t = 0.4 / 2^t, gamma_t = 0.04 eps_t,
    delta_t = 0.01 eps_t, four stages (gamma_4 = 1e-3, delta_4 = 2.5e-4), and the oracle's
    optimum of Eq. (dual-problem) at gamma_4 (its duality gap and infeasibility below 1e-8)."""
    inst = cr_synth.make_instance(200, 3, "maxaff", 0.1, 36)
    sched = dict(eps0=0.4, beta=2.0, kappa_gamma=0.04, kappa_delta=0.01, stages=4)
    eps_T = sched["eps0"] / sched["beta"] ** sched["stages"]
    gamma_T, delta_T = sched["kappa_gamma"] * eps_T, sched["kappa_delta"] * eps_T
    o = oracle.PAPG(inst.X, inst.ybar, gamma_T, oracle.lipschitz(inst.X, gamma_T), adaptive=True, upsilon=2.0,
                    restart=True)
    for _ in range(60):
        o.step(500, log=False)
        d = o.dual()
        y, xi = o.primal()
        c = oracle.certify(inst.X, inst.ybar, gamma_T, y, xi)
        if abs(d["lg"]) <= 1e-8 and np.sqrt(c["infeas_sq"] / (200 * 199)) <= 1e-8:
            break
    assert abs(d["lg"]) <= 1e-8 and np.sqrt(c["infeas_sq"] / (200 * 199)) <= 1e-8
    return inst, sched, gamma_T, delta_T, d


@pytest.mark.parametrize("precision,extra,infeas_tol", [(crgb.CR_FP64, {}, 1e-6), (crgb.CR_MIXED_TF32, ADAPT, 1e-5)])
def test_continuation_schedule_meets_the_delta_bound(continuation_case, precision, extra, infeas_tol):
    """Section 6's schedule with Section 5's stopping test at each stage (the infeasibility
    threshold above the precision's rounding floor of the pair pass): the last stage's
    multipliers are delta_T-optimal against the oracle's optimum, and Eq. (delta-bound),
    ||y - y*_gamma||^2 + gamma ||xi - xi*_gamma||^2 <= 2 (p*_gamma - g_gamma(lambda)), holds for
    the distance to the oracle's eta (p*_gamma - g_oracle <= 1e-8 taken from the oracle's gap)."""
    inst, sched, gamma_T, delta_T, d = continuation_case
    with crgb.Solver(inst.X, inst.ybar, gamma=0.1, precision=precision, check_every=25, **extra) as s:
        ok, g = s.solve_continuation(max_sweeps=100000, infeas_tol=infeas_tol, **sched)
        assert ok, repr(g)
        assert abs(s.L - oracle.lipschitz(inst.X, gamma_T)) <= 1e-12 * s.L
        y, xi = s.primal()
    assert abs(g["lagr_gap"]) <= delta_T or g["cert_primal"] - g["dual_g"] <= delta_T
    subopt = d["g"] + 1e-8 - g["dual_g"]  # >= p*_gamma - g_gamma(lambda)
    assert subopt <= delta_T, repr(g)
    dist = np.sqrt(np.sum((y - d["y"]) ** 2) + gamma_T * np.sum((xi - d["xi"]) ** 2))
    bound = np.sqrt(2.0 * subopt) + np.sqrt(2e-8)
    assert dist <= bound, (dist, bound)


def test_continuation_rejects_bad_schedules():
    inst = cr_synth.make_instance(64, 2, "sqnorm", 0.1, 37)
    with crgb.Solver(inst.X, inst.ybar, precision=crgb.CR_FP32) as s:
        for bad in (dict(beta=1.0), dict(eps0=0.0), dict(kappa_gamma=-1.0), dict(stages=0)):
            args = dict(eps0=0.1, beta=2.0, kappa_gamma=0.1, kappa_delta=0.1, stages=2, max_sweeps=10,
                        infeas_tol=1e-3)
            args.update(bad)
            with pytest.raises(crgb.CRError):
                s.solve_continuation(**args)
