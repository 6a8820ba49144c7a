"""Pins of the FP64 oracle to things other than itself (CPU only).

* the paper's matrices (Definition 1) built densely, and the spectral facts of
  Lemma "O1-constant" (sigma_max(A1) = sqrt(2N), ||T_l|| = sqrt(N));
* an exact dual solve by scipy's NNLS, itself checked by the KKT conditions;
* hand-derived worked examples (tests/golden/worked_examples.json);
* Theorem "rate" (Eq. primal-convergence) and the APG bound (Eq. apg-rate);
* noise-free convex data (Lemma 1 + Theorem "bound");
* weak duality and the feasibility of the certified repair.
Each is chosen so that a dropped term, a sign error or a transposed multiplier in
the oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import cr_synth
import oracle
from oracle import qp_dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _inst(N, n, seed, noise=0.1, family="sqnorm"):
    return cr_synth.make_instance(N, n, family, noise, seed)


def _run_to_convergence(X, yb, gamma, iters):
    L = oracle.lipschitz(X, gamma)
    o = oracle.PAPG(X, yb, gamma, L)
    log = o.step(iters)
    return o, log, L


# --------------------------------------------------------------------------- operators
@pytest.mark.parametrize("N,n,seed", [(5, 1, 0), (7, 3, 1), (9, 2, 2), (5, 80, 3), (4, 128, 4)])
def test_operators_match_definition1(N, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(N, n))
    A1, A2 = qp_dense.dense_A(X)
    y = rng.standard_normal(N)
    xi = rng.standard_normal((N, n))
    ce = oracle.c_apply(X, y, xi)
    assert np.allclose(qp_dense.theta_mat_to_vec(ce), A1 @ y + A2 @ xi.ravel(), atol=1e-13)
    assert np.all(np.diag(ce) == 0.0)
    th = np.abs(rng.standard_normal((N, N)))
    np.fill_diagonal(th, 0.0)
    a, b = oracle.ct_apply(X, th)
    tv = qp_dense.theta_mat_to_vec(th)
    assert np.allclose(a, A1.T @ tv, atol=1e-13)
    assert np.allclose(b.ravel(), A2.T @ tv, atol=1e-13)
    # a diagonal entry must not leak into C^T theta
    th2 = th.copy()
    np.fill_diagonal(th2, 5.0)
    a2, b2 = oracle.ct_apply(X, th2)
    assert np.array_equal(a2, a) and np.array_equal(b2, b)


@pytest.mark.parametrize("N", [3, 6, 11])
def test_lemma_o1_spectra(N):
    # Lemma "O1-constant": sigma_max(A1) = sqrt(2N), ||T_l|| = sqrt(N)
    X = np.random.default_rng(N).uniform(-1, 1, size=(N, 2))
    A1, A2 = qp_dense.dense_A(X)
    assert np.isclose(np.linalg.norm(A1, 2) ** 2, 2 * N, rtol=1e-12)
    for l in range(N):
        assert np.isclose(np.linalg.norm(qp_dense.T_matrix(l, N), 2) ** 2, N, rtol=1e-12)
    # sigma_max(A2) (block diagonal) against the oracle's per-block eigenvalues
    assert np.isclose(np.linalg.norm(A2, 2) ** 2, oracle.a2_sigma_sq(X), rtol=1e-11)
    # sigma_max(A2) <= B_x N
    Bx = np.sqrt((X ** 2).sum(1).max())
    assert np.linalg.norm(A2, 2) <= Bx * N + 1e-12


@pytest.mark.parametrize("gamma,N,n", [(1e-1, 9, 3), (1e-3, 9, 3), (1e-4, 9, 3), (1e-4, 6, 80), (1e-3, 5, 128)])
def test_lipschitz_is_tight_upper_bound(gamma, N, n):
    X = np.random.default_rng(4).uniform(-1, 1, size=(N, n))
    A1, A2 = qp_dense.dense_A(X)
    C = np.hstack([A1, A2])
    Ginv = np.concatenate([np.ones(N), np.full(N * n, 1.0 / gamma)])
    lam = np.linalg.eigvalsh((C * Ginv) @ C.T)[-1]
    L = oracle.lipschitz(X, gamma)
    s2 = np.linalg.norm(A2, 2) ** 2
    assert L >= lam * (1 - 1e-12)
    assert L <= lam * (1 + 2 * N * gamma / s2) * (1 + 1e-12)
    Lp = oracle.lipschitz(X, gamma, rule="paper")
    assert Lp >= np.linalg.norm(C, 2) ** 2 / gamma * (1 - 1e-12)


# --------------------------------------------------------------------------- exact solves
def _check_kkt(ref, X, yb, gamma, tol=1e-9):
    """The NNLS answer is the optimum of Eq. (regularize): feasible, complementary,
    stationary by construction."""
    ce = oracle.c_apply(X, ref["y"], ref["xi"])
    np.fill_diagonal(ce, 0.0)
    assert ce.min() >= -tol
    th = ref["theta"]
    assert th.min() >= 0
    assert abs(np.sum(th * ce)) <= tol * max(1.0, ref["p"])


@pytest.mark.parametrize("N,n,seed,gamma", [(6, 1, 0, 1e-2), (8, 2, 1, 1e-2), (10, 2, 2, 3e-2),
                                            (7, 3, 3, 1e-1)])
def test_papg_reaches_exact_solution(N, n, seed, gamma):
    inst = _inst(N, n, seed)
    X, yb = inst.X, inst.ybar
    ref = qp_dense.solve_nnls(X, yb, gamma)
    _check_kkt(ref, X, yb, gamma)
    o, log, L = _run_to_convergence(X, yb, gamma, 30000)
    y, xi = o.primal()
    assert abs(log["g"][-1] - ref["p"]) <= 1e-8 * max(1.0, ref["p"])
    assert np.abs(y - ref["y"]).max() <= 1e-8
    # primal objective at eta(theta^k) also converges
    assert abs(log["r"][-1] - ref["p"]) <= 1e-8 * max(1.0, ref["p"])


def test_worked_examples():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        X = np.array(c["X"], dtype=float)
        yb = np.array(c["ybar"], dtype=float)
        gamma = c["gamma"]
        # the listed multipliers certify the listed solution
        a, b = oracle.ct_apply(X, np.array(c["theta"]))
        assert np.allclose(np.array(c["y"]) - yb, a, atol=1e-15)
        assert np.allclose(gamma * np.array(c["xi"]), b, atol=1e-15)
        # the oracle iteration reaches it
        o, log, L = _run_to_convergence(X, yb, gamma, 20000)
        y, xi = o.primal()
        assert np.allclose(y, c["y"], atol=1e-9), c["name"]
        assert abs(log["g"][-1] - c["p"]) <= 1e-10, c["name"]
        # xi converges at the rate of Theorem "rate": gamma ||xi - xi*||^2 <= 2 (p* - g)
        gap = max(c["p"] - log["g"][-1], 0.0)
        assert gamma * np.sum((xi - np.array(c["xi"])) ** 2) <= 2 * gap + 1e-24, c["name"]
        assert np.allclose(xi, c["xi"], atol=1e-6), c["name"]
        # the exact dual solve agrees
        ref = qp_dense.solve_nnls(X, yb, gamma)
        assert abs(ref["p"] - c["p"]) <= 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_two_point_closed_form(seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(2, 3))
    yb = rng.standard_normal(2)
    gamma = 0.05
    cf = qp_dense.n2_closed_form(X, yb, gamma)
    o, log, L = _run_to_convergence(X, yb, gamma, 5000)
    y, xi = o.primal()
    assert np.allclose(y, cf["y"], atol=1e-10)
    assert np.allclose(xi, cf["xi"], atol=1e-9)
    assert abs(log["g"][-1] - cf["p"]) <= 1e-12
    assert abs(qp_dense.solve_nnls(X, yb, gamma)["p"] - cf["p"]) <= 1e-12


# --------------------------------------------------------------------------- bounds
def test_theorem_rate_and_apg_bound():
    N, n, gamma = 8, 2, 1e-2
    inst = _inst(N, n, 5)
    X, yb = inst.X, inst.ybar
    ref = qp_dense.solve_nnls(X, yb, gamma)
    L = oracle.lipschitz(X, gamma)
    o = oracle.PAPG(X, yb, gamma, L)
    th_star_sq = np.sum(ref["theta"] ** 2)
    for k in range(1, 301):
        log = o.step(1)
        g = log["g"][0]
        y, xi = o.primal()
        lhs = np.sum((y - ref["y"]) ** 2) + gamma * np.sum((xi - ref["xi"]) ** 2)
        # Theorem "rate" (Eq. primal-convergence)
        assert lhs <= 2 * (ref["p"] - g) + 1e-12
        # weak duality
        assert g <= ref["p"] + 1e-12
        # Eq. (apg-rate) with theta^0 = 0
        assert ref["p"] - g <= 2 * L * th_star_sq / (k + 1) ** 2 + 1e-12
        assert o.theta.min() >= 0 and np.all(np.diag(o.theta) == 0)


def test_dual_gradient_ascent_is_slower():
    N, n, gamma = 10, 2, 1e-2
    inst = _inst(N, n, 6)
    X, yb = inst.X, inst.ybar
    ref = qp_dense.solve_nnls(X, yb, gamma)
    L = oracle.lipschitz(X, gamma)
    acc = oracle.PAPG(X, yb, gamma, L, accel=True)
    pla = oracle.PAPG(X, yb, gamma, L, accel=False)
    ga = acc.step(400)["g"][-1]
    gp = pla.step(400)["g"][-1]
    assert ref["p"] - ga < ref["p"] - gp
    assert gp <= ref["p"] + 1e-12 and ga <= ref["p"] + 1e-12


@pytest.mark.parametrize("gamma", [1e-1, 1e-2, 1e-3])
def test_noise_free_convex_data(gamma):
    # ybar = ||x||^2 exactly: y* = ybar and xi = 2x is feasible, so ||xi*|| <= ||2X||_F;
    # Theorem "bound": ||y_{gamma,delta} - y*|| <= ||xi*|| sqrt(gamma) + sqrt(2 delta)
    inst = cr_synth.make_instance(12, 2, "sqnorm", 0.0, 7)
    X, yb = inst.X, inst.ybar
    ref = qp_dense.solve_nnls(X, yb, gamma)
    o, log, L = _run_to_convergence(X, yb, gamma, 4000)
    y, _ = o.primal()
    delta = max(ref["p"] - log["g"][-1], 0.0)
    bound = np.linalg.norm(2 * X) * np.sqrt(gamma) + np.sqrt(2 * delta)
    assert np.linalg.norm(y - yb) <= bound + 1e-12
    # and the Hoelder estimate itself at the exact solution
    assert np.linalg.norm(ref["y"] - yb) <= np.linalg.norm(2 * X) * np.sqrt(gamma) + 1e-9


def test_certified_repair_is_feasible_upper_bound():
    N, n, gamma = 9, 2, 1e-2
    inst = _inst(N, n, 8)
    X, yb = inst.X, inst.ybar
    ref = qp_dense.solve_nnls(X, yb, gamma)
    L = oracle.lipschitz(X, gamma)
    o = oracle.PAPG(X, yb, gamma, L)
    for _ in range(6):
        log = o.step(50)
        y, xi = o.primal()
        c = oracle.certify(X, yb, gamma, y, xi)
        xr = xi[c["m"]]
        ce = oracle.c_apply(X, c["yrep"], xr)
        np.fill_diagonal(ce, 0.0)
        assert ce.min() >= -1e-12                     # feasible repair
        assert c["P"] >= ref["p"] - 1e-12              # upper bound
        assert log["g"][-1] <= ref["p"] + 1e-12        # lower bound
        # infeasibility of eta(theta^k) recomputed from the pair values
        ce0 = oracle.c_apply(X, y, xi)
        np.fill_diagonal(ce0, 0.0)
        assert np.isclose(c["infeas_sq"], np.sum(np.minimum(ce0, 0) ** 2), rtol=1e-12, atol=1e-300)
    # a feasible input is returned unchanged
    c = oracle.certify(X, yb, gamma, ref["y"], ref["xi"])
    assert np.allclose(c["yrep"], ref["y"], atol=1e-9)


def test_dual_obj_identities():
    # g = r - <theta, C eta> and the closed form -1/2||a||^2 - a.ybar - ||b||^2/(2 gamma)
    N, n, gamma = 7, 2, 1e-2
    inst = _inst(N, n, 9)
    rng = np.random.default_rng(0)
    th = np.abs(rng.standard_normal((N, N))) * 1e-2
    np.fill_diagonal(th, 0.0)
    d = oracle.dual_obj(inst.X, inst.ybar, gamma, th)
    a, b = oracle.ct_apply(inst.X, th)
    g_cf = -0.5 * a @ a - a @ inst.ybar - np.sum(b * b) / (2 * gamma)
    assert np.isclose(d["g"], g_cf, rtol=1e-12, atol=1e-15)
    assert np.isclose(d["r"] - d["lg"], d["g"], rtol=1e-12, atol=1e-15)
    # brute force: g(theta) = min over eta of the Lagrangian, checked at random perturbations
    A1, A2 = qp_dense.dense_A(inst.X)
    tv = qp_dense.theta_mat_to_vec(th)

    def lag(y, xi):
        return (0.5 * np.sum((y - inst.ybar) ** 2) + 0.5 * gamma * np.sum(xi ** 2)
                - tv @ (A1 @ y + A2 @ xi.ravel()))

    base = lag(d["y"], d["xi"])
    assert np.isclose(base, d["g"], rtol=1e-12)
    for _ in range(20):
        dy = rng.standard_normal(N) * 1e-3
        dx = rng.standard_normal((N, n)) * 1e-3
        assert lag(d["y"] + dy, d["xi"] + dx) >= base - 1e-15


# ---------------------------------------------------------------- adaptive step (Section 4)
def test_adaptive_check_is_the_quadratic_identity():
    """g_gamma is a concave quadratic in theta, so the left side of Eq. (adaptive-check) minus
    g(theta~) minus the linear term is exactly -1/2 (||da||^2 + ||db||^2 / gamma) with
    (da, db) = C^T (theta - theta~); the GPU evaluates the check in that form."""
    rng = np.random.default_rng(7)
    inst = cr_synth.make_instance(9, 3, "maxaff", 0.1, 2)
    gamma = 1e-2
    for _ in range(3):
        tt = rng.random((9, 9)) * 0.3
        th = np.maximum(0.0, tt + rng.normal(0, 0.2, (9, 9)))
        np.fill_diagonal(tt, 0.0)
        np.fill_diagonal(th, 0.0)
        g = oracle.dual_obj(inst.X, inst.ybar, gamma, th)["g"]
        dt = oracle.dual_obj(inst.X, inst.ybar, gamma, tt)
        ceta = oracle.c_apply(inst.X, dt["y"], dt["xi"])        # grad g(theta~) = -C eta(theta~)
        lin = float(np.sum(-ceta * (th - tt)))
        da, db = oracle.ct_apply(inst.X, th - tt)
        quad = -0.5 * (float(da @ da) + float(np.sum(db * db)) / gamma)
        assert abs((g - dt["g"] - lin) - quad) <= 1e-10 * max(1.0, abs(quad))


def test_adaptive_oracle_follows_the_step_rule_and_reaches_the_optimum():
    """s_k = s_{k-1} upsilon^(l_k - 1) with s_0 = L (so log_upsilon(s_K / L) = sum (l_k - 1)),
    and the iterates reach the exact dense-QP solution like the constant step."""
    inst = cr_synth.make_instance(7, 2, "sqnorm", 0.1, 4)
    gamma = 1e-2
    L = oracle.lipschitz(inst.X, gamma)
    o = oracle.PAPG(inst.X, inst.ybar, gamma, L, adaptive=True, upsilon=2.0)
    o.step(3000, log=False)
    tr = np.array(o.trials)
    assert tr.min() >= 1
    expo = np.log(o.s[0] / L) / np.log(2.0)
    assert abs(expo - float(np.sum(tr - 2))) <= 1e-9
    ref = qp_dense.solve_nnls(inst.X, inst.ybar, gamma)
    y, xi = o.primal()
    assert np.linalg.norm(y - ref["y"]) <= 1e-6 * np.linalg.norm(ref["y"])
    d = o.dual()
    assert abs(d["g"] - ref["p"]) <= 1e-8 * abs(ref["p"])
    # the adaptive steps are longer than 1/L on this instance
    assert o.s[0] < L


def test_adaptive_step_needs_fewer_iterations():
    inst = cr_synth.make_instance(60, 2, "sqnorm", 0.1, 5)
    gamma = 1e-3
    L = oracle.lipschitz(inst.X, gamma)
    res = {}
    for ad in (False, True):
        o = oracle.PAPG(inst.X, inst.ybar, gamma, L, adaptive=ad)
        o.step(400, log=False)
        d = o.dual()
        res[ad] = (d["g"], abs(d["r"] - d["g"]) / d["r"])
    # the dual objective rises faster (both increase towards p*) and the gap is smaller
    assert res[True][0] > res[False][0]
    assert res[True][1] < res[False][1]


def test_adaptive_with_restart_reaches_the_optimum():
    """Function-value restart (t reset when g decreases) keeps the fixed point: the iterates
    reach the exact dense-QP solution."""
    inst = cr_synth.make_instance(8, 2, "maxaff", 0.1, 6)
    gamma = 1e-2
    L = oracle.lipschitz(inst.X, gamma)
    o = oracle.PAPG(inst.X, inst.ybar, gamma, L, adaptive=True, upsilon=2.0, restart=True)
    o.step(3000, log=False)
    ref = qp_dense.solve_nnls(inst.X, inst.ybar, gamma)
    y, _ = o.primal()
    assert np.linalg.norm(y - ref["y"]) <= 1e-6 * np.linalg.norm(ref["y"])
    assert abs(o.dual()["g"] - ref["p"]) <= 1e-8 * abs(ref["p"])
