"""Adaptive step size (with momentum restart) in the FP32 TMA sweep, the batched work-list and
the serving runtime: one instance solved alone, in a batch and in the server gives bitwise the
same iterates; a batch retires every instance at its gap with fewer sweeps than the constant
step; the FP32 path reaches the oracle's optimum."""
import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb

pytestmark = pytest.mark.gpu

ADAPT = dict(step_rule=crgb.CR_STEP_ADAPTIVE, upsilon=2.0, restart=1)


def test_fp32_single_adaptive_reaches_the_optimum():
    inst = cr_synth.make_instance(400, 6, "maxaff", 0.1, 11)
    gamma, tol = 1e-4, 1e-4
    L = oracle.lipschitz(inst.X, gamma)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_FP32, check_every=50,
                     **ADAPT) as s:
        assert s.describe()["sweep"] == "tma"
        ok, g = s.solve(tol, 60000)
    assert ok
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L, adaptive=True, upsilon=2.0, restart=True)
    for _ in range(300):
        ref.step(100, log=False)
        d = ref.dual()
        if abs(d["r"] - d["g"]) / d["r"] <= 1e-6:
            break
    assert g["dual_g"] <= d["g"] * (1.0 + 1e-5)
    assert d["g"] <= g["cert_primal"] * (1.0 + 1e-5)


def test_batch_adaptive_bitwise_matches_single():
    insts = [cr_synth.make_instance(N, n, "sqnorm", 0.1, 20 + i) for i, (N, n) in
             enumerate([(300, 2), (517, 5), (129, 12), (800, 3)])]
    solo = []
    for inst in insts:
        with crgb.Solver(inst.X, inst.ybar, gamma=1e-4, precision=crgb.CR_FP32, tile_cols=512, graph_iters=0,
                         **ADAPT) as s:
            s.step(37)
            solo.append(s.primal())
    with crgb.Batch(tile_cols=512, gamma=1e-4, graph_iters=0, check_every=1000, **ADAPT) as b:
        ids = [b.add(i.X, i.ybar, tol=0.0, max_iter=10 ** 6) for i in insts]
        b.step(37)
        for i, (y, xi) in zip(ids, solo):
            yb, xib = b.primal(i)
            assert np.array_equal(yb, y) and np.array_equal(xib, xi)


def test_batch_adaptive_retires_with_fewer_sweeps():
    insts = cr_synth.batch_workload(24, seed=3)
    res = {}
    for name, extra in (("const", {}), ("adapt", ADAPT)):
        with crgb.Batch(tile_cols=512, gamma=1e-4, graph_iters=20, check_every=100, **extra) as b:
            ids = [b.add(i.X, i.ybar, tol=1e-4, max_iter=60000) for i in insts]
            b.run()
            polls = [b.poll(i) for i in ids]
        res[name] = polls
    conv_a = sum(st == 0 for _, st, _ in res["adapt"])
    conv_c = sum(st == 0 for _, st, _ in res["const"])
    assert conv_a >= conv_c and conv_a >= 20
    sw_a = sum(info["sweeps"] for _, _, info in res["adapt"])
    sw_c = sum(info["sweeps"] for _, _, info in res["const"])
    assert sw_a < sw_c


def test_served_adaptive_results_equal_alone():
    """Under the adaptive step the served result is the instance solved alone for the same
    number of sweeps (the accept/reject decisions are the instance's own)."""
    import time
    rng = np.random.default_rng(4)
    insts = [cr_synth.make_instance(int(rng.integers(500, 1500)), int(rng.integers(2, 10)),
                                    ["sqnorm", "maxaff", "lse"][r % 3], 0.1, 2000 + r) for r in range(6)]
    gamma = 1e-3
    with crgb.Server(tile_cols=512, mem_cap_bytes=8 << 30, max_active=64, gamma=gamma, check_every=25, graph_iters=4,
                     **ADAPT) as srv:
        ids = []
        for inst in insts:
            ids.append(srv.submit(inst.X, inst.ybar, tol=1e-4, max_iter=3000))
            time.sleep(0.02)
        for r in ids:
            srv.wait(r, 300)
        res = [(srv.poll(r), srv.result(r)) for r in ids]
    for inst, ((state, status, info, lat), (y, xi)) in zip(insts, res):
        assert state == 2 and status in (0, 4)
        with crgb.Solver(inst.X, inst.ybar, gamma=gamma, tile_cols=512, graph_iters=0, **ADAPT) as s:
            s.step(int(info["sweeps"]))
            ys, xis = s.primal()
            assert s.gap()["k"] == info["k"]
        assert np.array_equal(y, ys) and np.array_equal(xi, xis), (inst.N, inst.n)
