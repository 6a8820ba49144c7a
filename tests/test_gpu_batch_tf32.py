"""Mixed-precision batches: the tensor-core sweep over a work-list of many instances.

With precision CR_MIXED_TF32 every instance with n <= 31 runs the tensor-core sweep (all of
them in one persistent launch over (instance, 128-row block, column split) items) and an
n = 32 instance the FP32 sweep.  Each instance computes in the batch exactly what it
computes alone with the same column-split width, so:

* a batch equals the single-instance runs bitwise (constant and adaptive step, instances
  that join mid-way, one n = 32 instance on the FP32 sweep beside the tensor-core ones);
* converged batch results agree with the FP64 oracle run for the same number of
  iterations at the reduced-precision tolerances (1e-4 on y, 1e-3 on xi, 1e-4 on g).
"""
import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb

pytestmark = pytest.mark.gpu

TF32 = crgb.CR_MIXED_TF32
# ragged row blocks (N not a multiple of 128), one-chunk tails, n from 1 to 32
SHAPES = [(300, 3), (517, 7), (1000, 10), (128, 16), (777, 2), (2048, 31), (95, 20), (1500, 5), (260, 32),
          (40, 1)]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _instances(shapes, seed0=500, family="sqnorm"):
    return [cr_synth.make_instance(N, n, family, 0.1, seed0 + i) for i, (N, n) in enumerate(shapes)]


def _single(inst, iters, **kw):
    prec = TF32 if inst.n <= crgb.CR_MAX_N_TF32 else crgb.CR_FP32
    with crgb.Solver(inst.X, inst.ybar, gamma=1e-4, tile_cols=512, graph_iters=0, precision=prec, **kw) as s:
        if prec == TF32:
            assert s.describe()["sweep"] == "tcgen05"
        s.step(iters)
        y, xi = s.primal()
        return y, xi, s.gap()


@pytest.mark.parametrize("rule", [crgb.CR_STEP_CONSTANT, crgb.CR_STEP_ADAPTIVE])
def test_tf32_batch_bitwise_matches_single(rule):
    insts = _instances(SHAPES)
    with crgb.Batch(tile_cols=512, gamma=1e-4, graph_iters=8, precision=TF32, step_rule=rule) as b:
        ids = [b.add(i.X, i.ybar, tol=0.0, max_iter=10**9) for i in insts]
        b.step(3)
        b.step(37)
        outs = [b.primal(i) for i in ids]
        infos = [b.poll(i)[2] for i in ids]
    for inst, (y, xi), info in zip(insts, outs, infos):
        ys, xis, gs = _single(inst, 40, step_rule=rule)
        assert np.array_equal(y, ys) and np.array_equal(xi, xis), (inst.N, inst.n, rel(y, ys), rel(xi, xis))
        assert info["k"] == gs["k"] and info["dual_g"] == gs["dual_g"]


def test_tf32_batch_instances_added_midway():
    insts = _instances(SHAPES[:6], seed0=600)
    with crgb.Batch(tile_cols=512, gamma=1e-4, graph_iters=4, precision=TF32) as b:
        ids = [b.add(i.X, i.ybar, tol=0.0, max_iter=10**9) for i in insts[:3]]
        b.step(11)
        ids += [b.add(i.X, i.ybar, tol=0.0, max_iter=10**9) for i in insts[3:]]
        b.step(9)
        outs = [b.primal(i) for i in ids]
    for inst, (y, xi), k in zip(insts, outs, [20, 20, 20, 9, 9, 9]):
        ys, xis, _ = _single(inst, k)
        assert np.array_equal(y, ys) and np.array_equal(xi, xis), (inst.N, inst.n)


def test_tf32_batch_converged_results_match_oracle():
    shapes = [(60, 2), (190, 4), (260, 17), (75, 3), (140, 31)]
    insts = _instances(shapes, seed0=700)
    gamma, tol = 1e-2, 1e-4
    with crgb.Batch(tile_cols=512, gamma=gamma, graph_iters=8, check_every=50, precision=TF32) as b:
        ids = [b.add(i.X, i.ybar, tol=tol, max_iter=200000) for i in insts]
        b.run()
        res = []
        for i in ids:
            done, status, info = b.poll(i)
            assert done and status == 0, (i, status, info)
            assert info["rel_gap"] <= tol
            res.append((info, b.primal(i)))
    for inst, (info, (y, xi)) in zip(insts, res):
        L = oracle.lipschitz(inst.X, gamma)
        o = oracle.PAPG(inst.X, inst.ybar, gamma, L)
        log = o.step(int(info["k"]))
        yr, xir = o.primal()
        assert rel(y, yr) <= 1e-4, (inst.N, inst.n, rel(y, yr))
        assert rel(xi, xir) <= 1e-3, (inst.N, inst.n, rel(xi, xir))
        assert abs(info["dual_g"] - log["g"][-1]) <= 1e-4 * abs(log["g"][-1])
