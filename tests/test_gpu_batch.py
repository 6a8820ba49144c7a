"""Batched solving (cr_batch_*): each instance in a batch computes what it computes alone.

* Same column-split width alone and in the batch -> bitwise identical iterates (the batch
  runs the same sweep/finalize code over a work-list).
* Instances added mid-way (different iteration counts in one launch) stay exact.
* Retirement at each instance's own tolerance; converged results agree with the FP64 oracle
  at the FP32 tolerances (1e-4 on y, 1e-3 on xi).
"""
import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb

pytestmark = pytest.mark.gpu

SHAPES = [(300, 3), (517, 7), (1000, 10), (128, 16), (777, 2), (2048, 12), (95, 20), (1500, 5)]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _instances(shapes, seed0=100, family="sqnorm"):
    return [cr_synth.make_instance(N, n, family, 0.1, seed0 + i) for i, (N, n) in enumerate(shapes)]


def test_batch_bitwise_matches_single():
    insts = _instances(SHAPES)
    with crgb.Batch(tile_cols=512, gamma=1e-4, graph_iters=8) as b:
        ids = [b.add(i.X, i.ybar, tol=0.0, max_iter=10**9) for i in insts]
        b.step(3)
        b.step(37)
        outs = [b.primal(i) for i in ids]
        infos = [b.poll(i)[2] for i in ids]
    for inst, (y, xi), info in zip(insts, outs, infos):
        with crgb.Solver(inst.X, inst.ybar, gamma=1e-4, tile_cols=512, graph_iters=0) as s:
            s.step(40)
            ys, xis = s.primal()
            gs = s.gap()
        assert np.array_equal(y, ys) and np.array_equal(xi, xis), (inst.N, inst.n, rel(y, ys))
        assert info["k"] == 40 and info["dual_g"] == gs["dual_g"]


def test_batch_instances_added_midway():
    insts = _instances(SHAPES[:5], seed0=200)
    with crgb.Batch(tile_cols=512, gamma=1e-4, graph_iters=4) as b:
        ids = [b.add(i.X, i.ybar, tol=0.0, max_iter=10**9) for i in insts[:3]]
        b.step(11)
        ids += [b.add(i.X, i.ybar, tol=0.0, max_iter=10**9) for i in insts[3:]]
        b.step(9)
        outs = [b.primal(i) for i in ids]
    iters = [20, 20, 20, 9, 9]
    for inst, (y, xi), k in zip(insts, outs, iters):
        with crgb.Solver(inst.X, inst.ybar, gamma=1e-4, tile_cols=512, graph_iters=0) as s:
            s.step(k)
            ys, xis = s.primal()
        assert np.array_equal(y, ys) and np.array_equal(xi, xis)


def test_batch_retires_each_instance_and_matches_oracle():
    shapes = [(60, 2), (90, 4), (120, 8), (75, 3)]
    insts = _instances(shapes, seed0=300)
    gamma, tol = 1e-2, 1e-4
    with crgb.Batch(tile_cols=512, gamma=gamma, graph_iters=8, check_every=50) as b:
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
        assert rel(y, yr) <= 1e-4
        assert rel(xi, xir) <= 1e-3
        assert abs(info["dual_g"] - log["g"][-1]) <= 1e-4 * abs(log["g"][-1])


def test_batch_autotune_and_remove():
    insts = _instances(SHAPES[:4], seed0=400)
    with crgb.Batch(tile_cols=512, gamma=1e-4, graph_iters=0) as b:
        ids = [b.add(i.X, i.ybar, tol=0.0, max_iter=10**9) for i in insts]
        w = b.autotune(2)
        assert w in (512, 1024, 2048, 4096, 1 << 30)
        b.step(5)
        b.remove(ids[1])
        b.step(5)
        y0, _ = b.primal(ids[0])
        with pytest.raises(crgb.CRError):
            b.primal(ids[1])
        done, status, info = b.poll(ids[0])
        assert info["k"] == 5 * 2 + 2 * 5 and not done
    with crgb.Solver(insts[0].X, insts[0].ybar, gamma=1e-4, graph_iters=0) as s:
        s.step(20)
        ys, _ = s.primal()
    assert rel(y0, ys) <= 1e-5


def test_instance_bytes_is_an_upper_bound():
    import torch
    for N, n in [(500, 4), (3000, 16)]:
        inst = cr_synth.make_instance(N, n, "sqnorm", 0.1, 1)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        with crgb.Batch(tile_cols=512, gamma=1e-4) as b:
            b.add(inst.X, inst.ybar)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert free0 - free1 <= crgb.cr_batch_instance_bytes(N, n) + (64 << 20)
