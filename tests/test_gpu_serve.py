"""Serving (cr_server_*): continuous batching gives every request what it gets alone.

Requests arrive while others are running, are admitted at the next block boundary and
share launches with them; each finished request is compared, bitwise, with the same
instance solved alone for the same number of iterations (same kernels, same 512-column
split).  Admission respects the device-memory cap.
"""
import time

import numpy as np
import pytest

import cr_synth
import paper_1608_02227_gb300 as crgb

pytestmark = pytest.mark.gpu


def _stream(count, seed=0, N_lo=600, N_hi=1800, n_lo=2, n_hi=12):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        N = int(rng.integers(N_lo, N_hi))
        n = int(rng.integers(n_lo, n_hi + 1))
        fam = ["sqnorm", "maxaff", "lse"][r % 3]
        out.append(cr_synth.make_instance(N, n, fam, 0.1, 1000 + r))
    return out


def test_served_results_equal_alone_and_requests_overlap():
    insts = _stream(8)
    gamma = 1e-3
    max_running = 0
    with crgb.Server(tile_cols=512, mem_cap_bytes=8 << 30, max_active=64, gamma=gamma, check_every=25, graph_iters=4) as srv:
        ids = []
        for inst in insts:
            ids.append(srv.submit(inst.X, inst.ybar, tol=1e-4, max_iter=3000))
            time.sleep(0.02)
            max_running = max(max_running, srv.stats()["running"])
        for r in ids:
            srv.wait(r, 300)
        res = [(srv.poll(r), srv.result(r)) for r in ids]
        stats = srv.stats()
    assert max_running >= 2, "requests never shared the GPU"
    assert stats["completed"] == len(insts)
    for inst, ((state, status, info, lat), (y, xi)) in zip(insts, res):
        assert state == 2 and status in (0, 4) and lat > 0
        with crgb.Solver(inst.X, inst.ybar, gamma=gamma, tile_cols=512, graph_iters=0) as s:
            s.step(int(info["k"]))
            ys, xis = s.primal()
        assert np.array_equal(y, ys) and np.array_equal(xi, xis), (inst.N, inst.n)


def test_admission_respects_the_memory_cap():
    insts = _stream(6, seed=1, N_lo=1500, N_hi=1600, n_lo=4, n_hi=4)
    need = max(crgb.cr_batch_instance_bytes(i.N, i.n) for i in insts)
    cap = 2 * need + need // 2           # room for two instances at a time
    with crgb.Server(tile_cols=512, mem_cap_bytes=cap, max_active=64, gamma=1e-3, check_every=20, graph_iters=4) as srv:
        ids = [srv.submit(i.X, i.ybar, tol=1e-4, max_iter=400) for i in insts]
        peak_running, saw_queue = 0, False
        deadline = time.time() + 300
        while srv.stats()["completed"] < len(ids) and time.time() < deadline:
            st = srv.stats()
            peak_running = max(peak_running, st["running"])
            saw_queue = saw_queue or st["queued"] > 0
            assert st["mem_used"] <= cap
            time.sleep(0.005)
        for r in ids:
            srv.wait(r, 60)
            assert srv.poll(r)[0] == 2
    assert peak_running <= 2 and saw_queue


def test_oversized_request_is_refused():
    inst = cr_synth.make_instance(3000, 8, "sqnorm", 0.1, 3)
    with crgb.Server(tile_cols=512, mem_cap_bytes=1 << 20, max_active=4) as srv:
        with pytest.raises(crgb.CRError) as e:
            srv.submit(inst.X, inst.ybar)
        assert e.value.status == 2


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_tf32_served_results_equal_alone():
    # mixed precision: tensor-core instances (n <= 31) and an n = 32 instance on the FP32
    # sweep share the server's launches; each equals its single-instance run bitwise
    insts = _stream(6, seed=4, N_lo=300, N_hi=1400, n_lo=2, n_hi=31)
    insts.append(cr_synth.make_instance(500, 32, "lse", 0.1, 1099))
    gamma = 1e-3
    with crgb.Server(tile_cols=512, mem_cap_bytes=8 << 30, max_active=64, gamma=gamma, check_every=25,
                     graph_iters=4, precision=crgb.CR_MIXED_TF32) as srv:
        ids = []
        for inst in insts:
            ids.append(srv.submit(inst.X, inst.ybar, tol=1e-4, max_iter=2000))
            time.sleep(0.02)
        for r in ids:
            srv.wait(r, 300)
        res = [(srv.poll(r), srv.result(r)) for r in ids]
    for inst, ((state, status, info, lat), (y, xi)) in zip(insts, res):
        assert state == 2 and status in (0, 4)
        prec = crgb.CR_MIXED_TF32 if inst.n <= crgb.CR_MAX_N_TF32 else crgb.CR_FP32
        with crgb.Solver(inst.X, inst.ybar, gamma=gamma, tile_cols=512, graph_iters=0, precision=prec) as s:
            s.step(int(info["k"]))
            ys, xis = s.primal()
        assert np.array_equal(y, ys) and np.array_equal(xi, xis), (inst.N, inst.n)


@pytest.mark.parametrize("precision", [crgb.CR_FP32, crgb.CR_MIXED_TF32])
def test_served_results_match_oracle(precision):
    # every request of a small mixed stream against the FP64 oracle run for the same number
    # of iterations (Figure "papg", constant step), at the reduced-precision tolerances:
    # 1e-4 on y, 1e-3 on xi (relative 2-norms and element by element), 1e-4 on g
    import oracle
    insts = _stream(5, seed=7, N_lo=120, N_hi=420, n_lo=2, n_hi=14)
    gamma = 1e-3
    with crgb.Server(tile_cols=512, mem_cap_bytes=4 << 30, max_active=16, gamma=gamma, check_every=50,
                     graph_iters=4, precision=precision) as srv:
        ids = [srv.submit(i.X, i.ybar, tol=1e-4, max_iter=1500) for i in insts]
        for r in ids:
            srv.wait(r, 300)
        res = [(srv.poll(r), srv.result(r)) for r in ids]
    for inst, ((state, status, info, lat), (y, xi)) in zip(insts, res):
        assert state == 2 and status in (0, 4), (status, info)
        L = oracle.lipschitz(inst.X, gamma)
        o = oracle.PAPG(inst.X, inst.ybar, gamma, L)
        log = o.step(int(info["k"]))
        yr, xir = o.primal()
        assert _rel(y, yr) <= 1e-4 and np.abs(y - yr).max() <= 1e-4 * np.abs(yr).max(), (inst.N, inst.n)
        assert _rel(xi, xir) <= 1e-3 and np.abs(xi - xir).max() <= 1e-3 * np.abs(xir).max(), (inst.N, inst.n)
        assert abs(info["dual_g"] - log["g"][-1]) <= 1e-4 * abs(log["g"][-1])
