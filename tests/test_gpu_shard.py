"""Row shards of the library (cr_shard_*) against the FP64 oracle, on one GPU.

Every box here has one GPU, so the ranks of a sharded job are emulated in one process: the
shards of a partition run their sweeps one after another, the exchange (the sum of the N + 1
values over the shards, an all_reduce in a real job) is formed on the device between the
launches, and every shard finishes the iteration from it.  No kernel waits on another.
Checked: y (every shard, every point), xi (each shard's rows, assembled) and g_gamma against the
oracle's iterates of Figure "papg" -- 1e-10 in FP64, the reduced-precision tolerances (1e-4 on
y, 1e-3 on xi, element by element and as 2-norms, 1e-4 on g) in FP32 and mixed precision --
and the argument checks of the shard entry points.
"""
import ctypes

import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb
from paper_1608_02227_gb300 import _capi
from paper_1608_02227_gb300.shard import Shard, partition

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def relmax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def _run_shards(inst, gamma, L, parts, iters, **opts):
    import torch
    stream = torch.cuda.Stream()  # one stream orders every shard's kernels and the exchange
    shards = [Shard(inst.X, inst.ybar, r0, rows, stream=stream, gamma=gamma, lipschitz=L, **opts)
              for r0, rows in parts]
    bufs = [sh.exchange_buffer() for sh in shards]
    try:
        for _ in range(iters):
            for sh, b in zip(shards, bufs):
                sh.sweep(b)
            with torch.cuda.stream(stream):
                total = torch.stack(bufs).sum(0)   # the exchange of a real job: all_reduce(sum)
                for b in bufs:
                    b.copy_(total)
            for sh, b in zip(shards, bufs):
                sh.finish(b)
        states = [sh.state() for sh in shards]
    finally:
        for sh in shards:
            sh.close()
    return states


@pytest.mark.parametrize("N,n,fam,prec,nparts", [(700, 5, "maxaff", crgb.CR_FP64, 3),
                                                 (700, 5, "maxaff", crgb.CR_FP32, 3),
                                                 (1000, 20, "lse", crgb.CR_MIXED_TF32, 2),
                                                 (300, 3, "sqnorm", crgb.CR_FP64, 2)])
def test_shards_follow_the_oracle(N, n, fam, prec, nparts):
    inst = cr_synth.make_instance(N, n, fam, 0.1, 40 + nparts)
    gamma = 1e-3
    L = oracle.lipschitz(inst.X, gamma)
    parts = partition(N, nparts)
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L)
    k = 0
    for iters in (1, 12, 60):
        log = ref.step(iters - k)
        k = iters
        y_r, xi_r = ref.primal()
        states = _run_shards(inst, gamma, L, parts, iters, precision=prec)
        xi = np.concatenate([s[1] for s in states])
        f64 = prec == crgb.CR_FP64
        ty, txi, tg = (1e-10, 1e-10, 1e-10) if f64 else (1e-4, 1e-3, 1e-4)
        for y, _, g in states:
            assert g["k"] == iters
            assert rel(y, y_r) <= ty and relmax(y, y_r) <= ty, (iters, rel(y, y_r))
            assert abs(g["dual_g"] - log["g"][-1]) <= tg * abs(log["g"][-1]), (iters, g, log["g"][-1])
        assert rel(xi, xi_r) <= txi and relmax(xi, xi_r) <= txi, (iters, rel(xi, xi_r), relmax(xi, xi_r))


def test_shard_argument_checks():
    import torch
    inst = cr_synth.make_instance(300, 3, "sqnorm", 0.1, 3)
    lib = _capi.load()
    opt = crgb.default_options(gamma=1e-3)
    ctx = ctypes.c_void_p()
    X = np.ascontiguousarray(inst.X)
    yb = np.ascontiguousarray(inst.ybar)
    args = (ctypes.c_void_p(X.ctypes.data), ctypes.c_void_p(yb.ctypes.data), 300, 3)
    # row0 not a multiple of 128, rows past N
    assert lib.cr_shard_create(*args, 100, 50, ctypes.byref(opt), None, ctypes.byref(ctx)) == crgb.CR_EINVAL
    assert lib.cr_shard_create(*args, 256, 60, ctypes.byref(opt), None, ctypes.byref(ctx)) == crgb.CR_EINVAL
    ad = crgb.default_options(gamma=1e-3, step_rule=crgb.CR_STEP_ADAPTIVE)
    assert lib.cr_shard_create(*args, 0, 128, ctypes.byref(ad), None, ctypes.byref(ctx)) == crgb.CR_EUNSUPPORTED
    with Shard(inst.X, inst.ybar, 128, 172, gamma=1e-3) as sh:
        # whole-instance entry points refuse a shard, and the exchange must be device memory
        assert lib.cr_dual_step(sh.ctx, 1) == crgb.CR_EINVAL
        host = np.zeros(301)
        assert lib.cr_shard_sweep(sh.ctx, ctypes.c_void_p(host.ctypes.data)) == crgb.CR_EINVAL
        b = sh.exchange_buffer()
        assert lib.cr_shard_sweep(sh.ctx, ctypes.c_void_p(b.data_ptr())) == 0
        sh.stream.synchronize()
    with Shard(inst.X, inst.ybar, 0, 300, gamma=1e-3) as sh:  # one shard holding every row
        b = sh.exchange_buffer()
        assert lib.cr_shard_sweep(sh.ctx, ctypes.c_void_p(b.data_ptr())) == 0
        sh.stream.synchronize()
    with crgb.Solver(inst.X, inst.ybar, gamma=1e-3) as s:
        b = torch.zeros(301, dtype=torch.float64, device="cuda")
        assert lib.cr_shard_sweep(s.ctx, ctypes.c_void_p(b.data_ptr())) == crgb.CR_EINVAL
