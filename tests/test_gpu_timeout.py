"""The bounded-wait failure path of the FP32 TMA sweep, made to run out without a fault.

cr_set_wait_limit bounds the consumer warps' waits for data to a few nanoseconds, so the
first wait that finds its stage still in flight gives up: the CTA sets its abort flag, the
producer stops issuing copies and waits for every copy it issued, and the device status
records CR_ETIMEOUT.  Nothing traps or hangs: each wait is bounded and the producer's drain
keeps its normal bound.  The test checks that the next convergence check reports
CR_ETIMEOUT, and that a new context in the same process still iterates exactly as the FP64
oracle does (the CUDA context stays usable).
"""
import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb
from paper_1608_02227_gb300 import _capi

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_consumer_wait_runs_out_and_reports_timeout():
    inst = cr_synth.make_instance(3000, 8, "maxaff", 0.05, 31)
    gamma = 1e-4
    L = oracle.lipschitz(inst.X, gamma)
    lib = _capi.load()
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_FP32, graph_iters=0) as s:
        assert s.describe()["sweep"] == "tma"
        assert lib.cr_set_wait_limit(s.ctx, 1) == 0
        s.step(2)
        with pytest.raises(crgb.CRError) as e:
            s.gap()
        assert e.value.status == crgb.CR_ETIMEOUT
    # the process and the device are fine: a fresh context matches the oracle
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L)
    ref.step(5, log=False)
    y_r, xi_r = ref.primal()
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_FP32, graph_iters=0) as s:
        s.step(5)
        y, xi = s.primal()
        g = s.gap()
    assert rel(y, y_r) <= 1e-4 and rel(xi, xi_r) <= 1e-3 and g["k"] == 5


def test_wait_limit_is_refused_off_the_tma_sweep():
    inst = cr_synth.make_instance(300, 4, "sqnorm", 0.1, 32)
    lib = _capi.load()
    with crgb.Solver(inst.X, inst.ybar, gamma=1e-3, precision=crgb.CR_MIXED_TF32) as s:
        assert lib.cr_set_wait_limit(s.ctx, 1) == crgb.CR_EUNSUPPORTED
    with crgb.Solver(inst.X, inst.ybar, gamma=1e-3, precision=crgb.CR_FP32) as s:
        assert lib.cr_set_wait_limit(s.ctx, -1) == crgb.CR_EINVAL
        assert lib.cr_set_wait_limit(s.ctx, 0) == 0
