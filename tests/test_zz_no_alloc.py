"""The allocation-free step-constant entry point (cr_lipschitz_noalloc).

Some callers cannot allocate device memory at the moment they need the step constant L:
an admission controller that budgets HBM before reserving it, a framework whose caching
allocator owns all of HBM, a latency-critical loop where cudaMalloc/cudaFree would
synchronise the device.  cr_lipschitz_noalloc serves them from a fixed scratch array.

Checked here, through the C ABI: on two calls in a row per case it returns the L that
cr_create computes (same kernels: 1e-10 relative) and the oracle's L (1e-9 relative); it
rejects sizes beyond its scratch, host pointers and a non-finite X.

This file is collected last on purpose: if the allocation-free path misbehaves, a run that
stops at the first failure has already run every other test.  It passes both alone in a
fresh process and after the other tests (the static scratch array is set up on first use
and cleared where needed on every call).
"""
import ctypes

import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb
from paper_1608_02227_gb300 import _capi

pytestmark = pytest.mark.gpu


def _noalloc(X_dev, gamma, rule):
    lib = _capi.load()
    L = ctypes.c_double(-1.0)
    st = lib.cr_lipschitz_noalloc(ctypes.c_void_p(X_dev.data_ptr()), int(X_dev.shape[0]), int(X_dev.shape[1]),
                                  float(gamma), int(rule), None, ctypes.byref(L))
    return st, L.value


def test_noalloc_matches_cr_create_and_oracle_on_two_calls_in_a_row():
    import torch
    cases = [(3000, 20, 1e-4, crgb.CR_L_HESSIAN, "lse"), (777, 7, 1e-3, crgb.CR_L_PAPER, "maxaff"),
             (900, 80, 1e-4, crgb.CR_L_HESSIAN, "exp"), (400, 128, 1e-4, crgb.CR_L_PAPER, "quad")]
    for N, n, gamma, rule, fam in cases:
        inst = cr_synth.make_instance(N, n, fam, 0.1, 5)
        with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz_rule=rule) as s:
            L_ref = s.L
        L_or = oracle.lipschitz(inst.X, gamma, rule="paper" if rule == crgb.CR_L_PAPER else "hessian")
        Xd = torch.tensor(inst.X, device="cuda")
        for call in range(2):
            st, L = _noalloc(Xd, gamma, rule)
            assert st == 0, _capi.load().cr_last_error()
            # same kernels and arithmetic as cr_create: equal within the tests' 1e-10 relative bar
            assert abs(L - L_ref) <= 1e-10 * L_ref, (call, N, n, L, L_ref)
            # the oracle forms every block and calls an eigensolver: 1e-9 relative
            assert abs(L - L_or) <= 1e-9 * L_or, (call, N, n, L, L_or)


def test_noalloc_rejects_what_its_scratch_cannot_hold():
    import torch
    lib = _capi.load()
    n_over = crgb.CR_MAX_N + 1
    Xd = torch.zeros((10, n_over), dtype=torch.float64, device="cuda")
    L = ctypes.c_double()
    assert lib.cr_lipschitz_noalloc(ctypes.c_void_p(Xd.data_ptr()), 10, n_over, 1e-4, 0, None, ctypes.byref(L)) == 1
    assert b"scratch" in lib.cr_last_error()
    Xh = np.zeros((10, 3))
    assert lib.cr_lipschitz_noalloc(ctypes.c_void_p(Xh.ctypes.data), 10, 3, 1e-4, 0, None, ctypes.byref(L)) == 1


def test_noalloc_rejects_non_finite_points_and_recovers():
    import torch
    lib = _capi.load()
    inst = cr_synth.make_instance(300, 5, "sqnorm", 0.1, 9)
    Xd = torch.tensor(inst.X, device="cuda")
    Xd[17, 3] = float("nan")
    L = ctypes.c_double()
    assert lib.cr_lipschitz_noalloc(ctypes.c_void_p(Xd.data_ptr()), 300, 5, 1e-4, 0, None, ctypes.byref(L)) == 1
    assert b"non-finite" in lib.cr_last_error()
    # the flag is cleared on the next call: a finite X gives the oracle's L again
    Xd[17, 3] = float(inst.X[17, 3])
    st, Lv = _noalloc(Xd, 1e-4, crgb.CR_L_HESSIAN)
    assert st == 0 and abs(Lv - oracle.lipschitz(inst.X, 1e-4)) <= 1e-9 * Lv
