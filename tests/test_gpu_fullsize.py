"""Parity at the benchmark's full sizes, in the configuration bench.py times.

The FP64 oracle runs the same iterations from scratch (Figure "papg", K = N) on the full
instance -- three iterations at N = 20000 hold four 3.2 GB arrays on the host and take
about two minutes on the host cores -- and the CUDA path is compared with it on sampled rows
of Lambda (rows chosen to cover the first, interior and ragged last 128-row blocks) and on
the whole primal recovery eta(lambda^k) = (y, xi).  The step constant L is computed by the
oracle and passed to the CUDA path (the library's own L is checked against it separately),
so nothing the CUDA path computes is fed to the oracle.  Tolerances are those of the
reduced-precision modes: 1e-4 on y, 1e-3 on xi and on the sampled multiplier rows, both as
relative 2-norms and element by element against the largest magnitude (a wrong edge tile of
a 20000-row Lambda moves the 2-norm too little to be seen); the library's L to 1e-9.
"""
import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb

pytestmark = pytest.mark.gpu

GAMMA = 1e-4  # bench.py's smoothing parameter
ITERS = 3     # the third iteration is the first with momentum


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def relmax(a, b):
    """Largest element-wise error, scaled by the largest magnitude of the reference."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _rows(N):
    return sorted({0, 1, 127, 128, 129, N // 3, N // 2 + 7, N - 129, N - 33, N - 2, N - 1})


@pytest.mark.parametrize("workload,precision", [("lse_N20000_n20", crgb.CR_MIXED_TF32),
                                                ("maxaff_N5000_n10", crgb.CR_FP32),
                                                ("maxaff_N5000_n10", crgb.CR_MIXED_TF32)])
def test_full_size_iterates_match_oracle(workload, precision):
    inst = cr_synth.workload(workload)
    N = inst.N
    L = oracle.lipschitz(inst.X, GAMMA)
    with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, precision=precision) as s:
        L_lib = s.describe()["L"]
    assert abs(L_lib - L) <= 1e-9 * L
    with crgb.Solver(inst.X, inst.ybar, gamma=GAMMA, lipschitz=L, precision=precision) as s:
        s.step(ITERS)
        y, xi = s.primal()
        rows = _rows(N)
        lam_rows = np.stack([s.lam(r, 1)[0] for r in rows])
    ref = oracle.PAPG(inst.X, inst.ybar, GAMMA, L)
    ref.step(ITERS, log=False)
    y_r, xi_r = ref.primal()
    th_rows = ref.theta[rows]
    del ref
    assert rel(y, y_r) <= 1e-4 and relmax(y, y_r) <= 1e-4, (rel(y, y_r), relmax(y, y_r))
    assert rel(xi, xi_r) <= 1e-3 and relmax(xi, xi_r) <= 1e-3, (rel(xi, xi_r), relmax(xi, xi_r))
    assert rel(lam_rows, th_rows) <= 1e-3
    for k, r in enumerate(rows):
        assert lam_rows[k].min() >= 0.0 and lam_rows[k][r] == 0.0
        assert rel(lam_rows[k], th_rows[k]) <= 1e-3, (r, rel(lam_rows[k], th_rows[k]))
        assert relmax(lam_rows[k], th_rows[k]) <= 1e-3, (r, relmax(lam_rows[k], th_rows[k]))
