"""Parity of the tensor-core sweep (CR_MIXED_TF32) with the FP64 CPU oracle.

Both contractions of the sweep (the residual xi_i.x_j and the row sums of Lambda.[X|1])
run as TF32 tensor-core products with a hi+lo split of every operand, so each product
carries a relative error of about 2^-20 against about 2^-24 for the FP32 sweep; Lambda
itself is stored in FP32 as in the FP32 mode.  Tolerances are those of the FP32 modes:
1e-4 on y, 1e-3 on xi, 1e-4 on the dual objective g.
"""
import numpy as np
import pytest

import cr_synth
import oracle
import paper_1608_02227_gb300 as crgb

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def relmax(a, b):
    """Largest element-wise error, scaled by the largest magnitude of the reference."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _check(inst, gamma, iters_list, tile_cols=0, graph_iters=32, accelerate=True):
    L = oracle.lipschitz(inst.X, gamma)
    ref = oracle.PAPG(inst.X, inst.ybar, gamma, L, accel=accelerate)
    with crgb.Solver(inst.X, inst.ybar, gamma=gamma, lipschitz=L, precision=crgb.CR_MIXED_TF32,
                     accelerate=int(accelerate), graph_iters=graph_iters, tile_cols=tile_cols) as s:
        assert s.describe()["sweep"] == "tcgen05"
        k = 0
        for it in iters_list:
            log = ref.step(it - k)
            s.step(it - k)
            k = it
            y_r, xi_r = ref.primal()
            y, xi = s.primal()
            g = s.gap()["dual_g"]
            lam = s.lam()
            rec = dict(k=it, ey=rel(y, y_r), exi=rel(xi, xi_r),
                       eg=abs(g - log["g"][-1]) / max(abs(log["g"][-1]), 1e-300),
                       elam=rel(lam, ref.theta), my=relmax(y, y_r), mxi=relmax(xi, xi_r),
                       mlam=relmax(lam, ref.theta))
            # element by element too: a wrong ragged edge tile barely moves a 2-norm
            assert rec["my"] <= 1e-4 and rec["mxi"] <= 1e-3 and rec["mlam"] <= 1e-3, rec
            assert rec["ey"] <= 1e-4, rec
            assert rec["exi"] <= 1e-3, rec
            assert rec["eg"] <= 1e-4, rec
            assert rec["elam"] <= 1e-3, rec
            assert lam.min() >= 0.0 and np.abs(np.diag(lam)).max() == 0.0
            # padding and the diagonal stay exactly zero
    return True


# sizes span several 128-row blocks and 32-column chunks with ragged tails; n from 1 to 31
@pytest.mark.parametrize("N,n,fam,seed", [(1000, 10, "maxaff", 0), (777, 20, "lse", 1), (450, 2, "sqnorm", 2),
                                          (300, 16, "sqnorm", 3), (129, 31, "sqnorm", 4), (40, 1, "sqnorm", 5),
                                          (2, 3, "sqnorm", 6), (31, 5, "maxaff", 7)])
def test_tf32_iterate_for_iterate(N, n, fam, seed):
    inst = cr_synth.make_instance(N, n, fam, 0.05, seed)
    _check(inst, 1e-4, [1, 10, 100])


@pytest.mark.parametrize("tile_cols", [128, 256])
def test_tf32_many_items_per_cta(tile_cols):
    # 40 row blocks x 40 (or 20) column splits: each CTA walks many items, and the last
    # split of every row block is a single 32-column chunk
    inst = cr_synth.make_instance(5000, 8, "maxaff", 0.05, 21)
    _check(inst, 1e-4, [1, 4, 12], tile_cols=tile_cols)


def test_tf32_gradient_ascent_mode():
    inst = cr_synth.make_instance(600, 4, "sqnorm", 0.1, 22)
    _check(inst, 1e-3, [5, 40], accelerate=False)


def test_tf32_graph_replay_and_repeat_runs_are_bitwise_identical():
    inst = cr_synth.make_instance(1300, 12, "lse", 0.05, 23)
    L = oracle.lipschitz(inst.X, 1e-4)
    res = []
    for g in (0, 16, 16):
        with crgb.Solver(inst.X, inst.ybar, gamma=1e-4, lipschitz=L, precision=crgb.CR_MIXED_TF32,
                         graph_iters=g) as s:
            s.step(3)
            s.step(41)
            y, xi = s.primal()
            res.append((y, xi, s.lam(0, 64)))
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            assert np.array_equal(a, b)


def test_tf32_agrees_with_fp32_sweep():
    inst = cr_synth.make_instance(2000, 20, "lse", 0.05, 24)
    L = oracle.lipschitz(inst.X, 1e-4)
    out = {}
    for p in (crgb.CR_FP32, crgb.CR_MIXED_TF32):
        with crgb.Solver(inst.X, inst.ybar, gamma=1e-4, lipschitz=L, precision=p) as s:
            s.step(50)
            out[p] = s.primal()
    assert rel(out[crgb.CR_MIXED_TF32][0], out[crgb.CR_FP32][0]) <= 1e-5
    assert rel(out[crgb.CR_MIXED_TF32][1], out[crgb.CR_FP32][1]) <= 1e-4


def test_tf32_rejects_n_32():
    inst = cr_synth.make_instance(100, 32, "sqnorm", 0.1, 25)
    with pytest.raises(crgb.CRError):
        crgb.Solver(inst.X, inst.ybar, gamma=1e-3, precision=crgb.CR_MIXED_TF32)
