"""The seeded input generators against the recipe they state (Section 5 for the paper-shaped
families; the named workloads, the batch and the serving stream by their definitions).  The
hidden parameters are recovered from noise-free draws."""
import itertools

import numpy as np
import pytest

import cr_synth


def _quad_features(X):
    n = X.shape[1]
    pairs = list(itertools.combinations_with_replacement(range(n), 2))
    F = np.stack([X[:, i] * X[:, j] * (1.0 if i == j else 2.0) for i, j in pairs], axis=1)
    return F, pairs


@pytest.mark.parametrize("n,seed", [(3, 0), (5, 1), (8, 2)])
def test_quad_family_has_condition_number_15(n, seed):
    inst = cr_synth.make_instance(400, n, "quad", 0.0, seed, x_dist="normal4")
    F, pairs = _quad_features(inst.X)
    coef, *_ = np.linalg.lstsq(F, 2.0 * inst.ybar, rcond=None)  # ybar = 1/2 x^T Q x
    Q = np.zeros((n, n))
    for c, (i, j) in zip(coef, pairs):
        Q[i, j] = Q[j, i] = c
    assert np.allclose(F @ coef, 2.0 * inst.ybar, rtol=1e-10, atol=1e-9)
    ev = np.linalg.eigvalsh(Q)
    assert ev[0] > 0
    assert abs(ev[-1] / ev[0] - 15.0) <= 1e-6


@pytest.mark.parametrize("n,seed", [(4, 0), (20, 3)])
def test_exp_family_slope_in_the_stated_box(n, seed):
    inst = cr_synth.make_instance(300, n, "exp", 0.0, seed, x_dist="normal4")
    p, *_ = np.linalg.lstsq(inst.X, np.log(inst.ybar), rcond=None)
    assert np.allclose(inst.X @ p, np.log(inst.ybar), atol=1e-9)
    assert p.min() >= 0.0 and p.max() <= 0.2


def test_section5_locations_noise_and_interior_points():
    N, n = 4000, 6
    clean = cr_synth.make_instance(N, n, "quad", 0.0, 7, x_dist="normal4")
    noisy = cr_synth.make_instance(N, n, "quad", 10.0, 7, x_dist="normal4")
    moved = cr_synth.make_instance(N, n, "quad", 0.0, 7, x_dist="normal4", interior_frac=0.3)
    # x ~ N(0, 4 I): mean 0, standard deviation 2 (sample of N n values)
    assert abs(clean.X.mean()) <= 0.05 and abs(clean.X.std() - 2.0) <= 0.05
    # noise N(0, 100): the same draw of X and f0, plus noise of standard deviation 10
    assert np.array_equal(noisy.X, clean.X)
    eps = noisy.ybar - clean.ybar
    assert abs(eps.mean()) <= 0.5 and abs(eps.std() - 10.0) <= 0.4
    # 30 % of the observations replaced by 1.3 ybar, the others unchanged
    changed = moved.ybar != clean.ybar
    assert changed.sum() == round(0.3 * N)
    assert np.allclose(moved.ybar[changed], 1.3 * clean.ybar[changed], rtol=1e-15)


def test_named_workloads_have_their_shapes():
    for name, spec in cr_synth.WORKLOADS.items():
        inst = cr_synth.workload(name, N=min(spec["N"], 300))
        assert inst.X.shape == (min(spec["N"], 300), spec["n"]) and inst.ybar.shape == (inst.N,)
        assert np.all(np.isfinite(inst.X)) and np.all(np.isfinite(inst.ybar))
    a, b = cr_synth.workload("maxaff_N5000_n10", N=200), cr_synth.workload("maxaff_N5000_n10", N=200)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.ybar, b.ybar)  # seeded


def test_batch_and_serving_streams_follow_their_ranges():
    insts = cr_synth.batch_workload(count=64, seed=0)
    assert len(insts) == 64
    assert all(100 <= i.N <= 4000 and 2 <= i.n <= 16 for i in insts)
    reqs = cr_synth.serving_stream(count=200, rate=20.0, seed=0, N_lo=200, N_hi=30000, materialize=False)
    t = np.array([r[0] for r in reqs])
    assert len(reqs) == 200 and np.all(np.diff(t) >= 0)
    # Poisson arrivals at 20 per second: mean gap 0.05 s
    assert abs(np.diff(t).mean() - 0.05) <= 0.015
