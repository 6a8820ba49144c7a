"""Seeded synthetic convex-regression inputs shared by the oracle side and the CUDA side.

This module only draws data.  It holds none of the method's arithmetic (no residuals,
no multipliers, no step sizes), so both the CPU oracle and the GPU library can be fed
from it without sharing any computation.

Draw order for every instance (fixed so that a seed names one dataset):
  1. the model parameters of f0 (a_k, b_k, Q, p ... in the order listed per family),
  2. the locations X, row-major (point by point),
  3. the additive noise.
All draws use ``numpy.random.default_rng(seed)``.

Families (Section 5 of the paper draws f0 from a family, adds zero-mean noise, Eq. (1)):
  "sqnorm"  f0(x) = ||x||_2^2
  "maxaff"  f0(x) = max_k (a_k . x + b_k),  a_k ~ N(0, I_n), b_k ~ N(0, 1)
  "lse"     f0(x) = log sum_k exp(a_k . x), a_k ~ N(0, I_n)
  "quad"    f0(x) = 1/2 x^T Q x, Q = V diag(s) V^T with condition number 15 (Section 5)
  "exp"     f0(x) = exp(p^T x), p ~ U[0, 0.2]^n (Section 5)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Instance",
    "make_instance",
    "workload",
    "batch_workload",
    "serving_stream",
    "WORKLOADS",
]


@dataclass
class Instance:
    """One convex-regression dataset: N points x_l in R^n with observations ybar_l."""

    X: np.ndarray          # (N, n) float64, row-major
    ybar: np.ndarray       # (N,) float64
    family: str
    seed: int
    noise: float
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def n(self) -> int:
        return int(self.X.shape[1])


def _f0(family: str, rng: np.random.Generator, n: int, n_pieces: int | None):
    """Draw the parameters of f0 and return a vectorised evaluator X -> f0(X)."""
    if family == "sqnorm":
        return lambda X: np.einsum("ij,ij->i", X, X)
    if family == "maxaff":
        K = n_pieces or 10
        A = rng.standard_normal((K, n))
        b = rng.standard_normal(K)
        return lambda X: np.max(X @ A.T + b, axis=1)
    if family == "lse":
        K = n_pieces or 8
        A = rng.standard_normal((K, n))

        def lse(X):
            Z = X @ A.T
            m = Z.max(axis=1, keepdims=True)
            return (m + np.log(np.exp(Z - m).sum(axis=1, keepdims=True)))[:, 0]

        return lse
    if family == "quad":
        Lam = rng.standard_normal((n, n))
        Qbar = Lam.T @ Lam
        U, s, Vt = np.linalg.svd(Qbar)
        # keep the singular vectors, map the singular values affinely onto [s_max/15, s_max]
        smax = s[0]
        if n > 1 and s[0] > s[-1]:
            s_new = smax / 15.0 + (s - s[-1]) * (smax - smax / 15.0) / (s[0] - s[-1])
        else:
            s_new = np.full_like(s, smax)
        Q = (U * s_new) @ U.T
        Q = 0.5 * (Q + Q.T)
        return lambda X: 0.5 * np.einsum("ij,jk,ik->i", X, Q, X)
    if family == "exp":
        p = rng.uniform(0.0, 0.2, size=n)
        return lambda X: np.exp(X @ p)
    raise ValueError(f"unknown family {family!r}")


def make_instance(
    N: int,
    n: int,
    family: str = "sqnorm",
    noise: float = 0.1,
    seed: int = 0,
    x_dist: str = "uniform",
    n_pieces: int | None = None,
    interior_frac: float = 0.0,
    interior_scale: float = 1.3,
) -> Instance:
    """Draw one instance.

    x_dist: "uniform" -> x ~ U[-1, 1]^n;  "normal4" -> x ~ N(0, 4 I_n) (Section 5).
    interior_frac: fraction of points whose observation is replaced by
    interior_scale * ybar (Section 5 moves 30% of the pairs to (x, 1.3 ybar)).
    """
    if N < 1 or n < 1:
        raise ValueError("N and n must be positive")
    rng = np.random.default_rng(seed)
    f = _f0(family, rng, n, n_pieces)
    if x_dist == "uniform":
        X = rng.uniform(-1.0, 1.0, size=(N, n))
    elif x_dist == "normal4":
        X = rng.normal(0.0, 2.0, size=(N, n))
    else:
        raise ValueError(f"unknown x_dist {x_dist!r}")
    eps = rng.normal(0.0, noise, size=N) if noise > 0 else np.zeros(N)
    ybar = f(X) + eps
    if interior_frac > 0:
        k = int(round(interior_frac * N))
        idx = rng.choice(N, size=k, replace=False)
        ybar[idx] = interior_scale * ybar[idx]
    X = np.ascontiguousarray(X, dtype=np.float64)
    ybar = np.ascontiguousarray(ybar, dtype=np.float64)
    return Instance(X=X, ybar=ybar, family=family, seed=seed, noise=noise,
                    meta={"x_dist": x_dist, "interior_frac": interior_frac})


# ---------------------------------------------------------------------------
# Named workloads (shapes and distributions of the single-instance runs)
# ---------------------------------------------------------------------------
WORKLOADS = {
    # N=200 points in 2-d, f0 = ||x||^2, noise sd 0.1, seed 0
    "sqnorm_N200_n2": dict(N=200, n=2, family="sqnorm", noise=0.1, seed=0),
    # N=5000 in 10-d, f0 = max of 10 affine pieces, noise sd 0.05
    "maxaff_N5000_n10": dict(N=5000, n=10, family="maxaff", noise=0.05, seed=0, n_pieces=10),
    # N=20000 in 20-d, f0 = log-sum-exp of 8 linear terms, noise sd 0.1
    "lse_N20000_n20": dict(N=20000, n=20, family="lse", noise=0.1, seed=0, n_pieces=8),
    # Section 5 shaped: 1/2 x^T Q x (cond 15), x ~ N(0,4), noise var 100, 30% scaled by 1.3
    "paper_quad_N2400_n20": dict(N=2400, n=20, family="quad", noise=10.0, seed=0,
                                 x_dist="normal4", interior_frac=0.3),
    "paper_exp_N2400_n80": dict(N=2400, n=80, family="exp", noise=10.0, seed=0,
                                x_dist="normal4", interior_frac=0.3),
}


def workload(name: str, **override) -> Instance:
    """Instance for a named workload; keyword overrides (e.g. N=1000) shrink it."""
    spec = dict(WORKLOADS[name])
    spec.update(override)
    return make_instance(**spec)


def batch_workload(count: int = 256, seed: int = 0, N_lo: int = 100, N_hi: int = 4000,
                   n_lo: int = 2, n_hi: int = 16, noise: float = 0.1):
    """Independent instances, N log-uniform in [N_lo, N_hi] (rounded), n uniform in
    {n_lo..n_hi}, f0 = ||x||^2.  Instance i is drawn from seed (seed + 1 + i); the
    sizes are drawn first from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    Ns = np.rint(np.exp(rng.uniform(math.log(N_lo), math.log(N_hi), size=count))).astype(int)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    return [make_instance(int(N), int(n), "sqnorm", noise, seed + 1 + i)
            for i, (N, n) in enumerate(zip(Ns, ns))]


def serving_stream(count: int = 500, rate: float = 20.0, seed: int = 0, N_lo: int = 200,
                   N_hi: int = 30000, n_lo: int = 2, n_hi: int = 32, noise: float = 0.1,
                   materialize: bool = True):
    """Poisson request stream: list of (arrival_time_s, Instance or spec dict).

    Inter-arrival times ~ Exp(rate); N log-uniform in [N_lo, N_hi]; n uniform in
    {n_lo..n_hi}; f0 uniform over {sqnorm, maxaff (10 pieces), lse (8 terms)}.
    Request r's data comes from seed (seed + 1 + r)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    Ns = np.rint(np.exp(rng.uniform(math.log(N_lo), math.log(N_hi), size=count))).astype(int)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    fams = rng.integers(0, 3, size=count)
    names = ["sqnorm", "maxaff", "lse"]
    out = []
    for r in range(count):
        spec = dict(N=int(Ns[r]), n=int(ns[r]), family=names[fams[r]], noise=noise,
                    seed=seed + 1 + r)
        out.append((float(t[r]), make_instance(**spec) if materialize else spec))
    return out
