"""Brute-force dense references for tiny instances (test infrastructure only).

These are built from the paper's definitions without the matrix-free loops of
``cr_oracle.c``, so that the oracle can be pinned to something other than itself:

* ``dense_A(X)``: A1 and A2 of Definition 1, T_l = [e_1 .. e_{l-1}, -1, e_l .. e_{N-1}],
  A1 = [T_1; ...; T_N], A2 = blkdiag(-T_l Xbar), rows in lexicographic (l1, l2) order.
* ``solve_nnls(X, ybar, gamma)``: the dual of Eq. (regularize) with every constraint
  dualised, max_{theta >= 0} g_gamma(theta), rewritten as the non-negative least
  squares problem min_{theta >= 0} ||A1^T theta + ybar||^2 + ||A2^T theta||^2 / gamma
  (since -g_gamma(theta) = 1/2||a + ybar||^2 - 1/2||ybar||^2 + 1/2||b||^2/gamma with
  (a, b) = C^T theta), solved by scipy's bounded-variable least squares (BVLS, an
  active-set method).  Its primal
  (y*, xi*) = (ybar + A1^T theta*, A2^T theta* / gamma) is then checked for
  feasibility and complementary slackness by the caller.
* ``n2_closed_form``: the exact solution of Eq. (regularize) for N = 2, derived from
  its KKT conditions (not printed in the paper).
"""
from __future__ import annotations

import numpy as np


def T_matrix(l: int, N: int) -> np.ndarray:
    """T_l of Definition 1 (0-based l): (N-1) x N, column l is -1, the other columns
    are the unit vectors e_1..e_{N-1} in order."""
    T = np.zeros((N - 1, N))
    r = 0
    for c in range(N):
        if c == l:
            T[:, c] = -1.0
        else:
            T[r, c] = 1.0
            r += 1
    return T


def dense_A(X):
    """(A1, A2) of Definition 1 for points X (N x n)."""
    X = np.asarray(X, dtype=np.float64)
    N, n = X.shape
    Ts = [T_matrix(l, N) for l in range(N)]
    A1 = np.vstack(Ts)
    A2 = np.zeros((N * (N - 1), N * n))
    for l in range(N):
        A2[l * (N - 1):(l + 1) * (N - 1), l * n:(l + 1) * n] = -Ts[l] @ X
    return A1, A2


def pair_order(N: int):
    """Row index -> (l1, l2) for the lexicographic order of Definition 1."""
    return [(i, j) for i in range(N) for j in range(N) if i != j]


def theta_vec_to_mat(v, N):
    M = np.zeros((N, N))
    for r, (i, j) in enumerate(pair_order(N)):
        M[i, j] = v[r]
    return M


def theta_mat_to_vec(M):
    N = M.shape[0]
    return np.array([M[i, j] for (i, j) in pair_order(N)])


def solve_nnls(X, ybar, gamma):
    """Exact dual solution for tiny N by NNLS.  Returns dict(theta (N x N), y, xi, p)."""
    from scipy.optimize import lsq_linear

    X = np.asarray(X, dtype=np.float64)
    ybar = np.asarray(ybar, dtype=np.float64)
    N, n = X.shape
    A1, A2 = dense_A(X)
    M = np.vstack([A1.T, A2.T / np.sqrt(gamma)])
    v = np.concatenate([-ybar, np.zeros(N * n)])
    th = lsq_linear(M, v, bounds=(0.0, np.inf), method="bvls", tol=1e-15,
                    max_iter=50 * M.shape[1]).x
    th = np.maximum(th, 0.0)
    a = A1.T @ th
    b = A2.T @ th
    y = ybar + a
    xi = (b / gamma).reshape(N, n)
    p = 0.5 * np.sum((y - ybar) ** 2) + 0.5 * gamma * np.sum(xi ** 2)
    return dict(theta=theta_vec_to_mat(th, N), y=y, xi=xi, p=p, A1=A1, A2=A2)


def n2_closed_form(X, ybar, gamma):
    """Solution of Eq. (regularize) for N = 2 points.

    With e = x2 - x1, d = ||e||, D = ybar2 - ybar1: the slope difference
    delta = y2 - y1 = D d^2 / (d^2 + 2 gamma); y1 = ybar1 - (delta - D)/2,
    y2 = ybar2 + (delta - D)/2; the subgradient that must carry the slope is
    (delta / d^2) e (xi2 if delta >= 0, else xi1), the other is 0;
    p* = (delta - D)^2 / 4 + gamma delta^2 / (2 d^2)."""
    X = np.asarray(X, dtype=np.float64)
    ybar = np.asarray(ybar, dtype=np.float64)
    e = X[1] - X[0]
    d2 = float(e @ e)
    D = float(ybar[1] - ybar[0])
    delta = D * d2 / (d2 + 2.0 * gamma)
    y = np.array([ybar[0] - (delta - D) / 2.0, ybar[1] + (delta - D) / 2.0])
    xi = np.zeros((2, X.shape[1]))
    if delta >= 0:
        xi[1] = (delta / d2) * e
    else:
        xi[0] = (delta / d2) * e
    p = (delta - D) ** 2 / 4.0 + gamma * delta ** 2 / (2.0 * d2)
    return dict(y=y, xi=xi, p=p)
