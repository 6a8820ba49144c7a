"""Step-size constant for the K = N dual (oracle side; test infrastructure only).

For K = N, C = [A1 A2] (Definition 3 with A3 = A1, A4 = A2) and the dual Hessian is
-C G^{-1} C^T with G = diag(I_N, gamma I_{Nn}) (Section 3, the generic QP).  So
    lambda_max(C G^{-1} C^T) = lambda_max(A1 A1^T + A2 A2^T / gamma)
                            <= sigma_max(A1)^2 + sigma_max(A2)^2 / gamma,
with sigma_max(A1)^2 = 2N exactly (Lemma "O1-constant") and, A2 being block diagonal
with blocks X_l = -T_l Xbar, sigma_max(A2)^2 = max_l lambda_max(X_l^T X_l), where
X_l^T X_l = sum_{j != l} (x_l - x_j)(x_l - x_j)^T (the paper's "Preprocess" computes
sigma_max(A4) = sigma_max(A2) for K = N).

rule "hessian" (default): L = 2N + sigma_max(A2)^2 / gamma, an upper bound on the
    Lipschitz constant of grad g_gamma that is tight to a factor (1 + 2N gamma /
    sigma_max(A2)^2).
rule "paper": L = (2N + sigma_max(A2)^2) / gamma >= sigma_max(C)^2 / gamma, an upper
    bound on the L_gamma of Eq. (lischitz).
"""
from __future__ import annotations

import numpy as np


def a2_sigma_sq(X, chunk: int = 64) -> float:
    """sigma_max(A2)^2 = max_l lambda_max( sum_{j != l} (x_l - x_j)(x_l - x_j)^T ),
    each n x n block formed from its definition and passed to an eigensolver."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, n = X.shape
    best = 0.0
    for l0 in range(0, N, chunk):
        l1 = min(N, l0 + chunk)
        D = X[l0:l1, None, :] - X[None, :, :]          # (c, N, n); the j = l row is 0
        S = np.einsum("cjk,cjm->ckm", D, D)
        ev = np.linalg.eigvalsh(S)[:, -1]
        best = max(best, float(ev.max()))
    return best


def lipschitz(X, gamma: float, rule: str = "hessian") -> float:
    N = X.shape[0]
    s2 = a2_sigma_sq(X)
    if rule == "hessian":
        return 2.0 * N + s2 / gamma
    if rule == "paper":
        return (2.0 * N + s2) / gamma
    raise ValueError(f"unknown rule {rule!r}")
