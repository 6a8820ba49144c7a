"""FP64 CPU oracle for the K = N dual smoothing method (arXiv 1608.02227).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  The CUDA library never imports, links or runs anything
here, and nothing here imports the library.

* ``cr_oracle.c`` holds the iteration (Figure "papg" with K = N), the matrix-free
  C and C^T maps, the dual and primal objectives and the certified upper bound; this
  module loads it with ctypes.
* ``lipschitz.py`` holds the step-size constant.
* ``qp_dense.py`` holds the brute-force dense references used to pin the oracle
  (Definition 1 matrices, an NNLS solve of the dual, the N = 2 closed form).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcr_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile cr_oracle.c with gcc (OpenMP) into oracle/_build/libcr_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i, d = ctypes.c_int, ctypes.c_double
            lib.cro_c_apply.argtypes = [i, i, _dp, _dp, _dp, _dp]
            lib.cro_ct_apply.argtypes = [i, i, _dp, _dp, _dp, _dp]
            lib.cro_eta_of_theta.argtypes = [i, i, _dp, _dp, d, _dp, _dp, _dp]
            lib.cro_primal_obj.argtypes = [i, i, _dp, d, _dp, _dp]
            lib.cro_primal_obj.restype = d
            lib.cro_dual_obj.argtypes = [i, i, _dp, _dp, d, _dp, _dp, _dp, _dp, _dp, _dp]
            lib.cro_dual_obj.restype = d
            lib.cro_papg.argtypes = [i, i, _dp, _dp, d, d, i, i, _dp, _dp, _dp, _dp, _dp, _dp]
            lib.cro_papg.restype = i
            lib.cro_papg_adaptive.argtypes = [i, i, _dp, _dp, d, d, d, i, i, i, _dp, _dp, _dp, _dp, _dp, _ip, _dp]
            lib.cro_papg_adaptive.restype = i
            lib.cro_certify.argtypes = [i, i, _dp, _dp, d, _dp, _dp, _dp, _ip, _dp]
            lib.cro_threads.restype = i
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads() -> int:
    return int(_load().cro_threads())


def c_apply(X, y, xi):
    """(C eta)_ij = y_j - y_i + xi_i.(x_i - x_j) for all ordered pairs, as an N x N array."""
    X, y, xi = _f64(X), _f64(y), _f64(xi)
    N, n = X.shape
    out = np.empty((N, N))
    _load().cro_c_apply(N, n, _p(X), _p(y), _p(xi), _p(out))
    return out


def ct_apply(X, theta):
    """C^T theta = (a, b) with a in R^N, b in R^{N x n}."""
    X, theta = _f64(X), _f64(theta)
    N, n = X.shape
    a = np.empty(N)
    b = np.empty((N, n))
    _load().cro_ct_apply(N, n, _p(X), _p(theta), _p(a), _p(b))
    return a, b


def eta_of_theta(X, ybar, gamma, theta):
    """Closed-form Step 1 minimiser: (y, xi) = (ybar + a, b / gamma)."""
    X, ybar, theta = _f64(X), _f64(ybar), _f64(theta)
    N, n = X.shape
    y = np.empty(N)
    xi = np.empty((N, n))
    _load().cro_eta_of_theta(N, n, _p(X), _p(ybar), float(gamma), _p(theta), _p(y), _p(xi))
    return y, xi


def primal_obj(ybar, gamma, y, xi):
    ybar, y, xi = _f64(ybar), _f64(y), _f64(xi)
    N, n = xi.shape
    return float(_load().cro_primal_obj(N, n, _p(ybar), float(gamma), _p(y), _p(xi)))


def dual_obj(X, ybar, gamma, theta):
    """Returns dict(g, r, lg, y, xi): g_gamma(theta), r_gamma(eta(theta)),
    <theta, C eta(theta)> and eta(theta)."""
    X, ybar, theta = _f64(X), _f64(ybar), _f64(theta)
    N, n = X.shape
    cbuf = np.empty((N, N))
    r = ctypes.c_double()
    lg = ctypes.c_double()
    y = np.empty(N)
    xi = np.empty((N, n))
    g = _load().cro_dual_obj(N, n, _p(X), _p(ybar), float(gamma), _p(theta), _p(cbuf),
                             ctypes.byref(r), ctypes.byref(lg), _p(y), _p(xi))
    return dict(g=float(g), r=float(r.value), lg=float(lg.value), y=y, xi=xi)


class PAPG:
    """State of the oracle iteration: (theta^{k-1}, theta~^k, t_k, k).

    ``step(iters)`` runs Figure "papg" (K = N) and returns per-iteration logs of
    g_gamma(theta^k), r_gamma(eta(theta^k)) and <theta^k, C eta(theta^k)>.  With
    ``adaptive=True`` Step 2 uses the adaptive step size of Section 4 (Eq. (adaptive-check),
    s_k = s_{k-1} upsilon^(l_k - 1), s_0 = L); the log then holds g and the trial counts."""

    def __init__(self, X, ybar, gamma, L, accel=True, theta0=None, adaptive=False, upsilon=2.0, restart=False):
        self.adaptive = bool(adaptive)
        self.restart = bool(restart)
        self.g_prev = np.array([np.nan])
        self.upsilon = float(upsilon)
        self.s = np.array([float(L)])    # s_0 = L (adaptive step rule)
        self.trials = []
        self.X = _f64(X)
        self.ybar = _f64(ybar)
        self.N, self.n = self.X.shape
        self.gamma = float(gamma)
        self.L = float(L)
        self.accel = bool(accel)
        th0 = np.zeros((self.N, self.N)) if theta0 is None else _f64(theta0).copy()
        self.theta = th0.copy()          # theta^{k-1}; after step(): theta^k
        self.theta_tilde = th0.copy()    # theta~^k (Iteration 0: theta~^1 = theta^0)
        self.t = np.array([1.0])         # t_1 = 1
        self.k = 0

    def step(self, iters=1, log=True):
        N, n = self.N, self.n
        if self.adaptive:
            tr = np.empty(iters, dtype=np.int32)
            lg_ = np.empty(iters) if log else None
            rc = _load().cro_papg_adaptive(N, n, _p(self.X), _p(self.ybar), self.gamma, self.L, self.upsilon,
                                           int(iters), int(self.accel), int(self.restart), _p(self.theta),
                                           _p(self.theta_tilde), _p(self.t), _p(self.s), _p(self.g_prev),
                                           tr.ctypes.data_as(_ip), _p(lg_))
            if rc == -1:
                raise MemoryError("oracle iteration could not allocate its work arrays")
            if rc == -2:
                raise FloatingPointError("no step passed the adaptive check")
            self.k += iters
            self.trials.extend(int(v) for v in tr)
            return dict(g=lg_, trials=tr) if log else None
        lg_ = np.empty(iters) if log else None
        lr_ = np.empty(iters) if log else None
        ll_ = np.empty(iters) if log else None
        rc = _load().cro_papg(N, n, _p(self.X), _p(self.ybar), self.gamma, self.L, int(iters),
                              int(self.accel), _p(self.theta), _p(self.theta_tilde), _p(self.t),
                              _p(lg_), _p(lr_), _p(ll_))
        if rc != 0:
            raise MemoryError("oracle iteration could not allocate its work arrays")
        self.k += iters
        if log:
            return dict(g=lg_, r=lr_, lg=ll_)
        return None

    def primal(self):
        """eta(theta^k) = (y^k, xi^k)."""
        return eta_of_theta(self.X, self.ybar, self.gamma, self.theta)

    def ab(self):
        """C^T theta^k."""
        return ct_apply(self.X, self.theta)

    def dual(self):
        return dual_obj(self.X, self.ybar, self.gamma, self.theta)

    def certify(self):
        y, xi = self.primal()
        return certify(self.X, self.ybar, self.gamma, y, xi)


def certify(X, ybar, gamma, y, xi):
    """Feasible repair of (y, xi) and its objective (an upper bound on p*_gamma).
    Returns dict(P=r_gamma(y_rep, xi_rep), infeas_sq=sum min(0,(C eta)_ij)^2,
    yrep, m)."""
    X, ybar, y, xi = _f64(X), _f64(ybar), _f64(y), _f64(xi)
    N, n = X.shape
    yrep = np.empty(N)
    m = np.empty(N, dtype=np.int32)
    out = np.empty(2)
    _load().cro_certify(N, n, _p(X), _p(ybar), float(gamma), _p(y), _p(xi), _p(yrep),
                        m.ctypes.data_as(_ip), _p(out))
    return dict(P=float(out[0]), infeas_sq=float(out[1]), yrep=yrep, m=m)


from .lipschitz import lipschitz, a2_sigma_sq  # noqa: E402

__all__ = ["build", "threads", "c_apply", "ct_apply", "eta_of_theta", "primal_obj",
           "dual_obj", "PAPG", "certify", "lipschitz", "a2_sigma_sq"]
