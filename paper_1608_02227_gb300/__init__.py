"""GB300 (sm_103a) library for the dual smoothing method of Aybat & Wang (arXiv 1608.02227).

Python binding of the C ABI in include/cr.h.  Every function here only marshals
arguments; every step of the method runs in the CUDA kernels of ``csrc/``.  Inputs may
be numpy arrays (host) or torch tensors (host or CUDA); outputs are numpy arrays unless
``device=True`` (torch CUDA tensors).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import (CR_ECUDA, CR_EINVAL, CR_ENOMEM, CR_ENOTCONV, CR_ENUMERIC, CR_ETIMEOUT, CR_EUNSUPPORTED,
                    CR_FP32, CR_FP64, CR_L_HESSIAN, CR_L_PAPER, CR_MAX_N, CR_MAX_N_BATCH, CR_MAX_N_TF32,
                    CR_MIXED_TF32, CR_OK, CR_STEP_ADAPTIVE, CR_STEP_CONSTANT, CRError,
                    cr_gap_info, cr_options, check)

__all__ = [
    "CR_FP64", "CR_FP32", "CR_MIXED_TF32", "CR_L_HESSIAN", "CR_L_PAPER", "CR_MAX_N", "CR_MAX_N_TF32",
    "CR_MAX_N_BATCH", "CRError", "CR_OK", "CR_EINVAL", "CR_ENOMEM", "CR_ECUDA", "CR_ENOTCONV", "CR_ETIMEOUT",
    "CR_ENUMERIC", "CR_EUNSUPPORTED",
    "CR_STEP_CONSTANT", "CR_STEP_ADAPTIVE",
    "default_options", "cr_create", "cr_dual_step", "cr_dual_step_timed", "cr_solve", "cr_primal",
    "cr_gap", "cr_lambda", "cr_lipschitz", "cr_iterations", "cr_describe", "cr_destroy", "Solver",
    "library_path", "Batch", "cr_batch_instance_bytes", "Server",
]


def library_path() -> str:
    return _capi.LIB_PATH


def _lib():
    return _capi.load()


def default_options(**kw) -> cr_options:
    o = cr_options()
    _lib().cr_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


def _ptr(a):
    """Data pointer of a C-contiguous float64 numpy array or torch tensor (host or CUDA)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise TypeError("tensors must be contiguous float64")
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return ctypes.c_void_p(arr.ctypes.data), arr


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream) if stream else None
    h = getattr(stream, "cuda_stream", None)
    if h is None:
        raise TypeError("stream must be a torch.cuda.Stream, an int handle or None")
    return ctypes.c_void_p(h) if h else None


def cr_create(X, ybar, opt: cr_options | None = None, stream=None):
    """Create a context for one instance; returns an opaque handle (ctypes.c_void_p)."""
    xp, xk = _ptr(X)
    yp, yk = _ptr(ybar)
    shape = tuple(getattr(xk, "shape", ()))
    if len(shape) != 2:
        raise ValueError("X must be 2-d (N x n)")
    N, n = int(shape[0]), int(shape[1])
    if int(np.prod(getattr(yk, "shape", (0,)))) != N:
        raise ValueError("ybar must have N entries")
    out = ctypes.c_void_p()
    st = _lib().cr_create(xp, yp, N, n, ctypes.byref(opt) if opt is not None else None,
                          _stream_handle(stream), ctypes.byref(out))
    check(st)
    return out


def cr_dual_step(ctx, iters: int):
    check(_lib().cr_dual_step(ctx, int(iters)))


def cr_dual_step_timed(ctx, iters: int):
    sw = ctypes.c_float()
    tot = ctypes.c_float()
    check(_lib().cr_dual_step_timed(ctx, int(iters), ctypes.byref(sw), ctypes.byref(tot)))
    return float(sw.value), float(tot.value)


def cr_solve(ctx, rel_gap_tol: float, max_iter: int):
    """Returns (converged: bool, record dict)."""
    g = cr_gap_info()
    st = _lib().cr_solve(ctx, float(rel_gap_tol), int(max_iter), ctypes.byref(g))
    if st not in (_capi.CR_OK, _capi.CR_ENOTCONV):
        check(st)
    return st == _capi.CR_OK, g.as_dict()


def cr_gap(ctx):
    g = cr_gap_info()
    check(_lib().cr_gap(ctx, ctypes.byref(g)))
    return g.as_dict()


def _shape_of(ctx):
    import json
    d = json.loads(cr_describe(ctx))
    return d["N"], d["n"]


def cr_primal(ctx, device: bool = False):
    """eta(lambda^k) = (y, xi) as float64 arrays (numpy, or torch CUDA tensors)."""
    N, n = _shape_of(ctx)
    if device:
        import torch
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        xi = torch.empty((N, n), dtype=torch.float64, device="cuda")
        check(_lib().cr_primal(ctx, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(xi.data_ptr())))
        return y, xi
    y = np.empty(N)
    xi = np.empty((N, n))
    check(_lib().cr_primal(ctx, ctypes.c_void_p(y.ctypes.data), ctypes.c_void_p(xi.ctypes.data)))
    return y, xi


def cr_lambda(ctx, row0: int = 0, rows: int | None = None, device: bool = False):
    """Rows [row0, row0+rows) of lambda^k as float64 (numpy, or a torch CUDA tensor)."""
    N, _ = _shape_of(ctx)
    rows = N - row0 if rows is None else rows
    if device:
        import torch
        out = torch.empty((rows, N), dtype=torch.float64, device="cuda")
        check(_lib().cr_lambda(ctx, row0, rows, ctypes.c_void_p(out.data_ptr()), N))
        return out
    out = np.empty((rows, N))
    check(_lib().cr_lambda(ctx, row0, rows, ctypes.c_void_p(out.ctypes.data), N))
    return out


def cr_lipschitz(ctx) -> float:
    v = ctypes.c_double()
    check(_lib().cr_lipschitz(ctx, ctypes.byref(v)))
    return float(v.value)


def cr_iterations(ctx) -> int:
    return int(_lib().cr_iterations(ctx))


def cr_describe(ctx) -> str:
    buf = ctypes.create_string_buffer(1024)
    check(_lib().cr_describe(ctx, buf, len(buf)))
    return buf.value.decode()


def cr_destroy(ctx):
    if ctx:
        _lib().cr_destroy(ctx)


class Solver:
    """Owning wrapper of one context (closes it on ``close()``/``with``)."""

    def __init__(self, X, ybar, stream=None, **options):
        self.opt = default_options(**options)
        self.ctx = cr_create(X, ybar, self.opt, stream)

    def step(self, iters=1):
        cr_dual_step(self.ctx, iters)

    def solve(self, tol, max_iter):
        return cr_solve(self.ctx, tol, max_iter)

    def gap(self):
        return cr_gap(self.ctx)

    def primal(self, device=False):
        return cr_primal(self.ctx, device)

    def lam(self, row0=0, rows=None, device=False):
        return cr_lambda(self.ctx, row0, rows, device)

    @property
    def L(self):
        return cr_lipschitz(self.ctx)

    @property
    def k(self):
        return cr_iterations(self.ctx)

    def describe(self):
        import json
        return json.loads(cr_describe(self.ctx))

    def set_gamma(self, gamma):
        """Continuation (Section 6): new gamma, warm start from lambda^k."""
        check(_lib().cr_set_gamma(self.ctx, float(gamma)))

    def solve_path(self, gammas, tols, max_sweeps):
        """cr_solve_path: returns (converged: bool, record of the last stage)."""
        g = np.ascontiguousarray(gammas, dtype=np.float64)
        t = np.ascontiguousarray(tols, dtype=np.float64)
        if g.shape != t.shape or g.ndim != 1 or g.size == 0:
            raise ValueError("gammas and tols must be equal-length non-empty 1-D sequences")
        rec = cr_gap_info()
        st = _lib().cr_solve_path(self.ctx, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(g.size), int(max_sweeps),
                                  ctypes.byref(rec))
        if st not in (_capi.CR_OK, _capi.CR_ENOTCONV):
            check(st)
        return st == _capi.CR_OK, rec.as_dict()

    def solve_continuation(self, eps0, beta, kappa_gamma, kappa_delta, stages, max_sweeps, infeas_tol=-1.0):
        """cr_solve_continuation (Section 6's schedule): returns (converged: bool, last record).
        infeas_tol >= 0 also accepts Section 5's practical test at each stage."""
        rec = cr_gap_info()
        st = _lib().cr_solve_continuation(self.ctx, float(eps0), float(beta), float(kappa_gamma), float(kappa_delta),
                                          float(infeas_tol), int(stages), int(max_sweeps), ctypes.byref(rec))
        if st not in (_capi.CR_OK, _capi.CR_ENOTCONV):
            check(st)
        return st == _capi.CR_OK, rec.as_dict()

    def checkpoint(self):
        """The iteration state as a host byte array (cr_checkpoint)."""
        nb = int(_lib().cr_checkpoint_bytes(self.ctx))
        buf = np.empty(nb, dtype=np.uint8)
        check(_lib().cr_checkpoint(self.ctx, ctypes.c_void_p(buf.ctypes.data), nb))
        return buf

    def restore(self, buf):
        """Loads a cr_checkpoint block into this context (same instance and options)."""
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        check(_lib().cr_restore(self.ctx, ctypes.c_void_p(b.ctypes.data), int(b.size)))

    def close(self):
        if self.ctx:
            cr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def cr_batch_instance_bytes(N: int, n: int) -> int:
    return int(_lib().cr_batch_instance_bytes(int(N), int(n)))


class Batch:
    """Many independent instances iterated together (cr_batch_* of include/cr.h)."""

    def __init__(self, stream=None, **options):
        self.opt = default_options(**options)
        self.handle = ctypes.c_void_p()
        check(_lib().cr_batch_create(ctypes.byref(self.opt), _stream_handle(stream), ctypes.byref(self.handle)))
        self.shapes = {}

    def add(self, X, ybar, tol=1e-4, max_iter=100000):
        xp, xk = _ptr(X)
        yp, yk = _ptr(ybar)
        N, n = int(xk.shape[0]), int(xk.shape[1])
        i = ctypes.c_int()
        check(_lib().cr_batch_add(self.handle, xp, yp, N, n, float(tol), int(max_iter), ctypes.byref(i)))
        self.shapes[i.value] = (N, n)
        return i.value

    def step(self, iters):
        a = ctypes.c_int()
        check(_lib().cr_batch_step(self.handle, int(iters), ctypes.byref(a)))
        return a.value

    def run(self):
        check(_lib().cr_batch_run(self.handle))

    def poll(self, i):
        done = ctypes.c_int()
        st = ctypes.c_int()
        g = cr_gap_info()
        check(_lib().cr_batch_poll(self.handle, int(i), ctypes.byref(done), ctypes.byref(st), ctypes.byref(g)))
        return bool(done.value), int(st.value), g.as_dict()

    def primal(self, i):
        N, n = self.shapes[i]
        y = np.empty(N)
        xi = np.empty((N, n))
        check(_lib().cr_batch_primal(self.handle, int(i), ctypes.c_void_p(y.ctypes.data),
                                     ctypes.c_void_p(xi.ctypes.data)))
        return y, xi

    def remove(self, i):
        check(_lib().cr_batch_remove(self.handle, int(i)))

    def autotune(self, iters=4):
        w = ctypes.c_int()
        check(_lib().cr_batch_autotune(self.handle, int(iters), ctypes.byref(w)))
        return w.value

    def close(self):
        if self.handle:
            _lib().cr_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (cr_server_* of include/cr.h)."""

    def __init__(self, mem_cap_bytes=60 << 30, max_active=256, stream=None, **options):
        self.opt = default_options(**options)
        self.handle = ctypes.c_void_p()
        check(_lib().cr_server_create(ctypes.byref(self.opt), int(mem_cap_bytes), int(max_active),
                                      _stream_handle(stream), ctypes.byref(self.handle)))
        self.shapes = {}

    def submit(self, X, ybar, tol=1e-4, max_iter=100000):
        xp, xk = _ptr(X)
        yp, yk = _ptr(ybar)
        N, n = int(xk.shape[0]), int(xk.shape[1])
        rid = ctypes.c_longlong()
        check(_lib().cr_server_submit(self.handle, xp, yp, N, n, float(tol), int(max_iter), ctypes.byref(rid)))
        self.shapes[rid.value] = (N, n)
        return rid.value

    def poll(self, rid):
        state = ctypes.c_int()
        st = ctypes.c_int()
        g = cr_gap_info()
        lat = ctypes.c_double()
        check(_lib().cr_server_poll(self.handle, int(rid), ctypes.byref(state), ctypes.byref(st), ctypes.byref(g),
                                    ctypes.byref(lat)))
        return int(state.value), int(st.value), g.as_dict(), float(lat.value)

    def wait(self, rid, timeout=600.0):
        check(_lib().cr_server_wait(self.handle, int(rid), float(timeout)))

    def result(self, rid):
        N, n = self.shapes[rid]
        y = np.empty(N)
        xi = np.empty((N, n))
        check(_lib().cr_server_result(self.handle, int(rid), ctypes.c_void_p(y.ctypes.data),
                                      ctypes.c_void_p(xi.ctypes.data)))
        return y, xi

    def release(self, rid):
        check(_lib().cr_server_release(self.handle, int(rid)))

    def stats(self):
        st = _capi.cr_serve_stats()
        check(_lib().cr_server_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.handle:
            _lib().cr_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
