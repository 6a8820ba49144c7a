"""ctypes declarations of the C ABI in include/cr.h (argument marshalling only).

The shared library is built in-tree by ``paper_1608_02227_gb300.build`` into
``paper_1608_02227_gb300/_build/libcrgb.so``.  Loading fails loudly when it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcrgb.so")

CR_OK, CR_EINVAL, CR_ENOMEM, CR_ECUDA, CR_ENOTCONV, CR_ETIMEOUT, CR_ENUMERIC, CR_EUNSUPPORTED = range(8)
CR_FP64, CR_FP32, CR_MIXED_TF32 = 0, 1, 2
CR_L_HESSIAN, CR_L_PAPER = 0, 1
CR_STEP_CONSTANT, CR_STEP_ADAPTIVE = 0, 1
CR_MAX_N = 128
CR_MAX_N_TF32 = 31
CR_MAX_N_BATCH = 32


class cr_options(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("lipschitz", ctypes.c_double),
        ("lipschitz_rule", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("accelerate", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("graph_iters", ctypes.c_int),
        ("tile_cols", ctypes.c_int),
        ("deterministic", ctypes.c_int),
        ("step_rule", ctypes.c_int),
        ("upsilon", ctypes.c_double),
        ("restart", ctypes.c_int),
        ("refresh_every", ctypes.c_int),
    ]


class cr_gap_info(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_longlong),
        ("dual_g", ctypes.c_double),
        ("primal_r", ctypes.c_double),
        ("lagr_gap", ctypes.c_double),
        ("infeas_norm", ctypes.c_double),
        ("rel_gap", ctypes.c_double),
        ("cert_primal", ctypes.c_double),
        ("cert_gap_rel", ctypes.c_double),
        ("step", ctypes.c_double),
        ("sweeps", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class cr_serve_stats(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_longlong),
        ("converged", ctypes.c_longlong),
        ("queued", ctypes.c_longlong),
        ("running", ctypes.c_longlong),
        ("mem_used", ctypes.c_longlong),
        ("mem_cap", ctypes.c_longlong),
        ("p50_s", ctypes.c_double),
        ("p99_s", ctypes.c_double),
        ("elapsed_s", ctypes.c_double),
        ("busy_s", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class CRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None

# (name, restype, argtypes) of every entry point in include/cr.h
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_SIGS = [
    ("cr_default_options", None, [ctypes.POINTER(cr_options)]),
    ("cr_create", ctypes.c_int, [_vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(cr_options), _vp,
                                 ctypes.POINTER(_vp)]),
    ("cr_dual_step", ctypes.c_int, [_vp, ctypes.c_int]),
    ("cr_solve", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_longlong, ctypes.POINTER(cr_gap_info)]),
    ("cr_primal", ctypes.c_int, [_vp, _vp, _vp]),
    ("cr_gap", ctypes.c_int, [_vp, ctypes.POINTER(cr_gap_info)]),
    ("cr_lambda", ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_longlong, _vp, ctypes.c_longlong]),
    ("cr_dual_step_timed", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float)]),
    ("cr_describe", ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_int]),
    ("cr_lipschitz", ctypes.c_int, [_vp, _dp]),
    ("cr_lipschitz_noalloc", ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_double, ctypes.c_int, _vp,
                                            _dp]),
    ("cr_iterations", ctypes.c_longlong, [_vp]),
    ("cr_set_wait_limit", ctypes.c_int, [_vp, ctypes.c_longlong]),
    ("cr_set_gamma", ctypes.c_int, [_vp, ctypes.c_double]),
    ("cr_solve_path", ctypes.c_int, [_vp, _dp, _dp, ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(cr_gap_info)]),
    ("cr_solve_continuation", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_longlong,
                                             ctypes.POINTER(cr_gap_info)]),
    ("cr_checkpoint_bytes", ctypes.c_longlong, [_vp]),
    ("cr_checkpoint", ctypes.c_int, [_vp, _vp, ctypes.c_longlong]),
    ("cr_restore", ctypes.c_int, [_vp, _vp, ctypes.c_longlong]),
    ("cr_destroy", None, [_vp]),
    ("cr_shard_create", ctypes.c_int, [_vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                                       ctypes.POINTER(cr_options), _vp, ctypes.POINTER(_vp)]),
    ("cr_shard_sweep", ctypes.c_int, [_vp, _vp]),
    ("cr_shard_finish", ctypes.c_int, [_vp, _vp]),
    ("cr_shard_state", ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(cr_gap_info)]),
    ("cr_batch_create", ctypes.c_int, [ctypes.POINTER(cr_options), _vp, ctypes.POINTER(_vp)]),
    ("cr_batch_add", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]),
    ("cr_batch_step", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("cr_batch_run", ctypes.c_int, [_vp]),
    ("cr_batch_poll", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(cr_gap_info)]),
    ("cr_batch_primal", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    ("cr_batch_remove", ctypes.c_int, [_vp, ctypes.c_int]),
    ("cr_batch_instance_bytes", ctypes.c_longlong, [ctypes.c_longlong, ctypes.c_int]),
    ("cr_batch_autotune", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("cr_batch_destroy", None, [_vp]),
    ("cr_server_create", ctypes.c_int, [ctypes.POINTER(cr_options), ctypes.c_longlong, ctypes.c_int, _vp,
                                        ctypes.POINTER(_vp)]),
    ("cr_server_submit", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    ("cr_server_poll", ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(cr_gap_info), _dp]),
    ("cr_server_wait", ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_double]),
    ("cr_server_result", ctypes.c_int, [_vp, ctypes.c_longlong, _vp, _vp]),
    ("cr_server_release", ctypes.c_int, [_vp, ctypes.c_longlong]),
    ("cr_server_stats", ctypes.c_int, [_vp, ctypes.POINTER(cr_serve_stats)]),
    ("cr_server_destroy", None, [_vp]),
    ("cr_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("cr_last_error", ctypes.c_char_p, []),
    ("cr_version", ctypes.c_int, []),
]


def symbols():
    """Names of the entry points the binding expects the library to export."""
    return [n for n, _, _ in _SIGS]


def load(path: str | None = None):
    """Load libcrgb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(
            f"CUDA library not built: {p} is missing; run `python -c \"import __graft_entry__ as g; g.build()\"`")
    lib = ctypes.CDLL(p)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status: int, lib=None):
    if status != CR_OK:
        lib = lib or load()
        raise CRError(status, f"{lib.cr_strerror(status).decode()}: {lib.cr_last_error().decode()}")
