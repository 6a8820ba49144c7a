"""Row sharding of the multipliers over several GPUs (cr_shard_* of include/cr.h).

Each rank holds the multipliers of the pairs (i, j) with i in its block of rows and every j.
An iteration of Figure "papg" (K = N) is the shard's sweep, one sum of N + 1 FP64 values over
all ranks (torch.distributed all_reduce: NCCL on GPUs), and the shard's finish; afterwards every
rank holds the same C_y^T lambda^k, y and objective values and xi of its own rows.

``partition`` splits the rows, ``Shard`` wraps one library shard, and ``ShardedSolver`` runs the
iteration protocol over any object with ``sweep(buf)``, ``finish(buf)`` and ``state()`` and any
in-place sum (``allreduce``), so the protocol is testable with a CPU stand-in of the shard.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import check, cr_gap_info

ALIGN = 128  # a shard starts at a multiple of the tensor-core sweep's 128-row items


def partition(N: int, parts: int, align: int = ALIGN):
    """Contiguous row blocks [(row0, rows), ...], one per part, starting at multiples of
    ``align`` and as equal in rows (so in pairs: every row has N - 1 of them) as that allows."""
    if parts < 1 or N < 2:
        raise ValueError("need N >= 2 and at least one part")
    units = (N + align - 1) // align
    if parts > units:
        raise ValueError(f"N = {N} has {units} blocks of {align} rows: at most {units} parts")
    out, start = [], 0
    for p in range(parts):
        u = units // parts + (1 if p < units % parts else 0)
        row0 = start * align
        end = min(N, (start + u) * align)
        out.append((row0, end - row0))
        start += u
    return out


class Shard:
    """One library shard (cr_shard_create): rows [row0, row0 + rows) of the multipliers.

    ``stream`` (a torch.cuda.Stream; a new one by default) orders the shard's kernels with the
    exchange: run the all_reduce of the exchange buffer on it (ShardedSolver does)."""

    def __init__(self, X, ybar, row0, rows, stream=None, **options):
        import torch

        from . import _ptr, default_options
        self.opt = default_options(**options)
        xp, xk = _ptr(X)
        yp, _ = _ptr(ybar)
        self.N, self.n = int(xk.shape[0]), int(xk.shape[1])
        self.row0, self.rows = int(row0), int(rows)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.ctx = ctypes.c_void_p()
        check(_capi.load().cr_shard_create(xp, yp, self.N, self.n, self.row0, self.rows, ctypes.byref(self.opt),
                                           ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.ctx)))

    def exchange_buffer(self):
        import torch
        with torch.cuda.stream(self.stream):
            return torch.zeros(self.N + 1, dtype=torch.float64, device="cuda")

    def sweep(self, buf):
        check(_capi.load().cr_shard_sweep(self.ctx, ctypes.c_void_p(buf.data_ptr())))

    def finish(self, buf):
        check(_capi.load().cr_shard_finish(self.ctx, ctypes.c_void_p(buf.data_ptr())))

    def state(self):
        """(y of every point, xi of the held rows, record)."""
        y = np.empty(self.N)
        xi = np.empty((self.rows, self.n))
        g = cr_gap_info()
        check(_capi.load().cr_shard_state(self.ctx, ctypes.c_void_p(y.ctypes.data), ctypes.c_void_p(xi.ctypes.data),
                                          ctypes.byref(g)))
        return y, xi, g.as_dict()

    def close(self):
        if self.ctx:
            _capi.load().cr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class ShardedSolver:
    """The iteration protocol of the row-sharded method on one rank: ``local`` is this rank's
    shard (``sweep(buf)`` writes its share of the N + 1 exchanged sums, ``finish(buf)`` completes
    the iteration from their sum over all ranks), ``allreduce(buf)`` sums ``buf`` over the ranks
    in place (torch.distributed.all_reduce in a job, NCCL on GPUs)."""

    def __init__(self, local, allreduce, buf):
        self.local = local
        self.allreduce = allreduce
        self.buf = buf
        self.k = 0

    def step(self, iters=1):
        stream = getattr(self.local, "stream", None)
        for _ in range(int(iters)):
            self.local.sweep(self.buf)
            if stream is not None:  # the shard's kernels and the exchange in one stream order
                import torch
                with torch.cuda.stream(stream):
                    self.allreduce(self.buf)
            else:
                self.allreduce(self.buf)
            self.local.finish(self.buf)
            self.k += 1

    def state(self):
        return self.local.state()
