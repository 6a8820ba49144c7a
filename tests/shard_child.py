"""One rank of the row-sharded iteration on CPU (gloo), launched by tests/test_shard_gloo.py
through torch.distributed.run.  The rank's shard is a plain FP64 numpy stand-in of the library's
shard (written for this test from the exchange contract of cr_shard_sweep / cr_shard_finish);
partition() and ShardedSolver (the product's protocol: sweep, all_reduce of N + 1 values,
finish) drive it.  Rank 0 writes what every rank holds to argv[1]."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import cr_synth  # noqa: E402
import oracle  # noqa: E402
from paper_1608_02227_gb300.shard import ShardedSolver, partition  # noqa: E402

GAMMA = 1e-3


class CpuShard:
    """Rows [row0, row0 + rows) of the multipliers; the exchange contract of the library shard."""

    def __init__(self, X, ybar, L, row0, rows):
        self.X, self.ybar, self.L = X, ybar, L
        self.N, self.n = X.shape
        self.r0, self.r1 = row0, row0 + rows
        self.P = np.zeros((rows, self.N))     # lambda^{k-1}
        self.Q = np.zeros((rows, self.N))     # lambda^{k-2}
        self.a = [np.zeros(self.N), np.zeros(self.N)]            # a^{k-1}, a^{k-2}
        self.b = [np.zeros((rows, self.n)), np.zeros((rows, self.n))]
        self.t, self.beta, self.k = 1.0, 0.0, 0
        self.rec = dict(g=0.0, r=0.0, lg=0.0)

    def sweep(self, buf):
        beta = self.beta
        at = (1 + beta) * self.a[0] - beta * self.a[1]
        bt = (1 + beta) * self.b[0] - beta * self.b[1]
        y = self.ybar + at
        xi = bt / GAMMA
        Xl = self.X[self.r0:self.r1]
        rho = y[self.r0:self.r1, None] - y[None, :] + (xi @ self.X.T) - np.sum(xi * Xl, axis=1)[:, None]
        lt = self.P + beta * (self.P - self.Q)
        lam = np.maximum(0.0, lt + rho / self.L)
        lam[np.arange(self.r1 - self.r0), np.arange(self.r0, self.r1)] = 0.0
        self.Q, self.P = self.P, lam
        r = lam.sum(axis=1)
        v = lam.sum(axis=0)
        v[self.r0:self.r1] -= r
        self.bk = r[:, None] * Xl - lam @ self.X
        buf[: self.N] = torch.from_numpy(v)
        buf[self.N] = float(np.sum(self.bk * self.bk))

    def finish(self, buf):
        a = buf[: self.N].numpy().copy()
        bb = float(buf[self.N])
        self.a = [a, self.a[0]]
        self.b = [self.bk, self.b[0]]
        aa, ay = float(a @ a), float(a @ self.ybar)
        self.rec = dict(g=-0.5 * aa - ay - bb / (2 * GAMMA), r=0.5 * aa + bb / (2 * GAMMA), lg=aa + ay + bb / GAMMA)
        tn = 0.5 * (1 + np.sqrt(1 + 4 * self.t * self.t))
        self.beta = (self.t - 1) / tn
        self.t = tn
        self.k += 1

    def state(self):
        return self.ybar + self.a[0], self.b[0] / GAMMA, dict(self.rec, k=self.k)


def main(out):
    dist.init_process_group("gloo")
    rank, ws = dist.get_rank(), dist.get_world_size()
    inst = cr_synth.make_instance(300, 3, "maxaff", 0.1, 17)
    L = oracle.lipschitz(inst.X, GAMMA)
    parts = partition(inst.N, ws)
    row0, rows = parts[rank]
    solver = ShardedSolver(CpuShard(inst.X, inst.ybar, L, row0, rows), dist.all_reduce,
                           torch.zeros(inst.N + 1, dtype=torch.float64))
    solver.step(25)
    y, xi, rec = solver.state()
    seen = dict(rank=rank, ws=ws, row0=row0, rows=rows, y=y.tolist(), xi=xi.tolist(), rec=rec, L=L)
    every = [None] * ws
    dist.all_gather_object(every, seen)
    if rank == 0:
        with open(out, "w") as fh:
            json.dump(every, fh)
    dist.destroy_process_group()


if __name__ == "__main__":
    main(sys.argv[1])
