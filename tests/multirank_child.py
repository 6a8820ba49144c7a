"""One rank of the multi-rank bench bookkeeping on CPU (gloo): launched by
tests/test_multirank.py through torch.distributed.run exactly as bench.py is for N > 1
GPUs, but with the gloo backend and no GPU.  Rank 0 writes what every rank saw to argv[1]."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main(out):
    dist.init_process_group("gloo")
    ws, rank, _ = bench._dist()
    inst = bench.rank_instance("sqnorm_N200_n2", rank)
    # a rank-dependent "timed region": the job is as slow as its slowest rank
    t_max = bench.max_over_ranks(10.0 + 3.0 * rank, ws, device="cpu")
    rate = bench.job_rate(inst.N * (inst.N - 1), 7, ws, t_max)
    dist.barrier()
    seen = dict(rank=rank, ws=ws, shape=list(inst.X.shape), ybar_sum=float(inst.ybar.sum()),
                x_first=float(inst.X[0, 0]), t_max=t_max, rate=rate)
    every = [None] * ws
    dist.all_gather_object(every, seen)
    if rank == 0:
        with open(out, "w") as fh:
            json.dump(every, fh)
    dist.destroy_process_group()


if __name__ == "__main__":
    main(sys.argv[1])
