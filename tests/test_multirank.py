"""The N > 1 bench path on CPU: two gloo ranks launched through torch.distributed.run (as the
GPU bench is, with 127.0.0.1 rendezvous).  Replicas: every rank holds its own instance of the
same shape (seed + rank), the timed region is the slowest rank's, and the whole-job rate counts
the pairs of all ranks.  The reference arm runs on rank 0 only."""
import argparse
import json
import os
import socket
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_share_the_bench_bookkeeping(tmp_path):
    out = tmp_path / "ranks.json"
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "multirank_child.py"), str(out)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    every = json.loads(out.read_text())
    assert [e["rank"] for e in every] == [0, 1] and all(e["ws"] == 2 for e in every)
    # the same shape, independent draws
    assert every[0]["shape"] == every[1]["shape"] == [200, 2]
    assert every[0]["ybar_sum"] != every[1]["ybar_sum"] and every[0]["x_first"] != every[1]["x_first"]
    # max over ranks, and the whole-job rate of 2 x N(N-1) pairs x 7 iterations over it
    assert all(e["t_max"] == 13.0 for e in every)
    assert all(abs(e["rate"] - 2 * 200 * 199 * 7 / 13.0e-3) <= 1e-6 * e["rate"] for e in every)


def test_single_rank_helpers():
    assert bench.max_over_ranks(4.5, 1) == 4.5
    assert bench.job_rate(100, 10, 1, 1000.0) == 1000.0
    a = bench.rank_instance("sqnorm_N200_n2", 0)
    b = bench.rank_instance("sqnorm_N200_n2", 0, N=50)
    assert a.X.shape == (200, 2) and b.X.shape == (50, 2)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(workload="sqnorm_N200_n2", steps=3, warmup=3, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
