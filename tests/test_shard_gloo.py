"""Row sharding of the multipliers (paper_1608_02227_gb300.shard) on CPU: two gloo ranks
launched through torch.distributed.run on 127.0.0.1, each holding one block of rows of Lambda
in a numpy stand-in of the library shard (tests/shard_child.py).  The product's partition and
iteration protocol (sweep, all_reduce of the N + 1 exchanged sums, finish) must reproduce the
FP64 oracle's iterates of Figure "papg": after 25 iterations y (every rank, every point), xi
(each rank's rows, assembled) and g_gamma within 1e-10."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import cr_synth
import oracle
from paper_1608_02227_gb300.shard import partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_blocks():
    assert partition(300, 2) == [(0, 256), (256, 44)]
    assert partition(700, 3) == [(0, 256), (256, 256), (512, 188)]
    assert partition(1024, 4) == [(0, 256), (256, 256), (512, 256), (768, 256)]
    for N, p in [(129, 2), (5000, 7), (20000, 8)]:
        parts = partition(N, p)
        assert parts[0][0] == 0 and sum(r for _, r in parts) == N
        assert all(r0 % 128 == 0 and r > 0 for r0, r in parts)
        assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(p - 1))
    with pytest.raises(ValueError):
        partition(200, 3)


def test_two_gloo_ranks_reproduce_the_oracle(tmp_path):
    out = tmp_path / "shards.json"
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "shard_child.py"), str(out)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    every = json.loads(out.read_text())
    assert [e["rank"] for e in every] == [0, 1]
    inst = cr_synth.make_instance(300, 3, "maxaff", 0.1, 17)
    ref = oracle.PAPG(inst.X, inst.ybar, 1e-3, every[0]["L"])
    log = ref.step(25)
    y_r, xi_r = ref.primal()
    xi = np.concatenate([np.asarray(e["xi"]) for e in every])
    for e in every:
        y = np.asarray(e["y"])
        assert np.abs(y - y_r).max() <= 1e-10 * np.abs(y_r).max()
        assert e["rec"]["k"] == 25
        assert abs(e["rec"]["g"] - log["g"][-1]) <= 1e-10 * abs(log["g"][-1])
    assert np.abs(xi - xi_r).max() <= 1e-10 * np.abs(xi_r).max()
