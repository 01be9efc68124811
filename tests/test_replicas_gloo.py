"""The multi-GPU path runs independent replicas (a pair does not shard); its host logic - launcher
environment, barrier, max-over-ranks timing, whole-job throughput, the split of a batch across
ranks - checked with two gloo ranks on the CPU, launched as torchrun would (RANK, WORLD_SIZE,
MASTER_ADDR = 127.0.0.1, MASTER_PORT in the environment)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import datetime, json, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
from paper_2106_07927_gb300 import replicas
ws, rank, local = replicas.env()
dist.init_process_group("gloo", init_method="env://", world_size=ws, rank=rank,
                        timeout=datetime.timedelta(seconds=60))
replicas.barrier()
units = [100.0, 300.0][rank]      # work this rank did
seconds = [1.0, 2.0][rank]        # its timed region
out = {
    "env": [ws, rank, local],
    "max": replicas.max_over_ranks(rank + 1.5),
    "sum": replicas.sum_over_ranks(10.0 * (rank + 1)),
    "throughput": replicas.job_throughput(units, seconds),
    "shards": {n: list(replicas.shard(n, ws, rank)) for n in (0, 1, 2, 7, 64)},
}
replicas.barrier()
print(json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_replicas():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for rank, r in enumerate(outs):
        assert r["env"] == [2, rank, rank]
        assert r["max"] == 2.5                  # slowest rank's value on every rank
        assert r["sum"] == 30.0
        assert r["throughput"] == 400.0 / 2.0   # all ranks' units over the slowest time
    for n in ("0", "1", "2", "7", "64"):
        a, b = outs[0]["shards"][n], outs[1]["shards"][n]
        assert sorted(a + b) == list(range(int(n)))  # every item exactly once
        assert abs(len(a) - len(b)) <= 1


def test_shard_alone_and_errors():
    from paper_2106_07927_gb300 import replicas
    assert list(replicas.shard(5, 1, 0)) == [0, 1, 2, 3, 4]
    assert [len(replicas.shard(10, 4, r)) for r in range(4)] == [3, 3, 2, 2]
    with pytest.raises(ValueError):
        replicas.shard(5, 2, 2)
    assert replicas.max_over_ranks(3.0) == 3.0  # no process group: the value itself
