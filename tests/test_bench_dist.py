"""The benchmark's multi-rank path on CPU: two gloo ranks (replicas, no data
collective), the barrier and the max-over-ranks timing reduction."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
os.environ["ACCSINK_BENCH_GLOO"] = "1"
rank, world = bench.dist_setup()
assert world == 2 and rank == int(os.environ["RANK"])
bench.barrier(world)
t = bench.max_over_ranks(1.0 + rank, world)
assert t == 2.0, t
seeds = {bench.replica_seed(r) for r in range(world)}
assert len(seeds) == world
print("ok", rank, t, flush=True)
dist.destroy_process_group()
'''


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_replicas_and_max_timing(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), ACCSINK_BENCH_GLOO="1")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        assert o.startswith("ok")
