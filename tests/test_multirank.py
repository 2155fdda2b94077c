"""The multi-process path of bench.py (replicas under torchrun): host barrier
and max-over-ranks timing over gloo, world size 2, on CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
world, rank, local = bench.dist_setup()
bench.barrier(world)
m = bench.max_over_ranks(float(10 * (rank + 1)), world)
print(json.dumps({{"rank": rank, "world": world, "max": m}}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def run_ranks(code, world=2, timeout=120):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=timeout)
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_barrier_and_max_over_ranks_gloo():
    outs = run_ranks(WORKER.format(root=ROOT))
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    assert all(l["world"] == 2 and l["max"] == 20.0 for l in lines)


REF = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench, argparse
world, rank, local = bench.dist_setup()
args = argparse.Namespace(workload="cube4_N1e4_exact_fp64", steps=1, warmup=0)
bench.oracle_searches_per_s.__defaults__ = (0.2, 64, 2_000_000)
line = bench.run_reference(args, world, rank)
print(json.dumps(line))
import torch.distributed as dist
dist.destroy_process_group()
"""


def test_reference_arm_rank0_only():
    outs = run_ranks(REF.format(root=ROOT))
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    real = [l for l in lines if l is not None]
    assert len(real) == 1 and real[0]["impl"] == "reference" and real[0]["value"] > 0
    assert real[0]["e2e"]["h2d_bytes_per_step"] == 0
