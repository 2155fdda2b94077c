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


SHARD_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import numpy as np
import torch.distributed as dist
import dd_inputs as I
from oracle import metric, nn
from paper_2012_00357_gb300.shard import merge_nearest
dist.init_process_group("gloo", init_method="env://")
rank, world = dist.get_rank(), dist.get_world_size()
C = I.isotropic_C()
data = I.make_dataset(3001, I.NONLINEAR, seed=12)
y = I.make_states(257, I.NONLINEAR, seed=13, spread=0.05)
zq = metric.to_z(y, C)
bounds = np.linspace(0, len(data), world + 1).astype(int)
lo, hi = bounds[rank], bounds[rank + 1]
i1, d1, _, _ = nn.nn_top2(metric.to_z(data[lo:hi].astype(np.float64), C), zq)
d, g = merge_nearest(d1, i1, lo)
f1, fd, _, _ = nn.nn_top2(metric.to_z(data.astype(np.float64), C), zq)
print(json.dumps({{"same_index": bool(np.array_equal(g.numpy(), f1)), "same_d2": bool(np.array_equal(d.numpy(), fd))}}))
dist.destroy_process_group()
"""


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_search_merge_equals_unsharded(world):
    """The data set split over ranks, each searched alone (oracle scan), and
    the per-query min-loc merge give exactly the unsharded exact answer."""
    outs = run_ranks(SHARD_WORKER.format(root=ROOT), world=world)
    for o in outs:
        r = json.loads(o.strip().splitlines()[-1])
        assert r["same_index"] and r["same_d2"]


def test_reference_arm_line_keeps_the_contract():
    """One process: the reference arm's JSON line carries the keys its
    contract names, on the arm's own workload, metric and unit."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "cube4_N1e4_exact_fp64", "--steps", "3", "--warmup", "3"], cwd=ROOT, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 3 and line["warmup"] == 3
    assert line["config"]["workload"] == "cube4_N1e4_exact_fp64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and isinstance(cb["sample"], str)
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
