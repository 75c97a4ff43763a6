"""The N > 1 launch of bench.py on CPU, over gloo (no GPU needed).

The path shards into independent replicas (one seeded problem per rank, no
collective on the data path), so what N > 1 adds is host logic: the job time is
the slowest rank's (an all-reduce MAX of the per-rank times), and under
torch.distributed.run only rank 0 prints the JSON line of the reference arm
while every rank exits 0.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _max_worker(rank, world, port, values, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    out[rank] = bench.max_over_ranks(values[rank], dist, "cpu")
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    """Every rank gets the slowest rank's time; one rank alone keeps its own."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    values = [1.5, 2.75]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_max_worker, args=(2, _free_port(), values, out), nprocs=2, join=True)
        assert dict(out) == {0: 2.75, 1: 2.75}


def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference launched as two ranks: both exit 0 and exactly one JSON line
    (rank 0's) is printed, with the contract's keys."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--workload", "c1",
           "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    for key in ("metric", "value", "unit", "steps", "warmup", "higher_is_better", "cpu_baseline", "e2e"):
        assert key in line
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
