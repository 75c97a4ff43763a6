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
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--cpu-sample", "c1",
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


# ---------------------------------------------------------------------------
# Wavelength / source sharding of one design problem (the path's multi-GPU form)
# ---------------------------------------------------------------------------
def test_shard_pairs_cover_every_pair_once():
    sys.path.insert(0, ROOT)
    from paper_2307_05388_gb300 import shard as SH
    for n_omega, n_src in ((8, 2), (2, 2), (3, 1), (1, 3), (5, 3)):
        for world in range(1, 11):
            seen = []
            sizes = []
            for rank in range(world):
                pairs = SH.shard_pairs(n_omega, n_src, world, rank)
                sizes.append(sum(len(s) for _, s in pairs))
                seen += [(w, s) for w, ss in pairs for s in ss]
                for ws, ss in SH.context_groups(pairs):
                    assert ws == list(range(ws[0], ws[0] + len(ws))) and ss
            assert sorted(seen) == [(w, s) for w in range(n_omega) for s in range(n_src)]
            assert max(sizes) - min(sizes) <= 1                      # balanced
    # whole wavelengths become one batched context; a split wavelength its own
    assert SH.context_groups(SH.shard_pairs(8, 2, 2, 1)) == [([4, 5, 6, 7], [0, 1])]
    assert SH.context_groups(SH.shard_pairs(3, 2, 4, 1)) == [([0], [1]), ([1], [0])]


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import numpy as np

    import workloads as W
    from paper_2307_05388_gb300 import autograd as AG
    from paper_2307_05388_gb300 import shard as SH
    from tests._oracle_solver import OracleSolver

    wl = W.make_small(22, 19, 4, (6, 5, 8, 7), n_omega=3, n_src=2, seed=31)
    k0 = 2 * np.pi / wl.wavelengths

    def make_problem(ws, ss):
        s = OracleSolver(wl.nx, wl.ny, wl.dx, k0[ws], wl.npml, wl.box)
        b = np.stack([wl.source_dense(i) for i in ss])
        b = np.broadcast_to(b, (len(ws),) + b.shape).copy()
        cols = np.array([wl.monitors[w][i].col for w in ws for i in ss], np.int32)
        g = np.stack([wl.monitors[w][i].values for w in ws for i in ss]).astype(np.complex128)
        return AG.DesignProblem(s, torch.from_numpy(wl.eps_bg.reshape(-1).copy()), torch.from_numpy(b),
                                torch.from_numpy(cols), torch.from_numpy(g))

    sp = SH.ShardedProblem(make_problem, wl.n_omega, wl.n_src, wl.box[2] * wl.box[3], "cpu")
    F, g = sp.iteration(torch.from_numpy(wl.eps_design().reshape(-1).copy()))
    out[rank] = (float(F), g.numpy().copy(), sp.n_pairs)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_iteration_equals_the_whole_problem(world):
    """Each gloo rank solves only its (wavelength, source) pairs (an oracle-backed stand-in for the
    solver); after the all-reduce every rank holds the objective and design gradient of the whole
    problem, equal to the oracle's unsharded design iteration."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import workloads as W
    from oracle import fdfd_oracle as O
    wl = W.make_small(22, 19, 4, (6, 5, 8, 7), n_omega=3, n_src=2, seed=31)
    F_ref, g_ref, _ = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sum(r[2] for r in res.values()) == wl.n_omega * wl.n_src
    for rank in range(world):
        F, g, _ = res[rank]
        assert abs(F - F_ref) <= 1e-12 * abs(F_ref)
        assert O.rel_err(g.reshape(wl.rho.shape) * W.DELTA_EPS, g_ref) <= 1e-12
