"""The multi-process paths of bench.py on the CPU (gloo, world size 2).

With N GPUs every rank lays out its own replica of the workload (the
components are independent, nothing is exchanged), and the reported value is
the units all ranks processed divided by the slowest rank's time.  The GPU
part needs GPUs; its over-ranks arithmetic and the reference arm's
single-printer rule do not, and are checked here."""
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
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, secs = bench.reduce_units_time(dist, float(1000 * (rank + 1)), 0.5 + rank, torch.device("cpu"))
    out[rank] = (units, secs)
    dist.barrier()
    dist.destroy_process_group()


def test_rate_over_ranks_sums_units_and_takes_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (3000.0, 1.5)


def test_rate_without_process_group():
    import bench
    assert bench.reduce_units_time(None, 7.0, 2.0) == (7.0, 2.0)


def test_reference_arm_under_torchrun_prints_one_line():
    """Two ranks on gloo: rank 0 times the FP64 oracle and prints one JSON
    line, the other exits without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"
