"""The multi-process paths of bench.py on the CPU (gloo, world size 2).

With N GPUs every rank lays out its own replica of the workload (the
components are independent, nothing is exchanged), and the reported value is
the units all ranks processed divided by the slowest rank's time.  The GPU
part needs GPUs; its over-ranks arithmetic and the reference arm's
single-printer rule do not, and are checked here.  So is the sharding of one
graph's components over ranks (Section 4: components are independent):
longest-processing-time packing within Graham's bound, the cost model's
agreement with the library, and two gloo ranks whose merged layout (the
oracle's, on the host) equals the one-rank layout bit for bit."""
import json
import os
import socket
import subprocess
import sys

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


# ------------------------------------------------- components sharded across ranks

def test_lpt_assigns_every_component_once_within_the_bound():
    """LPT on random costs: each item has one rank; on small instances the
    largest load is within (4/3 - 1/(3m)) of the brute-force optimum."""
    import itertools
    import numpy as np
    from paper_2403_03504_gb300 import shard
    rng = np.random.default_rng(5)
    for trial in range(40):
        m = int(rng.integers(2, 4))
        k = int(rng.integers(1, 10))
        costs = rng.integers(1, 100, k).astype(float)
        owner, load = shard.lpt_assign(costs, m)
        assert owner.shape == (k,) and set(owner) <= set(range(m))
        assert np.allclose(np.bincount(owner, weights=costs, minlength=m), load)
        best = min(max(np.bincount(np.array(a), weights=costs, minlength=m))
                   for a in itertools.product(range(m), repeat=k))
        assert load.max() <= (4 / 3 - 1 / (3 * m)) * best + 1e-9, (costs, m, load, best)


def test_cost_model_follows_the_split():
    import numpy as np
    from paper_2403_03504_gb300 import shard
    c = shard.component_costs([1, 2, 50, 51, 9000], kk_max_nodes=50, fa2_iters=10, kk_sweeps=200,
                              repulsion=shard.REP_AUTO, fmm_min_nodes=8192)
    assert c[0] == 0 and c[1] == 4 * 200 and c[2] == 2500 * 200
    assert c[3] == 51 ** 2 * 10 and c[4] == shard.FMM_PAIRS_PER_NODE * 9000 * 10


def test_cost_model_mirrors_the_library():
    """The planner's repulsion codes, its default crossover and its exact/FMM
    rule are the library's (header enum, bgl_params_default, and AUTO using
    the FMM from fmm_min_nodes nodes on)."""
    import re
    import paper_2403_03504_gb300 as bgl
    from paper_2403_03504_gb300 import shard
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bgl.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"BGL_REP_(EXACT|FMM|AUTO) = (\d+)", hdr))
    assert (shard.REP_EXACT, shard.REP_FMM, shard.REP_AUTO) == (enum["EXACT"], enum["FMM"], enum["AUTO"])
    assert (bgl.REP_EXACT, bgl.REP_FMM, bgl.REP_AUTO) == (enum["EXACT"], enum["FMM"], enum["AUTO"])
    p = bgl.params()
    import inspect
    defaults = inspect.signature(shard.component_costs).parameters
    assert defaults["fmm_min_nodes"].default == p.fmm_min_nodes
    for name in ("repulsion", "kk_max_nodes", "fa2_iters", "kk_sweeps"):
        assert defaults[name].default == getattr(p, name), name
    m = p.fmm_min_nodes
    c = shard.component_costs([m - 1, m], kk_max_nodes=50, fa2_iters=1, repulsion=shard.REP_AUTO, fmm_min_nodes=m)
    assert c[0] == (m - 1) ** 2 and c[1] == shard.FMM_PAIRS_PER_NODE * m


def _shard_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import oracle
    import synth
    from paper_2403_03504_gb300 import shard
    tx = synth.tx_lists(**synth.C1)
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    label, _ = oracle.components(og.off, og.adj)
    comp_off, _, nodes = oracle.component_order(label)
    costs = shard.component_costs(np.diff(comp_off), 50, 3, 5, shard.REP_EXACT)

    def layout_fn(n, s, d):
        return oracle.layout(oracle.graph_from_edges(n, s, d), fa2_iters=3, kk_sweeps=5, seed=1)

    merged, piece, comp_owner = shard.layout_sharded(og.n_nodes, og.src, og.dst, comp_off, nodes, costs, rank,
                                                     world, layout_fn, dist)
    out[rank] = (merged, len(piece[0]), comp_owner)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_layout_equals_one_rank_layout():
    """Two gloo ranks lay out their shares of the 1,000-transaction graph's
    components (the oracle as the layout) and gather: the merged result is
    bitwise the one-rank layout, every component laid out by one rank."""
    import numpy as np
    import oracle
    import synth
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    tx = synth.tx_lists(**synth.C1)
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    want = oracle.layout(og, fa2_iters=3, kk_sweeps=5, seed=1).astype(np.float32)
    assert np.array_equal(res[0][0], want) and np.array_equal(res[1][0], want)
    assert res[0][1] + res[1][1] == og.n_nodes
    assert np.array_equal(res[0][2], res[1][2]) and set(res[0][2]) == {0, 1}
