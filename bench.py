#!/usr/bin/env python
"""Benchmark of the layout pipeline on the 200k-transaction workload.

One step = the whole hot path on one synthetic transaction graph (200,000
transactions, ~4.8e5 addresses, seed 2): graph build, components, size
split, Kamada-Kawai on the components of at most 50 nodes, and 500
ForceAtlas2 iterations (FMM repulsion, p = 8, leaf 64) on the rest.
Metric: ForceAtlas2 node-updates per second = nodes in ForceAtlas2
components x iterations / step time.

  value  inputs resident in HBM before the timed region (bgl_graph_build_dev,
         bgl_layout_dev); L2 flushed between steps (256 MiB write)
  e2e    the same through the host-memory C ABI (bgl_graph_build,
         bgl_layout): host->device copy of the transaction lists and
         device->host copy of the coordinates inside every step

Multi-GPU: every rank lays out its own replica of the workload (the
components of one graph are independent, nothing is exchanged); value is the
sum of node-updates over ranks divided by the slowest rank's time.

--impl reference times the FP64 oracle (exact repulsion) on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FA2 node-updates/s (FMM vs exact) at stated force error; layout p50/p99 latency"
UNIT = "node-updates/s"
CONFIG_NAME = "fmm-fa2-200k-tx"

# P2P pair throughput peak: a pair issues 8 instructions (7 FP32-pipe ops and
# one MUFU reciprocal); an SM issues 4 warp instructions (128 lanes) per
# clock, so 16 pairs/clk/SM.  The FP32 pipe alone would allow 128 / 7 = 18.3
# pairs/clk/SM; the reciprocal's MUFU rate is measured by bgl_peak_probe.
# The SM count is read from the device, the clock from nvidia-smi.
PAIRS_PER_CLK = 16.0
NEAR_PROFILE = os.path.join(ROOT, "profiles", "near_kernel_fmm_c2_giant.md")
# serving: queued requests with equal parameters share a layout, up to 16 of
# them and 262,144 nodes in all
SERVE_BATCH = (16, 1 << 18)
NEAR_SOURCES = ("fmm.cu", "fmm.cuh", "p2p.cuh")


def near_source_digest() -> str:
    """Digest of the sources the near-field kernel is built from."""
    h = hashlib.sha256()
    for f in NEAR_SOURCES:
        with open(os.path.join(ROOT, "paper_2403_03504_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def near_traffic():
    """DRAM read + write bytes of one near-field launch from the committed ncu
    summary, used only while the kernel's sources are the ones it was
    captured on (the summary records their digest); otherwise None."""
    try:
        with open(NEAR_PROFILE) as fh:
            txt = fh.read()
    except OSError:
        return None, "no ncu summary"
    t = re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt)
    d = re.search(r"source_digest:\s*([0-9a-f]+)", txt)
    if not t or not d:
        return None, "ncu summary without traffic or source digest"
    if d.group(1) != near_source_digest():
        return None, "kernel sources changed since the ncu capture"
    return int(t.group(1)), "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, same sources"


def reduce_units_time(dist, units: float, seconds: float, device=None):
    """Whole-job totals over the ranks: the units all ranks processed and the
    slowest rank's time (every rank calls it; without a process group, the
    rank's own numbers)."""
    if dist is None:
        return units, seconds
    import torch
    t = torch.tensor([units, seconds], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    return float(t[0]), float(tmax[1])


def serve_session(bgl, g, n_requests, rate, seed, iters, min_nodes, max_nodes, slots=4, budget=120 << 30,
                  repulsion=None, batch=None):
    """Poisson arrivals (rate per second) of k-hop layout requests (k uniform
    in 1..4, seeds uniform over the graph's address nodes, redrawn until the
    neighbourhood has min_nodes..max_nodes nodes) served by a bgl Server
    (batch = (requests, nodes): queued requests share layouts up to those
    totals; None: one request per layout); returns latency percentiles
    (arrival -> coordinates on the host), throughput and sizes."""
    import ctypes
    lib = bgl._load()
    rng = np.random.default_rng(seed)
    sizes = g.sizes()
    lo_id, hi_id = sizes["n_nodes"] - sizes["n_addr"], sizes["n_nodes"]
    reqs = []
    n_c, m_c = ctypes.c_int64(), ctypes.c_int64()
    while len(reqs) < n_requests:
        sd, k = int(rng.integers(lo_id, hi_id)), int(rng.integers(1, 5))
        g.ctx.check(lib.bgl_graph_khop(g.h, sd, k, max_nodes, ctypes.byref(n_c), None, ctypes.byref(m_c), None, None))
        if min_nodes <= n_c.value <= max_nodes:
            reqs.append((sd, k, n_c.value))
    gaps = rng.exponential(1.0 / rate, n_requests)
    rep = bgl.REP_FMM if repulsion is None else repulsion
    p = bgl.params(seed=0, fa2_iters=iters, repulsion=rep, fmm_p=8, leaf_size=64, kk_max_nodes=50)
    srv = bgl.Server(g, slots=slots, hbm_budget=budget)
    if batch:
        srv.batching(*batch)
    t0 = time.perf_counter()
    arrive = t0 + np.cumsum(gaps)
    ids = []
    for (sd, k, _), ta in zip(reqs, arrive):
        dt = ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(sd, k, p, max_nodes=max_nodes))
    lat, sub, done, fps, peaks = [], [], [], [], []
    for rid in ids:
        st, n, t, b = srv.wait(rid)
        if st != 0:
            raise RuntimeError(f"serving request failed with status {st}")
        srv.fetch(rid, n)
        sub.append(t[0])
        done.append(t[2])
        lat.append(t[2] - t[0])
        fps.append(int(b[0]))
        peaks.append(int(b[1]))
    inflight = srv.inflight_max()
    batches, batched = srv.batch_stats()
    srv.close()
    lat_ms = 1e3 * np.array(lat)
    wall = max(done) - min(sub)            # the server's steady clock
    nodes = np.array([r[2] for r in reqs])
    return {
        "requests": n_requests, "rate_per_s": rate, "hops": "uniform 1..4", "fa2_iters": iters,
        "repulsion": {bgl.REP_FMM: "fmm p=8", bgl.REP_EXACT: "exact", bgl.REP_AUTO: "auto"}[rep],
        "nodes_min": int(nodes.min()), "nodes_p50": int(np.median(nodes)), "nodes_max": int(nodes.max()),
        "latency_ms_p50": float(np.percentile(lat_ms, 50)), "latency_ms_p99": float(np.percentile(lat_ms, 99)),
        "latency_ms_max": float(lat_ms.max()), "layouts_per_s": n_requests / wall,
        "node_updates_per_s": float(nodes.sum()) * iters / wall, "slots": slots, "hbm_budget_bytes": int(budget),
        "inflight_footprint_max_bytes": int(inflight), "peak_over_estimate_max": float(max(
            pk / fp for pk, fp in zip(peaks, fps))),
        "batching": {"max_requests": batch[0], "max_nodes": batch[1], "shared_layouts": batches,
                     "requests_in_shared_layouts": batched} if batch else None}


def run_serve(args, rank, world, dist, local):
    """Serving on the 3M-transaction graph (seed 4, ~1e7 nodes): Poisson
    stream of 50 requests/s for k-hop neighbourhoods of 100 to 2e6 nodes,
    300 ForceAtlas2 iterations with FMM (KK for components of <= 50 nodes)."""
    import synth
    import paper_2403_03504_gb300 as bgl
    tx = synth.tx_lists(**synth.C4)
    ctx = bgl.Context(local)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    n = args.requests or 100
    out = serve_session(bgl, g, n, 50.0, 5, 300, 100, 2_000_000, slots=args.slots,
                        batch=SERVE_BATCH if args.batch else None)
    if rank == 0:
        print(json.dumps({"metric": "served k-hop layouts: latency (arrival -> coordinates on the host)",
                          "value": out["latency_ms_p99"], "unit": "ms (p99)", "higher_is_better": False,
                          "n_gpus": world, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": "serve-khop-3m-tx", "n_tx": tx.n_tx, "seed": 4,
                                     "n_nodes": g.sizes()["n_nodes"]}, "serving": out}), flush=True)
    g.destroy()
    ctx.close()


def run_precision(args, rank, world, dist, local):
    """Precision study at scale: the 3M-transaction graph (seed 4, ~1e7 nodes),
    200 ForceAtlas2 iterations with FMM p = 12 on its giant component, then,
    at those positions, the repulsion with the M2L in FP32 and in BF16 on the
    tensor cores, each against the FP64 oracle's exact sum on 10,000 sampled
    nodes and against the GPU's FP32 exact sum on every node."""
    import synth
    import oracle
    import paper_2403_03504_gb300 as bgl
    if rank != 0:
        return
    tx = synth.tx_lists(**synth.C4)
    ctx = bgl.Context(local)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    vs = nodes[coff[0]:coff[1]]
    n = len(vs)
    off, _ = g.csr()
    mass = (np.diff(off)[vs] + 1).astype(np.float64)
    x0, y0 = oracle.init_positions(0, vs)
    xy0 = np.stack([x0, y0], 1).astype(np.float32)
    t0 = time.perf_counter()
    xy, _ = g.fa2_step(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=12), 200, xy0)
    run_s = time.perf_counter() - t0
    exact = g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy).astype(np.float64)
    sample = np.sort(np.random.default_rng(0).choice(n, 10_000, replace=False))
    t1 = time.perf_counter()
    o = oracle.fa2_forces(xy[:, 0], xy[:, 1], mass, np.zeros(n + 1, np.int64), np.zeros(0, np.int32),
                          1.0, 1.0, targets=sample)
    oracle_s = time.perf_counter() - t1
    ref = o["frep"]
    den = np.sqrt(np.mean(np.sum(ref ** 2, 1)))
    out = {"n_tx": tx.n_tx, "giant_nodes": n, "fmm_p": 12, "fa2_iters": 200, "fa2_seconds": run_s,
           "oracle_sample": int(len(sample)), "oracle_seconds": oracle_s, "oracle_cores": oracle.threads(),
           "gpu_exact_vs_oracle_rms": float(np.sqrt(np.mean(np.sum((exact[sample] - ref) ** 2, 1))) / den)}
    for name, bf in (("fp32", 0), ("bf16", 1)):
        pq = bgl.params(repulsion=bgl.REP_FMM, fmm_p=12, m2l_bf16=bf)
        f = g.fa2_repulsion(0, pq, xy).astype(np.float64)
        e = np.hypot(*(f[sample] - ref).T) / o["srep"]
        out[name] = {
            "rms_rel_vs_oracle": float(np.sqrt(np.mean(np.sum((f[sample] - ref) ** 2, 1))) / den),
            "max_norm_err_vs_oracle": float(e.max()),
            "rms_rel_vs_gpu_exact": float(np.sqrt(np.mean(np.sum((f - exact) ** 2, 1)) /
                                                  np.mean(np.sum(exact ** 2, 1)))),
            "ms_down": g.fmm_stats(0, pq, xy, reps=3)["ms_down"],
        }
        out[name]["ms_total"] = g.fmm_stats(0, pq, xy, reps=3)["ms_total"]
    print(json.dumps({"metric": "FMM M2L precision at scale: RMS relative repulsion error vs the FP64 oracle",
                      "value": out["bf16"]["rms_rel_vs_oracle"], "unit": "relative RMS (BF16 M2L)",
                      "higher_is_better": False, "n_gpus": world, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "precision-3m-tx", "seed": 4}, "precision": out}), flush=True)
    g.destroy()
    ctx.close()


def c3_edges():
    """The batched-components graph: 1e5 forest components of 3-200 nodes,
    then 2e3 of 200-5,000 (node ids consecutive per component)."""
    import synth
    ss, us, vs = synth.forest(**synth.C3_SMALL)
    sm, um, vm = synth.forest(**synth.C3_MID)
    n_small = int(ss.sum())
    n = n_small + int(sm.sum())
    u = np.concatenate([us, um + n_small]).astype(np.int32)
    v = np.concatenate([vs, vm + n_small]).astype(np.int32)
    return n, u, v


def c3_kk_kernels(bgl, local):
    """Profiling case: the Kamada-Kawai size classes of the batched layout
    alone (no ForceAtlas2 iterations), twice, launched from the host."""
    import torch
    n, u, v = c3_edges()
    ctx = bgl.Context(local)
    g = bgl.Graph.from_edges(ctx, n, u, v)
    g.components(labels=False)
    p_kk = bgl.params(seed=0, fa2_iters=0, repulsion=bgl.REP_AUTO, kk_max_nodes=200)
    d_xy = torch.empty((n, 2), dtype=torch.float32, device=torch.device("cuda", local))
    ms = []
    for _ in range(2):
        t = time.perf_counter()
        g.layout_dev(p_kk, d_xy)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t) * 1e3)
    print(json.dumps({"kernels_only": True, "workload": "c3-kk", "kk_components": int(g.split(200)[0]),
                      "layout_ms": ms}))
    g.destroy()
    ctx.close()


def c3_measure(bgl, local, steps, warmup, iters=50, rank=0, world=1, dist=None):
    """Batched components: 100,000 forest components of 3-200 nodes (KK, at
    most 200 nodes) and 2,000 of 200-5,000 nodes (ForceAtlas2, exact or FMM
    repulsion chosen per component size by measurement), one layout per step:
    the KK size classes run beside the ForceAtlas2 iterations in one graph
    launch.  With several ranks each lays out its share of the components
    (longest-processing-time packing).  Returns the step times, the KK-only
    times and the ForceAtlas2 node-updates/s."""
    import torch
    from paper_2403_03504_gb300 import shard

    n, u, v = c3_edges()
    ctx = bgl.Context(local)
    stream = torch.cuda.Stream(device=torch.device("cuda", local))
    ctx.set_stream(stream)
    iters = min(iters, 50)
    p = bgl.params(seed=0, fa2_iters=iters, repulsion=bgl.REP_AUTO, fmm_min_nodes=-1, kk_max_nodes=200)
    p_kk = bgl.params(seed=0, fa2_iters=0, repulsion=bgl.REP_AUTO, fmm_min_nodes=-1, kk_max_nodes=200)
    g_all = bgl.Graph.from_edges(ctx, n, u, v)
    g_all.components(labels=False)
    n_kk_all, n_fa2_all = g_all.split(200)
    coff, _, nodes = g_all.component_nodes()
    if world > 1:
        # this rank's share: every node id, the edges of its components only
        costs = shard.component_costs(np.diff(coff), 200, iters, p.kk_sweeps, shard.REP_EXACT)
        owner, _ = shard.lpt_assign(costs, world)
        own = shard.node_owner(coff, nodes, owner, n)
        u, v = shard.share_edges(u, v, own, rank)
        g_all.destroy()
        g = bgl.Graph.from_edges(ctx, n, u, v)
        g.components(labels=False)
    else:
        g = g_all
    n_kk, n_fa2 = g.split(200)
    coff_r, _, _ = g.component_nodes()
    fa2_nodes = int(coff_r[n_fa2])
    d_xy = torch.empty((n, 2), dtype=torch.float32, device=torch.device("cuda", local))

    def timed(params, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, b in ev:
            with torch.cuda.stream(stream):
                a.record(stream)
            g.layout_dev(params, d_xy)
            with torch.cuda.stream(stream):
                b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    for _ in range(max(warmup, 3)):
        g.layout_dev(p, d_xy)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = bgl.launch_count()
    step_ms = timed(p, steps)
    launches = (bgl.launch_count() - launches0) // max(steps, 1)
    kk_ms = timed(p_kk, steps)
    upd, total_s = reduce_units_time(dist, float(fa2_nodes) * iters * steps, sum(step_ms) / 1e3,
                                     torch.device("cuda", local))
    out = {"workload": "c3-batched-100k", "n_nodes": n, "kk_components": int(n_kk_all),
           "fa2_components": int(n_fa2_all), "fa2_iters": iters, "kk_max_nodes": 200, "kk_sweeps": 200,
           "repulsion": "auto, exact/FMM crossover measured (fmm_min_nodes = -1)",
           "ms_per_step": 1e3 * total_s / steps, "step_ms": step_ms, "kk_only_ms": kk_ms,
           "fa2_node_updates_per_s": upd / total_s, "layouts_per_s": steps / total_s,
           "gpu_launches_per_step": int(launches)}
    g.destroy()
    ctx.close()
    return out


def run_c3(args, rank, world, dist, local):
    """The batched-components workload as its own bench line."""
    import paper_2403_03504_gb300 as bgl
    if args.kernels_only:
        if rank == 0:
            c3_kk_kernels(bgl, local)
        return
    c3 = c3_measure(bgl, local, args.steps, args.warmup, args.iters, rank, world, dist)
    if rank == 0:
        print(json.dumps({
            "metric": "C3 batched layout: FA2 node-updates/s with KK on 1e5 components",
            "value": c3["fa2_node_updates_per_s"], "unit": "node-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": c3["ms_per_step"], "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "dtype": "f32", "data": "synthetic",
            "config": {k: c3[k] for k in ("workload", "n_nodes", "kk_components", "fa2_components", "fa2_iters",
                                          "kk_max_nodes", "kk_sweeps", "repulsion")},
            "kk_only_ms": c3["kk_only_ms"], "layouts_per_s": c3["layouts_per_s"],
            "gpu_launches": c3["gpu_launches_per_step"], "step_ms": c3["step_ms"]}), flush=True)


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def oracle_force_error(bgl, g, giant_xy, n_sample=2000, seed=2):
    """FMM repulsion at the final layout against the FP64 oracle's exact sum on
    a uniform sample of the giant component's nodes: RMS relative error and
    the largest normalised error e_i = |dF_i| / (kr m_i sum_j m_j / d_ij),
    for p = 8 and p = 16, beside each one's truncation ceiling."""
    import oracle
    coff, _, nodes = g.component_nodes()
    off, adj = g.csr()
    vs = nodes[coff[0]:coff[1]]
    pos = np.full(len(off) - 1, -1, np.int64)
    pos[vs] = np.arange(len(vs))
    loff = np.zeros(len(vs) + 1, np.int64)
    loff[1:] = np.cumsum(np.diff(off)[vs])
    ladj = pos[np.concatenate([adj[off[v]:off[v + 1]] for v in vs])].astype(np.int32)
    mass = np.diff(loff) + 1.0
    sample = np.sort(np.random.default_rng(seed).choice(len(vs), n_sample, replace=False))
    t0 = time.perf_counter()
    o = oracle.fa2_forces(giant_xy[:, 0], giant_xy[:, 1], mass, loff, ladj, 1.0, 1.0, targets=sample)
    out = {"oracle_sample": n_sample, "oracle_seconds": time.perf_counter() - t0}
    rho = 2 ** 0.5 / (4 - 2 ** 0.5)
    ref = o["frep"]
    for pp in (8, 16):
        f = g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=pp, leaf_size=64), giant_xy)[sample]
        e = np.hypot(*(f - ref).T) / o["srep"]
        out[f"p{pp}_rms_rel_vs_oracle"] = float(np.sqrt(np.mean(np.sum((f - ref) ** 2, 1)) /
                                                        np.mean(np.sum(ref ** 2, 1))))
        out[f"p{pp}_max_e_vs_oracle"] = float(e.max())
        out[f"p{pp}_ceiling"] = max(2 * (1 + rho) * rho ** (pp + 1) / (1 - rho), 2e-5)
    return out


def cpu_oracle_rate(tx, budget_s: float, giant_only=True):
    """Exact FP64 ForceAtlas2 force evaluations per second on the giant
    component, timed on a bounded sample of target nodes (each node update
    is one full force evaluation plus an O(1) step)."""
    import oracle
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    label, _ = oracle.components(og.off, og.adj)
    comp_off, _, nodes = oracle.component_order(label)
    vs = nodes[comp_off[0]:comp_off[1]]
    pos = np.full(og.n_nodes, -1, np.int64)
    pos[vs] = np.arange(len(vs))
    loff = np.zeros(len(vs) + 1, np.int64)
    loff[1:] = np.cumsum(np.diff(og.off)[vs])
    ladj = pos[np.concatenate([og.adj[og.off[v]:og.off[v + 1]] for v in vs])].astype(np.int32)
    mass = np.diff(loff) + 1.0
    x, y = oracle.init_positions(0, vs)
    rng = np.random.default_rng(0)
    k = 64
    t0 = time.perf_counter()
    oracle.fa2_forces(x, y, mass, loff, ladj, targets=rng.choice(len(vs), k, replace=False))
    dt = time.perf_counter() - t0
    k2 = int(max(64, min(len(vs), k * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.fa2_forces(x, y, mass, loff, ladj, targets=rng.choice(len(vs), k2, replace=False))
    dt2 = time.perf_counter() - t0
    return dict(value=k2 / dt2, unit=UNIT, cores=oracle.threads(), kind="oracle",
                sample=f"exact FP64 forces (repulsion, attraction, gravity) of {k2} random nodes of the "
                       f"{len(vs)}-node giant component at its initial positions, {dt2:.1f} s; "
                       f"node-updates/s = nodes evaluated / time"), len(vs)


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: node-updates/s on bounded samples."""
    if rank != 0:
        return
    import synth
    import oracle
    tx = synth.tx_lists(**synth.C2)
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    label, _ = oracle.components(og.off, og.adj)
    comp_off, _, nodes = oracle.component_order(label)
    vs = nodes[comp_off[0]:comp_off[1]]
    pos = np.full(og.n_nodes, -1, np.int64)
    pos[vs] = np.arange(len(vs))
    loff = np.zeros(len(vs) + 1, np.int64)
    loff[1:] = np.cumsum(np.diff(og.off)[vs])
    ladj = pos[np.concatenate([og.adj[og.off[v]:og.off[v + 1]] for v in vs])].astype(np.int32)
    mass = np.diff(loff) + 1.0
    x, y = oracle.init_positions(0, vs)
    rng = np.random.default_rng(0)
    per_step = 512
    for _ in range(args.warmup):
        oracle.fa2_forces(x, y, mass, loff, ladj, targets=rng.choice(len(vs), 32, replace=False))
    times = []
    for _ in range(args.steps):
        tg = rng.choice(len(vs), per_step, replace=False)
        t0 = time.perf_counter()
        oracle.fa2_forces(x, y, mass, loff, ladj, targets=tg)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    sample = (f"per step: exact FP64 forces of {per_step} random nodes of the {len(vs)}-node giant component "
              f"(one node update each)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CONFIG_NAME, "n_tx": 200000, "seed": 2, "giant_nodes": int(len(vs))},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bgl", choices=["bgl", "reference"])
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--leaf", type=int, default=64, help="FMM leaf size (points per leaf box at most)")
    ap.add_argument("--exact-iters", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-c3", action="store_true", help="leave the batched-components object out of the line")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "serve", "precision"],
                    help="c2: the headline 200k-transaction graph; c3: 1e5 small + 2e3 mid-size components; "
                         "serve: k-hop layout requests on the 3M-transaction graph; "
                         "precision: FP32 against BF16 M2L on the 3M-transaction graph's giant component")
    ap.add_argument("--requests", type=int, default=0, help="serving requests (0: 40 in the c2 line, 100 for serve)")
    ap.add_argument("--slots", type=int, default=4, help="serving workers")
    ap.add_argument("--batch", type=int, default=1, help="serving: 1 batches queued requests (SERVE_BATCH), 0 does not")
    ap.add_argument("--timed-only", action="store_true",
                    help="profiling case: warm-up and timed steps only (no end-to-end leg, no diagnostics); "
                         "prints the device-resident step times")
    ap.add_argument("--kernels-only", action="store_true",
                    help="profiling case: FMM and exact repulsion on the giant component only "
                         "(with --workload c3: the Kamada-Kawai classes of the batched layout only)")
    ap.add_argument("--positions", default="",
                    help="with --kernels-only: giant-component positions from this .npy file "
                         "(written by --save-positions) instead of N(0, 300^2) points")
    ap.add_argument("--save-positions", default="",
                    help="write the giant component's final positions of the timed layout to this .npy file")
    args = ap.parse_args()
    rank, world, local = env_rank()

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import synth
    import paper_2403_03504_gb300 as bgl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload in ("c3", "serve", "precision"):
        {"c3": run_c3, "serve": run_serve, "precision": run_precision}[args.workload](args, rank, world, dist, local)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    tx = synth.tx_lists(**synth.C2)
    stream = torch.cuda.Stream(device=dev)
    ctx = bgl.Context(local)
    ctx.set_stream(stream)
    p = bgl.params(seed=0, fa2_iters=args.iters, repulsion=bgl.REP_AUTO, fmm_p=args.p, leaf_size=args.leaf,
                   kk_max_nodes=50, fmm_min_nodes=8192)

    # device-resident inputs
    d_in = [torch.from_numpy(a).to(dev) for a in (tx.in_off, tx.in_addr.view(np.int64), tx.out_off,
                                                  tx.out_addr.view(np.int64))]
    # pinned host inputs / output for the end-to-end leg
    h_in = [torch.from_numpy(a).pin_memory() for a in (tx.in_off, tx.in_addr.view(np.int64), tx.out_off,
                                                       tx.out_addr.view(np.int64))]
    torch.cuda.synchronize()

    g0 = bgl.Graph.build_dev(ctx, tx.n_tx, len(tx.in_addr), len(tx.out_addr), *d_in)
    g0.components(labels=False)
    if args.kernels_only:
        # a few launches of each repulsion kernel on the 5.5e5-node giant component
        coff, _, nodes = g0.component_nodes()
        if args.positions:
            xy0 = np.ascontiguousarray(np.load(args.positions), dtype=np.float32)
            assert xy0.shape == (int(coff[1] - coff[0]), 2), xy0.shape
        else:
            xy0 = np.random.default_rng(0).normal(0, 300, (int(coff[1] - coff[0]), 2)).astype(np.float32)
        for _ in range(3):
            g0.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=args.p), xy0)
        g0.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy0)
        # three whole ForceAtlas2 iterations (FMM, attraction, gravity, speed, update)
        g0.fa2_step(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=args.p), 3, xy0)
        ctx.sync()
        print(json.dumps({"kernels_only": True, "giant": int(coff[1] - coff[0])}))
        return
    n_nodes = g0.sizes()["n_nodes"]
    n_kk, n_fa2 = g0.split(p.kk_max_nodes)
    coff, _, nodes = g0.component_nodes()
    fa2_nodes = int(coff[n_fa2])
    giant = int(coff[1] - coff[0])
    d_xy = torch.empty((n_nodes, 2), dtype=torch.float32, device=dev)
    h_xy = torch.empty((n_nodes, 2), dtype=torch.float32).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step_dev():
        g = bgl.Graph.build_dev(ctx, tx.n_tx, len(tx.in_addr), len(tx.out_addr), *d_in)
        g.components(labels=False)
        g.layout_dev(p, d_xy)
        g.destroy()

    def step_e2e():
        g = bgl.Graph.build(ctx, *(t.numpy() for t in h_in[:1]), h_in[1].numpy().view(np.uint64),
                            h_in[2].numpy(), h_in[3].numpy().view(np.uint64))
        g.components(labels=False)
        g.layout(p, out=h_xy.numpy())
        g.destroy()

    for _ in range(args.warmup if args.timed_only else max(args.warmup, 3)):
        step_dev()
    ctx.sync()

    # ---------------------------------------------------------------- timed: device-resident
    launches0 = bgl.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))                     # L2 flush, outside the event pair
                ev[k][0].record(stream)
            step_dev()
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = (bgl.launch_count() - launches0) // max(args.steps, 1)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    if args.timed_only:
        if rank == 0:
            # launches_before: the library's kernel launches before the timed
            # region (a profiler's skip count, plus the framework's own kernels)
            print(json.dumps({"timed_only": True, "step_ms": step_ms, "gpu_launches": int(launches),
                              "launches_before": int(launches0)}), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    total_s = sum(step_ms) / 1e3
    upd_rank = float(fa2_nodes) * args.iters * args.steps
    upd, total_s = reduce_units_time(dist, upd_rank, total_s, dev)
    value = upd / total_s

    # ---------------------------------------------------------------- timed: end to end (host buffers)
    step_e2e()
    e2e_times = []
    if dist:
        dist.barrier()
    for k in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_e2e()
        e2e_times.append(time.perf_counter() - t0)
    e2e_upd, e2e_s = reduce_units_time(dist, upd_rank, sum(e2e_times), dev)
    e2e_value = e2e_upd / e2e_s
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = h_xy.numel() * 4 + 8 * (len(coff))          # coordinates + component offsets

    # ---------------------------------------------------------------- diagnostics (not timed)
    xy_final = d_xy.cpu().numpy()
    giant_xy = np.ascontiguousarray(xy_final[nodes[coff[0]:coff[1]]])
    if args.save_positions:
        np.save(args.save_positions, giant_xy)
    stats = g0.fmm_stats(0, p, giant_xy, reps=5)
    leaf_s = stats["ms_near"] / 1e3
    achieved = stats["p2p_pairs"] / leaf_s
    exact = bgl.params(seed=0, repulsion=bgl.REP_EXACT)
    g0.fa2_step(0, exact, 1, giant_xy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g0.fa2_step(0, exact, args.exact_iters, giant_xy)
    exact_s = time.perf_counter() - t0
    exact_rate = giant * args.exact_iters / exact_s
    f_ex = g0.fa2_repulsion(0, exact, giant_xy)
    errs = {}
    for pp in (8, 16):
        f_f = g0.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=pp), giant_xy)
        rms = float(np.sqrt(np.mean(np.sum((f_f - f_ex) ** 2, 1)) / np.mean(np.sum(f_ex ** 2, 1))))
        errs[f"p{pp}_rms_rel"] = rms
    # M2L precision study at p = 12: FP32 CUDA cores versus BF16 tensor cores
    m2l_prec = {"fmm_p": 12, "reference": "GPU FP32 exact sum at the final layout"}
    for name, bf in (("fp32", 0), ("bf16", 1)):
        pq = bgl.params(repulsion=bgl.REP_FMM, fmm_p=12, m2l_bf16=bf)
        f_f = g0.fa2_repulsion(0, pq, giant_xy)
        m2l_prec[f"{name}_rms_rel"] = float(np.sqrt(np.mean(np.sum((f_f - f_ex) ** 2, 1)) /
                                                    np.mean(np.sum(f_ex ** 2, 1))))
        st = g0.fmm_stats(0, pq, giant_xy, reps=5)
        m2l_prec[f"{name}_ms_down"] = st["ms_down"]
        m2l_prec[f"{name}_ms_total"] = st["ms_total"]
    m2l_prec["m2l_translations"] = stats["m2l"]
    p16 = bgl.params(seed=0, fa2_iters=args.iters, repulsion=bgl.REP_AUTO, fmm_p=16)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = bgl.Graph.build_dev(ctx, tx.n_tx, len(tx.in_addr), len(tx.out_addr), *d_in)
    g.components(labels=False)
    g.layout_dev(p16, d_xy)
    g.destroy()
    torch.cuda.synchronize()
    p16_s = time.perf_counter() - t0

    # the assembly into one frame (Section 4): the same layout with and without it
    p_asm = bgl.params(**{k: getattr(p, k) for k, _ in bgl.Params._fields_})
    p_asm.assemble = 1
    asm_ms = []
    for params_k in (p, p_asm, p, p_asm):
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a_ev.record(stream)
        g0.layout_dev(params_k, d_xy)
        with torch.cuda.stream(stream):
            b_ev.record(stream)
        torch.cuda.synchronize()
        asm_ms.append(a_ev.elapsed_time(b_ev))
    assembly = {"ms": 0.5 * ((asm_ms[1] - asm_ms[0]) + (asm_ms[3] - asm_ms[2])), "components": int(len(coff) - 1),
                "kk_max_nodes": int(p.kk_max_nodes)}

    # served layouts of k-hop neighbourhoods of this graph (latency)
    serving = serve_session(bgl, g0, args.requests or 40, 50.0, 2, 300, 100, 2_000_000, slots=4, budget=64 << 30)
    # the same requests, up to 60k nodes each, with FMM and with exact repulsion
    # the same 40 requests served with FMM and with exact repulsion, with
    # batching on (it takes the exact ones), and exact one request per layout
    serving_vs_exact = {name: serve_session(bgl, g0, args.requests or 40, 50.0, 3, 300, 100, 60_000, slots=4,
                                            budget=64 << 30, repulsion=rep, batch=bt)
                        for name, rep, bt in (("fmm", bgl.REP_FMM, SERVE_BATCH), ("exact", bgl.REP_EXACT, SERVE_BATCH),
                                              ("exact_unbatched", bgl.REP_EXACT, None))}

    clocks = clk.summary()
    # the batched-components workload (10^5 KK + 2,000 ForceAtlas2 components), two steps
    c3 = c3_measure(bgl, local, 2, 3) if world == 1 and not args.no_c3 else None
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    probe = ctx.peak_probe()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = clocks.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or 2070.0
    pair_peak = sms * sm_max_mhz * 1e6 * PAIRS_PER_CLK
    traffic, traffic_note = near_traffic()
    cpu = None
    if not args.no_cpu and world == 1:
        cpu, _ = cpu_oracle_rate(tx, args.cpu_budget)
        errs.update(oracle_force_error(bgl, g0, giant_xy))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": CONFIG_NAME, "n_tx": tx.n_tx, "seed": 2, "n_nodes": n_nodes,
                   "fa2_nodes": fa2_nodes, "giant_nodes": giant, "kk_components": n_kk, "fa2_iters": args.iters,
                   "repulsion": "fmm", "fmm_p": args.p, "leaf_size": args.leaf, "kk_max_nodes": 50, "kk_sweeps": 200,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": "fmm near field (P2P, near_kernel)", "achieved": achieved / 1e9,
                     "peak": pair_peak / 1e9, "unit": "Gpairs/s", "frac": achieved / pair_peak,
                     "traffic": traffic, "traffic_unit": "bytes per launch", "traffic_source": traffic_note,
                     "peak_source": f"derived: {sms} SMs (device) x {sm_max_mhz:.0f} MHz (nvidia-smi max) x 128 "
                                    "issue lanes/clk / 8 instructions per pair = 16 pairs/clk/SM",
                     "peak_probe": probe},
        "force_error": {"reference": "GPU FP32 exact sum at the final layout (rms_rel); FP64 oracle on 2000 "
                                     "sampled nodes (vs_oracle)", **errs},
        "serving_vs_exact": serving_vs_exact,
        "c3": c3,
        "exact_fa2": {"value": exact_rate, "unit": UNIT, "iters": args.exact_iters, "nodes": giant},
        "fmm_p16_step_ms": 1e3 * p16_s,
        "m2l_precision": m2l_prec,
        "assembly": assembly,
        "serving": serving,
        "fmm_profile": stats,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "step_ms": step_ms,
        "e2e_step_ms": [1e3 * t for t in e2e_times],
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
