"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package; the layout library never does.  It wraps
``oracle.c`` (compiled here with gcc, OpenMP, no fast-math, no FMA
contraction) with numpy-facing functions, and composes them into the whole
layout of Section 4 (``layout``) in plain Python.

Paper map: Section 2 -> graph_build / undirected_csr; Section 4 ->
components / component_order / layout; Section 3.1 -> bfs_apsp,
floyd_warshall, kk_*; Section 3.2 -> fa2_forces, fa2_energy, fa2_run.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "orc_splitmix64_stream": ([ctypes.c_uint64, _I64, _VP], None),
                "orc_init_positions": ([ctypes.c_uint64, _I64, _VP, _VP, _VP], None),
                "orc_graph_build": ([_I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I64),
                "orc_undirected_csr": ([_I64, _I64, _VP, _VP, _VP, _VP], _I64),
                "orc_components": ([_I64, _VP, _VP, _VP], _I64),
                "orc_component_order": ([_I64, _VP, _VP, _VP, _VP], _I64),
                "orc_bfs_apsp": ([_I64, _VP, _VP, _VP], None),
                "orc_floyd_warshall": ([_I64, _VP, _VP, _VP], None),
                "orc_kk_energy": ([_I64, _VP, _VP, _VP, _D], _D),
                "orc_kk_grad_hess": ([_I64, _VP, _VP, _VP, _D, _I64, _VP], None),
                "orc_kk_run": ([_I64, _VP, _VP, _VP, _D, _I64, _D, _VP, _VP], _I64),
                "orc_fa2_forces": ([_I64, _VP, _VP, _VP, _VP, _VP, _D, _D, _I64, _VP] + [_VP] * 8, None),
                "orc_fa2_energy": ([_I64, _VP, _VP, _VP, _VP, _VP, _D, _D], _D),
                "orc_fa2_run": ([_I64, _VP, _VP, _VP, _VP, _VP, _D, _D, _D, _D, _D, ctypes.c_int32,
                                 _I64, _VP, _VP, _VP, _VP], None),
                "orc_threads": ([], ctypes.c_int),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_VP)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def threads() -> int:
    return int(_load().orc_threads())


# ---------------------------------------------------------------- Section 2

@dataclass
class Graph:
    n_tx: int
    n_nodes: int
    addr: np.ndarray      # uint64 [n_addr], address key of node n_tx + k
    src: np.ndarray       # int32 [m] directed edges sorted by (src, dst)
    dst: np.ndarray
    off: np.ndarray       # int64 [n+1] undirected CSR
    adj: np.ndarray       # int32 [2E]
    n_undirected: int

    @property
    def deg(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int32)


def graph_build(in_off, in_addr, out_off, out_addr) -> Graph:
    lib = _load()
    in_off = _c(in_off, np.int64)
    out_off = _c(out_off, np.int64)
    in_addr = _c(in_addr, np.uint64)
    out_addr = _c(out_addr, np.uint64)
    n_tx = len(in_off) - 1
    total = int(in_off[-1] + out_off[-1])
    addr = np.zeros(max(total, 1), np.uint64)
    src = np.zeros(max(total, 1), np.int32)
    dst = np.zeros(max(total, 1), np.int32)
    ne = ctypes.c_int64()
    n_addr = lib.orc_graph_build(n_tx, _p(in_off), _p(in_addr), _p(out_off), _p(out_addr),
                                 _p(addr), _p(src), _p(dst), ctypes.byref(ne))
    n = n_tx + n_addr
    src, dst = src[:ne.value].copy(), dst[:ne.value].copy()
    off, adj, E = undirected_csr(n, src, dst)
    return Graph(n_tx, n, addr[:n_addr].copy(), src, dst, off, adj, E)


def graph_from_edges(n, u, v) -> Graph:
    """Generic graph on nodes 0..n-1 (Section 5: other domains)."""
    u = _c(u, np.int32)
    v = _c(v, np.int32)
    pairs = np.unique(np.stack([u, v], 1), axis=0) if len(u) else np.zeros((0, 2), np.int32)
    src = np.ascontiguousarray(pairs[:, 0], np.int32)
    dst = np.ascontiguousarray(pairs[:, 1], np.int32)
    off, adj, E = undirected_csr(n, src, dst)
    return Graph(0, n, np.zeros(0, np.uint64), src, dst, off, adj, E)


def undirected_csr(n, src, dst):
    lib = _load()
    src = _c(src, np.int32)
    dst = _c(dst, np.int32)
    off = np.zeros(n + 1, np.int64)
    adj = np.zeros(max(2 * len(src), 1), np.int32)
    E = lib.orc_undirected_csr(n, len(src), _p(src), _p(dst), _p(off), _p(adj))
    return off, adj[:2 * E].copy(), int(E)


# ---------------------------------------------------------------- Section 4

def components(off, adj):
    lib = _load()
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    n = len(off) - 1
    label = np.zeros(n, np.int32)
    nc = lib.orc_components(n, _p(off), _p(adj), _p(label))
    return label, int(nc)


def component_order(label):
    """(comp_off[int64 nc+1], comp_label[int32 nc], nodes[int32 n]) ordered by size desc, label asc."""
    lib = _load()
    label = _c(label, np.int32)
    n = len(label)
    comp_off = np.zeros(n + 1, np.int64)
    comp_label = np.zeros(max(n, 1), np.int32)
    nodes = np.zeros(max(n, 1), np.int32)
    nc = lib.orc_component_order(n, _p(label), _p(comp_off), _p(comp_label), _p(nodes))
    return comp_off[:nc + 1].copy(), comp_label[:nc].copy(), nodes[:n].copy()


def subgraph(off, adj, nodes):
    """CSR of the subgraph induced by `nodes` (ascending), with local ids."""
    nodes = np.asarray(nodes, np.int64)
    loc = {int(v): i for i, v in enumerate(nodes)}
    loff = np.zeros(len(nodes) + 1, np.int64)
    rows = []
    for i, v in enumerate(nodes):
        r = [loc[int(w)] for w in adj[off[v]:off[v + 1]] if int(w) in loc]
        rows.append(r)
        loff[i + 1] = loff[i] + len(r)
    ladj = np.array([w for r in rows for w in r], np.int32)
    return loff, ladj


# ---------------------------------------------------------------- Section 3.1

def bfs_apsp(off, adj):
    lib = _load()
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    n = len(off) - 1
    d = np.zeros((n, n), np.int32)
    lib.orc_bfs_apsp(n, _p(off), _p(adj), _p(d))
    return d


def floyd_warshall(off, adj):
    lib = _load()
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    n = len(off) - 1
    d = np.zeros((n, n), np.int32)
    lib.orc_floyd_warshall(n, _p(off), _p(adj), _p(d))
    return d


def kk_energy(x, y, d, l=1.0) -> float:
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    d = _c(d, np.int32)
    return float(_load().orc_kk_energy(len(x), _p(x), _p(y), _p(d), l))


def kk_grad_hess(x, y, d, l, m):
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    d = _c(d, np.int32)
    out = np.zeros(5)
    _load().orc_kk_grad_hess(len(x), _p(x), _p(y), _p(d), l, m, _p(out))
    return out


def kk_run(x, y, d, l=1.0, sweeps=200, tol=0.0):
    """Returns (x, y, energy_per_sweep, skipped, sweeps_done); inputs are not modified."""
    x = np.array(x, np.float64)
    y = np.array(y, np.float64)
    d = _c(d, np.int32)
    e = np.zeros(max(sweeps, 1))
    done = ctypes.c_int64()
    sk = _load().orc_kk_run(len(x), _p(x), _p(y), _p(d), l, sweeps, tol, _p(e), ctypes.byref(done))
    return x, y, e[:done.value].copy(), int(sk), int(done.value)


# ---------------------------------------------------------------- Section 3.2

def fa2_forces(x, y, mass, off, adj, kr=1.0, kg=1.0, targets=None):
    """Returns dict of frep, fatt, fgrav (each [nt, 2]), sabs [nt] (sum of the
    magnitudes of all contributions) and srep [nt] (repulsion terms only)."""
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    mass = _c(mass, np.float64)
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    n = len(x)
    tg = None if targets is None else _c(targets, np.int64)
    nt = n if tg is None else len(tg)
    o = [np.zeros(nt) for _ in range(8)]
    _load().orc_fa2_forces(n, _p(x), _p(y), _p(mass), _p(off), _p(adj), kr, kg, nt, _p(tg),
                           *[_p(a) for a in o])
    return dict(frep=np.stack([o[0], o[1]], 1), fatt=np.stack([o[2], o[3]], 1),
                fgrav=np.stack([o[4], o[5]], 1), sabs=o[6], srep=o[7])


def fa2_energy(x, y, mass, off, adj, kr=1.0, kg=1.0) -> float:
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    mass = _c(mass, np.float64)
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    return float(_load().orc_fa2_energy(len(x), _p(x), _p(y), _p(mass), _p(off), _p(adj), kr, kg))


@dataclass
class FA2State:
    x: np.ndarray
    y: np.ndarray
    fpx: np.ndarray
    fpy: np.ndarray
    sg: float = 1.0


def fa2_run(x, y, mass, off, adj, iters, kr=1.0, kg=1.0, ks=0.1, ksmax=10.0, tau=1.0, variant=0,
            state: FA2State | None = None):
    """Runs `iters` iterations from (x, y) with F_{-1} = 0, s_G = 1 (or from `state`).

    Returns (state, stats[iters, 3] = swg, trc, s_G)."""
    if state is None:
        state = FA2State(np.array(x, np.float64), np.array(y, np.float64), np.zeros(len(x)),
                         np.zeros(len(x)), 1.0)
    mass = _c(mass, np.float64)
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    sg = ctypes.c_double(state.sg)
    stats = np.zeros((max(iters, 1), 3))
    _load().orc_fa2_run(len(state.x), _p(state.x), _p(state.y), _p(mass), _p(off), _p(adj), kr, kg,
                        ks, ksmax, tau, variant, iters, _p(state.fpx), _p(state.fpy), ctypes.byref(sg),
                        _p(stats))
    state.sg = sg.value
    return state, stats[:iters]


# ---------------------------------------------------------------- initial positions

def splitmix64_stream(seed, n):
    out = np.zeros(n, np.uint64)
    _load().orc_splitmix64_stream(seed, n, _p(out))
    return out


def init_positions(seed, ids):
    ids = _c(ids, np.int64)
    x = np.zeros(len(ids))
    y = np.zeros(len(ids))
    _load().orc_init_positions(seed, len(ids), _p(ids), _p(x), _p(y))
    return x, y


# ---------------------------------------------------------------- Section 4: whole layout

def layout(g: Graph, kk_max_nodes=50, fa2_iters=50, kr=1.0, kg=1.0, ks=0.1, ksmax=10.0, tau=1.0,
           variant=0, kk_l=1.0, kk_sweeps=200, kk_tol=0.0, seed=0):
    """Per-component layouts in each component's own frame (Section 4).

    Components with at most kk_max_nodes nodes: Kamada-Kawai from the
    initial positions scaled by l * diam / 2; larger: ForceAtlas2 with exact
    repulsion from the initial positions.  Returns xy [n, 2] (float64)."""
    label, _ = components(g.off, g.adj)
    comp_off, _, nodes = component_order(label)
    deg = np.diff(g.off)
    xy = np.zeros((g.n_nodes, 2))
    for c in range(len(comp_off) - 1):
        vs = nodes[comp_off[c]:comp_off[c + 1]]
        loff, ladj = subgraph(g.off, g.adj, vs)
        x, y = init_positions(seed, vs)
        if len(vs) <= kk_max_nodes:
            d = bfs_apsp(loff, ladj)
            diam = int(d.max()) if len(vs) > 1 else 0
            x *= kk_l * diam / 2.0
            y *= kk_l * diam / 2.0
            x, y, _, _, _ = kk_run(x, y, d, kk_l, kk_sweeps, kk_tol)
        else:
            st, _ = fa2_run(x, y, deg[vs] + 1.0, loff, ladj, fa2_iters, kr, kg, ks, ksmax, tau, variant)
            x, y = st.x, st.y
        xy[vs, 0] = x
        xy[vs, 1] = y
    return xy
