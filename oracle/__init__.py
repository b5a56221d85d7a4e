"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package; the layout library never does.  It wraps
``oracle.c`` (compiled here with gcc, OpenMP, no fast-math, no FMA
contraction) with numpy-facing functions, and composes them into the whole
layout of Section 4 (``layout``) in plain Python.

Paper map: Section 2 -> graph_build / undirected_csr; Section 4 ->
components / component_order / layout, and the assembly of the component
layouts into one frame -> assemble (meta_keys, meta_tree, tree_distances,
kkw_*); Section 3.1 -> bfs_apsp, floyd_warshall, kk_*; Section 3.2 ->
fa2_forces, fa2_energy, fa2_run.
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
                "orc_kk_step": ([_VP, _D, _VP, _VP], ctypes.c_int),
                "orc_fa2_forces": ([_I64, _VP, _VP, _VP, _VP, _VP, _D, _D, _I64, _VP] + [_VP] * 8, None),
                "orc_fa2_energy": ([_I64, _VP, _VP, _VP, _VP, _VP, _D, _D], _D),
                "orc_fa2_run": ([_I64, _VP, _VP, _VP, _VP, _VP, _D, _D, _D, _D, _D, ctypes.c_int32,
                                 _I64, _VP, _VP, _VP, _VP], None),
                "orc_threads": ([], ctypes.c_int),
                "orc_kkw_energy": ([_I64, _VP, _VP, _VP], _D),
                "orc_kkw_grad_hess": ([_I64, _VP, _VP, _VP, _I64, _VP], None),
                "orc_kkw_run": ([_I64, _VP, _VP, _VP, _D, _I64, _VP], _I64),
                "orc_tree_distances": ([_I64, _VP, _VP, _VP], None),
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


def kk_step(g, H, l):
    """The safeguarded 2x2 Newton step of one node (Section 3.1): g the
    half-gradient (2,), H the half-Hessian (2, 2), l the step-length cap.
    Returns (step (2,), moved)."""
    o = np.array([g[0], g[1], H[0][0], H[0][1], H[1][1]], np.float64)
    dx, dy = ctypes.c_double(0.0), ctypes.c_double(0.0)
    moved = _load().orc_kk_step(_p(o), float(l), ctypes.byref(dx), ctypes.byref(dy))
    return np.array([dx.value, dy.value]), bool(moved)


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


# ---------------------------------------------------------------- Section 4: assembly

KAPPA = 1.0                       # the "constant" added to every meta-edge length
META_SALT = 0x5851F42D4C957F2D    # separates the order stream from the position streams


def kkw_energy(x, y, d) -> float:
    return float(_load().orc_kkw_energy(len(x), _p(_c(x, np.float64)), _p(_c(y, np.float64)), _p(_c(d, np.float64))))


def kkw_grad_hess(x, y, d, m):
    out = np.zeros(5)
    _load().orc_kkw_grad_hess(len(x), _p(_c(x, np.float64)), _p(_c(y, np.float64)), _p(_c(d, np.float64)), m,
                              _p(out))
    return out


def kkw_run(x, y, d, cap, sweeps):
    """Returns (x, y, energy_per_sweep); inputs are not modified."""
    x = np.array(x, np.float64)
    y = np.array(y, np.float64)
    e = np.zeros(max(sweeps, 1))
    _load().orc_kkw_run(len(x), _p(x), _p(y), _p(_c(d, np.float64)), cap, sweeps, _p(e))
    return x, y, e[:sweeps].copy()


def tree_distances(parent, length):
    parent = _c(parent, np.int64)
    m = len(parent)
    d = np.zeros((m, m))
    _load().orc_tree_distances(m, _p(parent), _p(_c(length, np.float64)), _p(d))
    return d


def meta_keys(seed, n):
    """Random order of the components (Section 4): key of component c is the
    first SplitMix64 output from state (seed ^ META_SALT) ^ (c * 0x9E3779B97F4A7C15)."""
    keys = np.zeros(n, np.uint64)
    base = (int(seed) ^ META_SALT) & 0xFFFFFFFFFFFFFFFF
    for c in range(n):
        st = base ^ ((c * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF)
        keys[c] = splitmix64_stream(st, 1)[0]
    return keys


def meta_tree(sizes):
    """Each item after the first is linked to the largest earlier item (the
    first of equals); returns parent indices (-1 for item 0)."""
    parent = np.full(len(sizes), -1, np.int64)
    best = 0
    for k in range(1, len(sizes)):
        parent[k] = best
        if sizes[k] > sizes[best]:
            best = k
    return parent


def assemble(off, adj, comp_off, nodes, xy, K, seed=0, sweeps=200, kappa=KAPPA):
    """Assembly of per-component layouts into one frame (Section 4).

    1. Rescale: each component is centred on its centroid and scaled so that
       its mean edge length is 1 (no edges: scale 1); its radius is the
       largest distance of a node from the centroid after scaling.
    2. Order: components sorted by meta_keys (random order).
    3. Levels: the ordered items are cut into consecutive chunks of at most
       K; in a chunk each item links to the largest earlier one (size =
       nodes), with edge length r_a + r_b + kappa (half the diameters plus a
       constant); Kamada-Kawai on the chunk's weighted tree (path lengths as
       distances, init SplitMix64 by item index with seed + level + 1,
       scaled by half the largest distance, steps capped at the mean edge
       length) gives item centres; the chunk is centred on their mean and
       becomes one item of the next level with radius max(|centre| + r) and
       size the sum.  Repeat until one item is left.
    4. Compose: a node's position is its scaled local position plus the
       offset of every item containing it.
    Returns dict(xy, rank, parent0, scale, centroid, radius, levels) where
    levels[L] = dict(parent, length, centres, offsets, radius, size)."""
    C = len(comp_off) - 1
    xy = np.asarray(xy, np.float64)
    scale = np.ones(C)
    centroid = np.zeros((C, 2))
    radius = np.zeros(C)
    sizes = np.diff(comp_off).astype(np.int64)
    local = np.zeros_like(xy)
    for c in range(C):
        vs = nodes[comp_off[c]:comp_off[c + 1]]
        p = xy[vs]
        tot, cnt = 0.0, 0
        for v in vs:
            for w in adj[off[v]:off[v + 1]]:
                if w > v:
                    tot += float(np.hypot(*(xy[v] - xy[w])))
                    cnt += 1
        if cnt > 0 and tot > 0.0:
            scale[c] = cnt / tot
        centroid[c] = p.mean(0)
        q = (p - centroid[c]) * scale[c]
        local[vs] = q
        radius[c] = float(np.max(np.hypot(q[:, 0], q[:, 1]))) if len(vs) > 0 else 0.0
    order = np.lexsort((np.arange(C), meta_keys(seed, C)))   # by key, then index
    rank = np.empty(C, np.int64)
    rank[order] = np.arange(C)
    item_r = radius[order].copy()
    item_n = sizes[order].copy()
    levels = []
    parent0 = None
    level = 0
    while len(item_r) > 1 or level == 0:
        m_all = len(item_r)
        parent = np.full(m_all, -1, np.int64)
        length = np.zeros(m_all)
        offsets = np.zeros((m_all, 2))
        centres = np.zeros((m_all, 2))
        nxt_r, nxt_n = [], []
        for a in range(0, m_all, K):
            b = min(m_all, a + K)
            m = b - a
            par = meta_tree(item_n[a:b])
            ln = np.zeros(m)
            for k in range(1, m):
                ln[k] = item_r[a + k] + item_r[a + par[k]] + kappa
            parent[a:b] = np.where(par >= 0, par + a, -1)
            length[a:b] = ln
            if m == 1:
                q = np.zeros((1, 2))
            else:
                d = tree_distances(par, ln)
                x, y = init_positions(seed + level + 1, np.arange(a, b))
                half = d.max() / 2.0
                cap = ln[1:].mean()
                x, y, _ = kkw_run(x * half, y * half, d, cap, sweeps)
                q = np.stack([x, y], 1)
            centres[a:b] = q
            ctr = q.mean(0)
            offsets[a:b] = q - ctr
            nxt_r.append(float(np.max(np.hypot(*(q - ctr).T) + item_r[a:b])))
            nxt_n.append(int(item_n[a:b].sum()))
        levels.append(dict(parent=parent, length=length, centres=centres, offsets=offsets,
                           radius=item_r.copy(), size=item_n.copy()))
        if level == 0:
            parent0 = parent
        item_r = np.array(nxt_r)
        item_n = np.array(nxt_n, np.int64)
        level += 1
        if len(item_r) == 1:
            break
    out = local.copy()
    for c in range(C):
        vs = nodes[comp_off[c]:comp_off[c + 1]]
        idx = rank[c]
        shift = np.zeros(2)
        for L in range(len(levels)):
            shift += levels[L]["offsets"][idx]
            idx //= K
        out[vs] += shift
    return dict(xy=out, rank=rank, parent0=parent0, scale=scale, centroid=centroid, radius=radius, levels=levels)


# ---------------------------------------------------------------- neighbourhoods (serving requests)

def khop(off, adj, seed, k):
    """Nodes within k undirected hops of seed (ascending ids) and the edges
    among them in local ids (u < v, each once), by a plain breadth-first
    search; for small graphs."""
    dist = {int(seed): 0}
    frontier = [int(seed)]
    for h in range(k):
        nxt = []
        for x in frontier:
            for w in adj[off[x]:off[x + 1]]:
                w = int(w)
                if w not in dist:
                    dist[w] = h + 1
                    nxt.append(w)
        frontier = nxt
    ids = np.array(sorted(dist), np.int64)
    local = {int(g): i for i, g in enumerate(ids)}
    edges = set()
    for g in ids:
        for w in adj[off[g]:off[g + 1]]:
            w = int(w)
            if w in local and local[w] != local[int(g)]:
                a, b = sorted((local[int(g)], local[w]))
                edges.add((a, b))
    return ids, sorted(edges)
