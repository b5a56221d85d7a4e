"""Python binding of the GB300 layout library (include/bgl.h).

Argument marshalling only: every step of the layout runs in the CUDA kernels
of ``libbgl.so``.  The library must have been built (``build()``, or
``__graft_entry__.build()``); importing this package without it raises.

Host arrays are numpy arrays; device arrays are anything with an integer
device address (a ``torch.Tensor`` on the context's device, or an int).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = ["BglError", "Context", "Graph", "Params", "Server", "params", "build", "lib_path", "launch_count", "FMM_STATS",
           "REP_EXACT", "REP_FMM", "REP_AUTO"]

REP_EXACT, REP_FMM, REP_AUTO = 0, 1, 2

_STATUS = {0: "BGL_OK", -1: "BGL_EINVAL", -2: "BGL_ENOMEM", -3: "BGL_ECUDA", -4: "BGL_ETIMEOUT",
           -5: "BGL_ENUMERIC", -6: "BGL_ESTATE"}


class BglError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of bgl_params (field order and types must match the header)."""
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("kk_max_nodes", ctypes.c_int32),
        ("fa2_iters", ctypes.c_int32),
        ("kr", ctypes.c_double),
        ("kg", ctypes.c_double),
        ("ks", ctypes.c_double),
        ("ksmax", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("repulsion", ctypes.c_int32),
        ("fmm_p", ctypes.c_int32),
        ("leaf_size", ctypes.c_int32),
        ("fmm_min_nodes", ctypes.c_int32),
        ("swing_variant", ctypes.c_int32),
        ("kk_sweeps", ctypes.c_int32),
        ("kk_l", ctypes.c_double),
        ("kk_tol", ctypes.c_double),
        ("assemble", ctypes.c_int32),
        ("m2l_bf16", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib_path() -> str:
    return _build.LIB


def build(force: bool = False) -> str:
    return _build.build(force=force)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libbgl.so is not built ({_build.LIB}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    VP, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    PP = ctypes.POINTER(ctypes.c_void_p)
    P64 = ctypes.POINTER(ctypes.c_int64)
    sigs = {
        "bgl_ctx_create": ([ctypes.c_int, PP], I32),
        "bgl_ctx_destroy": ([VP], None),
        "bgl_ctx_set_stream": ([VP, VP], I32),
        "bgl_ctx_sync": ([VP], I32),
        "bgl_last_error": ([VP], ctypes.c_char_p),
        "bgl_params_default": ([ctypes.POINTER(Params)], None),
        "bgl_graph_build": ([VP, I64, VP, VP, VP, VP, PP], I32),
        "bgl_graph_build_dev": ([VP, I64, I64, I64, VP, VP, VP, VP, PP], I32),
        "bgl_graph_from_edges": ([VP, I64, I64, VP, VP, PP], I32),
        "bgl_graph_sizes": ([VP, P64, P64, P64, P64], I32),
        "bgl_graph_addresses": ([VP, VP], I32),
        "bgl_graph_edges": ([VP, VP, VP], I32),
        "bgl_graph_csr": ([VP, VP, VP], I32),
        "bgl_degrees": ([VP, VP], I32),
        "bgl_graph_destroy": ([VP], I32),
        "bgl_components": ([VP, VP, P64], I32),
        "bgl_component_nodes": ([VP, VP, VP, VP], I32),
        "bgl_split": ([VP, I32, P64, P64], I32),
        "bgl_layout": ([VP, ctypes.POINTER(Params), VP], I32),
        "bgl_layout_dev": ([VP, ctypes.POINTER(Params), VP], I32),
        "bgl_kk_distances": ([VP, I64, VP], I32),
        "bgl_kk_run": ([VP, I64, ctypes.POINTER(Params), VP], I32),
        "bgl_fa2_forces": ([VP, I64, ctypes.POINTER(Params), VP, VP], I32),
        "bgl_fa2_repulsion": ([VP, I64, ctypes.POINTER(Params), VP, VP], I32),
        "bgl_fa2_step": ([VP, I64, ctypes.POINTER(Params), I32, VP, VP], I32),
        "bgl_fa2_session_begin": ([VP, I64, ctypes.POINTER(Params), VP], I32),
        "bgl_fa2_session_advance": ([VP, I32, VP], I32),
        "bgl_fa2_session_positions": ([VP, VP, P64], I32),
        "bgl_state_save": ([VP, VP, ctypes.POINTER(ctypes.c_size_t)], I32),
        "bgl_assemble": ([VP, ctypes.POINTER(Params), VP, VP, VP, VP, VP, VP, VP], I32),
        "bgl_graph_khop": ([VP, I64, I32, I64, P64, VP, P64, VP, VP], I32),
        "bgl_server_create": ([VP, I32, I64, PP], I32),
        "bgl_server_submit": ([VP, I64, I32, I64, ctypes.POINTER(Params), P64], I32),
        "bgl_server_wait": ([VP, I64, P64, VP, VP], I32),
        "bgl_server_fetch": ([VP, I64, VP, VP], I32),
        "bgl_server_stats": ([VP, P64], I32),
        "bgl_server_batching": ([VP, I32, I64], I32),
        "bgl_server_batch_stats": ([VP, P64, P64], I32),
        "bgl_server_destroy": ([VP], I32),
        "bgl_state_load": ([VP, VP, ctypes.c_size_t], I32),
        "bgl_fmm_stats": ([VP, I64, ctypes.POINTER(Params), VP, I32, VP], I32),
        "bgl_launch_count": ([], I64),
        "bgl_fa2_iteration_noalloc": ([VP, I64, VP, VP, VP, VP, VP, VP, VP, ctypes.POINTER(Params)], I32),
        "bgl_debug_fail_alloc": ([VP, I64], I32),
        "bgl_peak_probe": ([VP, VP], I32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


FMM_STATS = ("boxes", "leaves", "depth", "p2p_pairs", "m2l", "m2p", "p2l", "ms_points", "ms_tree", "ms_lists",
             "ms_up", "ms_down", "ms_near", "ms_far", "ms_total", "sortmode_rel_diff", "sort_skip", "w_heavy")


class Server:
    """Continuous-batching layout server on a resident graph (bgl_server_*)."""

    def __init__(self, graph: "Graph", slots: int = 4, hbm_budget: int = 64 << 30):
        self._lib = _load()
        self.graph = graph
        h = ctypes.c_void_p()
        graph.ctx.check(self._lib.bgl_server_create(graph.h, slots, hbm_budget, ctypes.byref(h)))
        self.h = h

    def submit(self, seed: int, hops: int, p: "Params", max_nodes: int = 1 << 30) -> int:
        rid = ctypes.c_int64()
        st = self._lib.bgl_server_submit(self.h, seed, hops, max_nodes, ctypes.byref(p), ctypes.byref(rid))
        if st != 0:
            raise BglError(st, "bgl_server_submit")
        return rid.value

    def wait(self, rid: int):
        """Blocks; returns (status, n_nodes, times[3], bytes[2])."""
        n = ctypes.c_int64()
        t = np.zeros(3)
        b = np.zeros(2, np.int64)
        st = self._lib.bgl_server_wait(self.h, rid, ctypes.byref(n), _hp(t), _hp(b))
        return st, n.value, t, b

    def fetch(self, rid: int, n: int):
        ids = np.zeros(max(n, 1), np.int32)
        xy = np.zeros((max(n, 1), 2), np.float32)
        st = self._lib.bgl_server_fetch(self.h, rid, _hp(ids), _hp(xy))
        if st != 0:
            raise BglError(st, "bgl_server_fetch")
        return ids[:n], xy[:n]

    def inflight_max(self) -> int:
        v = ctypes.c_int64()
        self._lib.bgl_server_stats(self.h, ctypes.byref(v))
        return v.value

    def batching(self, max_requests: int, max_nodes: int):
        """Queued requests with equal parameters share one layout, up to
        max_requests of them and max_nodes nodes in all (1: off)."""
        st = self._lib.bgl_server_batching(self.h, max_requests, max_nodes)
        if st != 0:
            raise BglError(st, "bgl_server_batching")

    def batch_stats(self):
        """(layouts that served several requests, requests they served)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._lib.bgl_server_batch_stats(self.h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def close(self):
        if self.h:
            self._lib.bgl_server_destroy(self.h)
            self.h = None


def launch_count() -> int:
    """Kernels launched through the library by this process so far."""
    return int(_load().bgl_launch_count())


def params(**kw) -> Params:
    """bgl_params with the library defaults, overridden by keyword."""
    p = Params()
    _load().bgl_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _hp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dp(x):
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Context:
    """A bgl_ctx: one CUDA device, a stream and a device memory pool."""

    def __init__(self, device: int = 0):
        self._lib = _load()
        h = ctypes.c_void_p()
        st = self._lib.bgl_ctx_create(device, ctypes.byref(h))
        if st != 0:
            raise BglError(st, f"bgl_ctx_create({device}) failed")
        self.h = h
        self.device = device

    def check(self, st: int):
        if st != 0:
            raise BglError(st, self._lib.bgl_last_error(self.h).decode())

    def set_stream(self, stream=None):
        """Use a CUDA stream (torch.cuda.Stream, raw handle int, or None for the context's own)."""
        if stream is None:
            ptr = None
        elif isinstance(stream, int):
            ptr = ctypes.c_void_p(stream)
        else:
            ptr = ctypes.c_void_p(stream.cuda_stream)
        self.check(self._lib.bgl_ctx_set_stream(self.h, ptr))

    def sync(self):
        self.check(self._lib.bgl_ctx_sync(self.h))

    def fa2_iteration_noalloc(self, n, d_off, d_adj, d_mass, d_xy, d_fprev, d_f, d_sg, p: Params):
        """One exact-repulsion ForceAtlas2 iteration on device arrays without
        allocating (bgl_fa2_iteration_noalloc); arguments are device tensors or
        addresses, queued on the context's stream."""
        self.check(self._lib.bgl_fa2_iteration_noalloc(self.h, n, _dp(d_off), _dp(d_adj), _dp(d_mass), _dp(d_xy),
                                                       _dp(d_fprev), _dp(d_f), _dp(d_sg), ctypes.byref(p)))

    def peak_probe(self) -> dict:
        """Measured FP32 lanes, MUFU reciprocals and repulsion pairs per SM
        clock (bgl_peak_probe), and the SM count."""
        out = np.zeros(5)
        self.check(self._lib.bgl_peak_probe(self.h, _hp(out)))
        return {"fp32_lanes_per_clk_sm": out[0], "mufu_rcp_per_clk_sm": out[1], "pairs_per_clk_sm": out[2],
                "packed_pairs_per_clk_sm": out[4], "sms": int(out[3])}

    def debug_fail_alloc(self, after: int):
        """Test aid: the device allocation after `after` more successful ones
        fails with BGL_ENOMEM (-1: never)."""
        self.check(self._lib.bgl_debug_fail_alloc(self.h, after))

    def close(self):
        if self.h:
            self._lib.bgl_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Graph:
    """A device-resident graph (bgl_graph)."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle
        self._lib = ctx._lib

    # ---------------------------------------------------------- construction
    @classmethod
    def build(cls, ctx: Context, in_off, in_addr, out_off, out_addr) -> "Graph":
        in_off = _arr(in_off, np.int64)
        out_off = _arr(out_off, np.int64)
        in_addr = _arr(in_addr, np.uint64)
        out_addr = _arr(out_addr, np.uint64)
        h = ctypes.c_void_p()
        ctx.check(ctx._lib.bgl_graph_build(ctx.h, len(in_off) - 1, _hp(in_off), _hp(in_addr), _hp(out_off),
                                           _hp(out_addr), ctypes.byref(h)))
        return cls(ctx, h)

    @classmethod
    def build_dev(cls, ctx: Context, n_tx, n_in, n_out, d_in_off, d_in_addr, d_out_off, d_out_addr) -> "Graph":
        h = ctypes.c_void_p()
        ctx.check(ctx._lib.bgl_graph_build_dev(ctx.h, n_tx, n_in, n_out, _dp(d_in_off), _dp(d_in_addr),
                                               _dp(d_out_off), _dp(d_out_addr), ctypes.byref(h)))
        return cls(ctx, h)

    @classmethod
    def from_edges(cls, ctx: Context, n, u, v) -> "Graph":
        u = _arr(u, np.int32)
        v = _arr(v, np.int32)
        h = ctypes.c_void_p()
        ctx.check(ctx._lib.bgl_graph_from_edges(ctx.h, n, len(u), _hp(u), _hp(v), ctypes.byref(h)))
        return cls(ctx, h)

    def destroy(self):
        if self.h:
            st = self._lib.bgl_graph_destroy(self.h)
            self.h = None
            self.ctx.check(st)

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                self._lib.bgl_graph_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # ---------------------------------------------------------- queries
    def sizes(self):
        n, a, d, u = (ctypes.c_int64() for _ in range(4))
        self.ctx.check(self._lib.bgl_graph_sizes(self.h, ctypes.byref(n), ctypes.byref(a), ctypes.byref(d),
                                                 ctypes.byref(u)))
        return dict(n_nodes=n.value, n_addr=a.value, n_dir_edges=d.value, n_undir_edges=u.value)

    def addresses(self):
        s = self.sizes()
        out = np.zeros(s["n_addr"], np.uint64)
        self.ctx.check(self._lib.bgl_graph_addresses(self.h, _hp(out)))
        return out

    def edges(self):
        s = self.sizes()
        src = np.zeros(s["n_dir_edges"], np.int32)
        dst = np.zeros(s["n_dir_edges"], np.int32)
        self.ctx.check(self._lib.bgl_graph_edges(self.h, _hp(src), _hp(dst)))
        return src, dst

    def csr(self):
        s = self.sizes()
        off = np.zeros(s["n_nodes"] + 1, np.int64)
        adj = np.zeros(2 * s["n_undir_edges"], np.int32)
        self.ctx.check(self._lib.bgl_graph_csr(self.h, _hp(off), _hp(adj)))
        return off, adj

    def degrees(self):
        out = np.zeros(self.sizes()["n_nodes"], np.int32)
        self.ctx.check(self._lib.bgl_degrees(self.h, _hp(out)))
        return out

    # ---------------------------------------------------------- Section 4
    def components(self, labels: bool = True):
        nc = ctypes.c_int64()
        lab = np.zeros(self.sizes()["n_nodes"], np.int32) if labels else None
        self.ctx.check(self._lib.bgl_components(self.h, _hp(lab) if labels else None, ctypes.byref(nc)))
        self.n_comp = nc.value
        return (lab, nc.value) if labels else nc.value

    def component_nodes(self):
        nc = self.n_comp
        off = np.zeros(nc + 1, np.int64)
        lab = np.zeros(nc, np.int32)
        nodes = np.zeros(self.sizes()["n_nodes"], np.int32)
        self.ctx.check(self._lib.bgl_component_nodes(self.h, _hp(off), _hp(lab), _hp(nodes)))
        return off, lab, nodes

    def split(self, kk_max_nodes: int):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self.ctx.check(self._lib.bgl_split(self.h, kk_max_nodes, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def layout(self, p: Params | None = None, out: np.ndarray | None = None):
        """Coordinates [n_nodes, 2] (float32) in node-id order; `out` may be a
        preallocated (e.g. pinned) float32 array of that shape."""
        p = p or params()
        if out is None:
            out = np.zeros((self.sizes()["n_nodes"], 2), np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == 2 * self.sizes()["n_nodes"]
        self.ctx.check(self._lib.bgl_layout(self.h, ctypes.byref(p), _hp(out)))
        return out

    def layout_dev(self, p: Params, d_xy_out):
        self.ctx.check(self._lib.bgl_layout_dev(self.h, ctypes.byref(p), _dp(d_xy_out)))

    # ---------------------------------------------------------- per component
    def kk_distances(self, c: int, n_c: int):
        d = np.zeros((n_c, n_c), np.int32)
        self.ctx.check(self._lib.bgl_kk_distances(self.h, c, _hp(d)))
        return d

    def kk_run(self, c: int, p: Params, xy):
        xy = np.array(xy, np.float32, order="C")
        self.ctx.check(self._lib.bgl_kk_run(self.h, c, ctypes.byref(p), _hp(xy)))
        return xy

    def fa2_forces(self, c: int, p: Params, xy):
        xy = _arr(xy, np.float32)
        f = np.zeros_like(xy)
        self.ctx.check(self._lib.bgl_fa2_forces(self.h, c, ctypes.byref(p), _hp(xy), _hp(f)))
        return f

    def fa2_repulsion(self, c: int, p: Params, xy):
        xy = _arr(xy, np.float32)
        f = np.zeros_like(xy)
        self.ctx.check(self._lib.bgl_fa2_repulsion(self.h, c, ctypes.byref(p), _hp(xy), _hp(f)))
        return f

    def fmm_stats(self, c: int, p: Params, xy, reps: int = 3) -> dict:
        xy = _arr(xy, np.float32)
        out = np.zeros(len(FMM_STATS))
        self.ctx.check(self._lib.bgl_fmm_stats(self.h, c, ctypes.byref(p), _hp(xy), reps, _hp(out)))
        return dict(zip(FMM_STATS, out.tolist()))

    def fa2_step(self, c: int, p: Params, iters: int, xy):
        xy = np.array(xy, np.float32, order="C")
        stats = np.zeros((max(iters, 1), 3))
        self.ctx.check(self._lib.bgl_fa2_step(self.h, c, ctypes.byref(p), iters, _hp(xy), _hp(stats)))
        return xy, stats[:iters]

    def assemble(self, p: Params, xy):
        """Assembly of per-component layouts (node-id order) into one frame
        (Section 4); returns (xy, info) with per-component rank, parent (by
        rank), scale, radius and level-0 centres (by rank)."""
        xy = _arr(xy, np.float32)
        nc = self.n_comp
        out = np.zeros_like(xy)
        rank = np.zeros(nc, np.int64)
        parent = np.zeros(nc, np.int64)
        scale = np.zeros(nc, np.float32)
        radius = np.zeros(nc, np.float32)
        centre = np.zeros((nc, 2), np.float32)
        self.ctx.check(self._lib.bgl_assemble(self.h, ctypes.byref(p), _hp(xy), _hp(out), _hp(rank), _hp(parent),
                                              _hp(scale), _hp(radius), _hp(centre)))
        return out, dict(rank=rank, parent=parent, scale=scale, radius=radius, centre=centre)

    def khop(self, seed: int, hops: int, max_nodes: int):
        """k-hop neighbourhood: (resident node ids, u, v) or None if larger than max_nodes."""
        n, m = ctypes.c_int64(), ctypes.c_int64()
        self.ctx.check(self._lib.bgl_graph_khop(self.h, seed, hops, max_nodes, ctypes.byref(n), None,
                                                ctypes.byref(m), None, None))
        if n.value < 0:
            return None
        ids = np.zeros(n.value, np.int32)
        u = np.zeros(max(m.value, 1), np.int32)
        v = np.zeros(max(m.value, 1), np.int32)
        self.ctx.check(self._lib.bgl_graph_khop(self.h, seed, hops, max_nodes, ctypes.byref(n), _hp(ids),
                                                ctypes.byref(m), _hp(u), _hp(v)))
        return ids, u[:m.value], v[:m.value]

    # resumable ForceAtlas2 run and its checkpoint
    def session_begin(self, c: int, p: Params, xy) -> None:
        xy = _arr(xy, np.float32)
        self._session_n = len(xy)
        self.ctx.check(self._lib.bgl_fa2_session_begin(self.h, c, ctypes.byref(p), _hp(xy)))

    def session_advance(self, iters: int):
        stats = np.zeros((max(iters, 1), 3))
        self.ctx.check(self._lib.bgl_fa2_session_advance(self.h, iters, _hp(stats)))
        return stats[:iters]

    def session_positions(self, n: int):
        xy = np.zeros((n, 2), np.float32)
        done = ctypes.c_int64(0)
        self.ctx.check(self._lib.bgl_fa2_session_positions(self.h, _hp(xy), ctypes.byref(done)))
        return xy, int(done.value)

    def state_save(self) -> bytes:
        need = ctypes.c_size_t(0)
        self.ctx.check(self._lib.bgl_state_save(self.h, None, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        self.ctx.check(self._lib.bgl_state_save(self.h, buf, ctypes.byref(need)))
        return buf.raw[:need.value]

    def state_load(self, data: bytes) -> None:
        buf = ctypes.create_string_buffer(data, len(data))
        self.ctx.check(self._lib.bgl_state_load(self.h, buf, len(data)))
