"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and by the oracle.

Holds no arithmetic of the layout method: it only draws transaction lists,
forests of small components and random point sets.  The C generator
(``gen.c``) is compiled in place with gcc on first use.

Workloads (stand-ins for the paper's daily bitcoin graphs, Section 2 and
Section 4 / Figs. 4-5):

* ``C1``: 1,000 transactions, seed 1 (about 2.5k addresses).
* ``C2``: 200,000 transactions, seed 2 (about 4.8e5 addresses).
* ``C4``: 3,000,000 transactions, seed 4 (about 7e6 addresses).
* ``C3``: forest of 100,000 components, sizes log-uniform in [3, 200],
  seed 3, plus 2,000 components log-uniform in [200, 5000], seed 33.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

C1 = dict(seed=1, n_tx=1000)
C2 = dict(seed=2, n_tx=200_000)
C4 = dict(seed=4, n_tx=3_000_000)
C3_SMALL = dict(seed=3, n_comp=100_000, lo=3.0, hi=200.0)
C3_MID = dict(seed=33, n_comp=2_000, lo=200.0, hi=5000.0)


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so next to it (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.synth_tx_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64, i64p, i64p]
            lib.synth_tx_sizes.restype = None
            lib.synth_tx_generate.argtypes = [ctypes.c_uint64, ctypes.c_int64] + [ctypes.c_void_p] * 4
            lib.synth_tx_generate.restype = ctypes.c_int64
            lib.synth_forest_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_void_p, i64p, i64p]
            lib.synth_forest_sizes.restype = None
            lib.synth_forest_edges.argtypes = [ctypes.c_uint64, ctypes.c_int64] + [ctypes.c_void_p] * 3
            lib.synth_forest_edges.restype = None
            lib.synth_splitmix64_stream.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            lib.synth_splitmix64_stream.restype = None
            lib.synth_zipf_sample.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
            lib.synth_zipf_sample.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class TxLists:
    """Per-transaction input and output address lists in CSR form."""

    def __init__(self, in_off, in_addr, out_off, out_addr, n_addr_created):
        self.in_off = in_off
        self.in_addr = in_addr
        self.out_off = out_off
        self.out_addr = out_addr
        self.n_addr_created = n_addr_created

    @property
    def n_tx(self) -> int:
        return len(self.in_off) - 1

    @property
    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.in_off, self.in_addr, self.out_off, self.out_addr))


def tx_lists(seed: int, n_tx: int) -> TxLists:
    """Transaction lists of the recipe in gen.c (inputs, outputs, preferential reuse)."""
    lib = _load()
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    lib.synth_tx_sizes(seed, n_tx, ctypes.byref(a), ctypes.byref(b))
    in_off = np.zeros(n_tx + 1, np.int64)
    out_off = np.zeros(n_tx + 1, np.int64)
    in_addr = np.zeros(a.value, np.uint64)
    out_addr = np.zeros(b.value, np.uint64)
    n_addr = lib.synth_tx_generate(seed, n_tx, _p(in_off), _p(in_addr), _p(out_off), _p(out_addr))
    return TxLists(in_off, in_addr, out_off, out_addr, int(n_addr))


def forest(seed: int, n_comp: int, lo: float, hi: float):
    """Forest of random recursive trees with ~10% extra edges.

    Returns (sizes[int64 n_comp], u[int32 m], v[int32 m]); node ids are
    consecutive per component."""
    lib = _load()
    sizes = np.zeros(n_comp, np.int64)
    nn = ctypes.c_int64()
    ne = ctypes.c_int64()
    lib.synth_forest_sizes(seed, n_comp, lo, hi, _p(sizes), ctypes.byref(nn), ctypes.byref(ne))
    u = np.zeros(ne.value, np.int32)
    v = np.zeros(ne.value, np.int32)
    lib.synth_forest_edges(seed, n_comp, _p(sizes), _p(u), _p(v))
    return sizes, u, v


def forest_of_sizes(seed: int, sizes):
    """The recipe of `forest` (random recursive trees, round(0.1 (n - 1))
    extra edges each where they fit) with the given component sizes.

    Returns (sizes[int64], u[int32 m], v[int32 m])."""
    lib = _load()
    sizes = np.ascontiguousarray(sizes, np.int64)
    ne = 0
    for n in sizes.tolist():
        extra = int(math.floor(0.1 * (n - 1) + 0.5))
        ne += (n - 1) + min(extra, n * (n - 1) // 2 - (n - 1))
    u = np.zeros(ne, np.int32)
    v = np.zeros(ne, np.int32)
    lib.synth_forest_edges(seed, len(sizes), _p(sizes), _p(u), _p(v))
    return sizes, u, v


def points(seed: int, n: int, kind: str = "uniform", scale: float = 1.0):
    """Random 2-D point sets (float32) for force tests.

    kind = "uniform": uniform in [-scale, scale)^2.
    kind = "clustered": a mixture of Gaussian clusters with widely varying
    widths and weights (mimics converged force layouts: dense hubs, sparse
    periphery)."""
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        xy = rng.uniform(-scale, scale, size=(n, 2))
    elif kind == "clustered":
        k = max(1, n // 500)
        centres = rng.uniform(-scale, scale, size=(k, 2))
        widths = scale * 10.0 ** rng.uniform(-3.5, -0.5, size=k)
        w = rng.pareto(1.2, size=k) + 1e-3
        lab = rng.choice(k, size=n, p=w / w.sum())
        xy = centres[lab] + rng.normal(size=(n, 2)) * widths[lab, None]
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(xy.astype(np.float32))


def splitmix64_stream(seed: int, n: int) -> np.ndarray:
    """The generator's SplitMix64: first n outputs from state `seed` (test hook)."""
    out = np.zeros(n, np.uint64)
    _load().synth_splitmix64_stream(seed, n, _p(out))
    return out


def zipf_sample(seed: int, N: int, n: int) -> np.ndarray:
    """n draws of the generator's Zipf(1.2) sampler on {1..N} (test hook)."""
    out = np.zeros(n, np.int64)
    _load().synth_zipf_sample(seed, N, n, _p(out))
    return out
