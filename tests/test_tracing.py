"""NVTX ranges of the library, seen through an NVTX injection library
(tests/nvtx_recorder.c) that records every push and pop.

Each check runs in a child process started with NVTX_INJECTION64_PATH set,
because NVTX binds its callbacks at the first NVTX call of a process.
On CPU: a C-ABI call (bgl_ctx_create, which fails without a GPU) is one
balanced range named after the entry point.  On the GPU: layouts of the
1,000-transaction graph with the FMM and with the exact sum show the ranges
of every phase (graph build, components, size split, Kamada-Kawai, the
ForceAtlas2 iterations and their force, swing/traction and update steps),
nested inside the call that ran them and balanced."""
import os
import shutil
import subprocess
import sys

import pytest

import paper_2403_03504_gb300 as bgl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))

DUMP = r"""
import ctypes
def dump(rec):
    rec.nvtx_recorder_dump.restype = ctypes.c_size_t
    rec.nvtx_recorder_dump.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    buf = ctypes.create_string_buffer(1 << 20)
    rec.nvtx_recorder_dump(buf, 1 << 20)
    print("@@RECORD@@")
    print(buf.value.decode(), end="")
"""

CTX_ONLY = DUMP + r"""
import sys
rec = ctypes.CDLL(sys.argv[2])
lib = ctypes.CDLL(sys.argv[1])
h = ctypes.c_void_p()
st = lib.bgl_ctx_create(0, ctypes.byref(h))
if st == 0:
    lib.bgl_ctx_destroy(h)
dump(rec)
"""

LAYOUT = DUMP + r"""
import sys
sys.path.insert(0, sys.argv[3])
rec = ctypes.CDLL(sys.argv[2])
import synth
import paper_2403_03504_gb300 as bgl
tx = synth.tx_lists(**synth.C1)
ctx = bgl.Context(0)
g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
g.components(labels=False)
g.layout(bgl.params(fa2_iters=3, repulsion=bgl.REP_FMM, fmm_p=8, leaf_size=64, kk_max_nodes=50))
g.layout(bgl.params(fa2_iters=3, repulsion=bgl.REP_EXACT, kk_max_nodes=50))
g.destroy()
ctx.close()
dump(rec)
"""


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


@pytest.fixture(scope="module")
def recorder(tmp_path_factory):
    inc = _cuda_include()
    if not os.path.exists(os.path.join(inc, "nvtx3", "nvToolsExt.h")):
        pytest.skip("NVTX headers not found")
    out = str(tmp_path_factory.mktemp("nvtx") / "libnvtx_recorder.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-I", inc, "-o", out,
                           os.path.join(HERE, "nvtx_recorder.c"), "-lpthread"])
    return out


def _run(script, recorder):
    bgl.build()
    env = dict(os.environ, NVTX_INJECTION64_PATH=recorder)
    r = subprocess.run([sys.executable, "-c", script, bgl.lib_path(), recorder, ROOT], capture_output=True,
                       text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    rec = r.stdout.split("@@RECORD@@\n", 1)[1]
    return [line for line in rec.split("\n") if line]


def _tree(events):
    """(name, depth) of every push; asserts that pushes and pops balance."""
    depth, out = 0, []
    for e in events:
        if e == "-":
            depth -= 1
            assert depth >= 0, "pop without a push"
        else:
            assert e.startswith("+")
            out.append((e[1:], depth))
            depth += 1
    assert depth == 0, "unbalanced ranges"
    return out


def test_abi_call_is_one_named_range(recorder):
    ev = _run(CTX_ONLY, recorder)
    assert _tree(ev)[:1] == [("bgl_ctx_create", 0)]


@pytest.mark.gpu
def test_layout_phases_are_nested_ranges(recorder):
    tree = _tree(_run(LAYOUT, recorder))
    names = [n for n, _ in tree]
    top = [n for n, d in tree if d == 0]
    for call in ("bgl_ctx_create", "bgl_graph_build", "bgl_components", "bgl_layout"):
        assert call in top, (call, top)
    for phase in ("graph build (Section 2)", "components (Section 4)", "size split (Section 4)",
                  "ForceAtlas2 iterations (Section 3.2)", "ForceAtlas2: attraction and gravity (Section 3.2)",
                  "ForceAtlas2: repulsion by the FMM (Section 3.2.1)", "ForceAtlas2: exact repulsion (Section 3.2)",
                  "ForceAtlas2: swing and traction (Section 3.2)", "ForceAtlas2: node update (Section 3.2)"):
        assert phase in names, phase
    assert any(n.startswith("Kamada-Kawai: size classes") for n in names)
    assert any(n.startswith("Kamada-Kawai: Newton sweeps") for n in names)
    assert any(n.startswith("ForceAtlas2 iteration:") for n in names)
    # the phases sit inside the calls that ran them
    depth = dict(tree)
    assert depth["graph build (Section 2)"] >= 1
    assert depth["ForceAtlas2: repulsion by the FMM (Section 3.2.1)"] > \
        depth["ForceAtlas2 iteration: forces, swing/traction, update (Section 3.2)"] > \
        depth["ForceAtlas2 iterations (Section 3.2)"] >= 1
