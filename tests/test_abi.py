"""CPU checks of the C ABI: the library builds, loads, exports every declared
entry point, and the Python mirror of bgl_params matches the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2403_03504_gb300 as bgl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bgl.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bgl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    bgl.build()
    return ctypes.CDLL(bgl.lib_path())


def test_header_declares_entry_points():
    names = _declared()
    for must in ("bgl_graph_build", "bgl_components", "bgl_split", "bgl_layout", "bgl_fa2_step",
                 "bgl_kk_run", "bgl_graph_build_dev", "bgl_layout_dev", "bgl_state_save", "bgl_state_load",
                 "bgl_fa2_session_begin", "bgl_fa2_session_advance", "bgl_fa2_session_positions"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", bgl.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(bgl_[a-z0-9_]+)\b", out))
    assert set(_declared()) <= exported


def test_params_layout_matches_header(tmp_path):
    fields = [f for f, _ in bgl.Params._fields_]
    prog = tmp_path / "p.c"
    body = "\n".join(f'printf("%zu ", offsetof(bgl_params, {f}));' for f in fields)
    prog.write_text(f"""
#include <stddef.h>
#include <stdio.h>
#include "bgl.h"
int main(void) {{ {body} printf("%zu\\n", sizeof(bgl_params)); return 0; }}
""")
    exe = tmp_path / "p"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [getattr(bgl.Params, f).offset for f in fields] + [ctypes.sizeof(bgl.Params)]
    assert got == want


def test_params_defaults(lib):
    p = bgl.params()
    assert p.kk_max_nodes == 50 and p.fa2_iters == 50 and p.fmm_p == 8 and p.leaf_size == 64
    assert p.kr == 1.0 and p.kg == 1.0 and p.ks == 0.1 and p.ksmax == 10.0 and p.tau == 1.0
    assert p.kk_sweeps == 200 and p.kk_l == 1.0 and p.repulsion == bgl.REP_AUTO


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # entry points that validate before touching the device
    assert lib.bgl_ctx_create(0, None) == -1
    assert lib.bgl_state_save(None, None, None) == -1
    assert lib.bgl_state_load(None, None, 0) == -1
    assert lib.bgl_fa2_session_advance(None, 1, None) == -1
    lib.bgl_graph_sizes.argtypes = [ctypes.c_void_p] * 5
    assert lib.bgl_graph_sizes(None, None, None, None, None) == -1
    lib.bgl_last_error.restype = ctypes.c_char_p
    lib.bgl_last_error.argtypes = [ctypes.c_void_p]
    assert lib.bgl_last_error(None) == b"context is NULL"


def test_every_entry_point_cites_its_passage():
    """Each declaration of bgl.h is documented by a comment -- its own, or the
    note of its group since the last section divider -- that names the
    paper's section it implements, or says that the paper has no
    counterpart (library plumbing and measurement aids)."""
    src = open(HEADER).read()
    comments = [(m.start(), m.end(), m.group(0)) for m in re.finditer(r"/\*.*?\*/", src, flags=re.S)]
    missing = []
    for m in re.finditer(r"\n(?:bgl_status|void|int64_t|const char \*)\s*(bgl_[a-z0-9_]+)\s*\(", src):
        group = []
        for c in reversed([c for c in comments if c[1] <= m.start()]):
            group.append(c[2])
            if c[2].startswith("/* ----"):
                break
        if not any(re.search(r"Section|counterpart", c) for c in group):
            missing.append(m.group(1))
    assert not missing, missing
