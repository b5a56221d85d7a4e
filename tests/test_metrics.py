"""Per-iteration JSON-lines metrics of a ForceAtlas2 run
(paper_2403_03504_gb300.metrics).

CPU: the chunking, numbering, fields and timing split, against a stand-in
session whose per-iteration statistics are known.  GPU: a logged run gives
bitwise the positions and the (swing, traction, s_G) of every iteration of
one bgl_fa2_step call, also when it is split by a checkpoint and resumed in
a rebuilt graph."""
import io
import json

import numpy as np
import pytest

import synth
from paper_2403_03504_gb300 import metrics


class _FakeGraph:
    """Session stand-in: iteration k has swing k, traction 2k, s_G 1/k."""

    def __init__(self, n):
        self.n, self.done, self.calls = n, 0, []

    def component_nodes(self):
        # a 3-node component 0 before the session's component 1
        return np.array([0, 3, 3 + self.n], np.int64), None, None

    def session_begin(self, c, p, xy):
        assert len(xy) == self.n
        self.done = 0

    def session_advance(self, iters):
        self.calls.append(iters)
        k = np.arange(self.done + 1, self.done + iters + 1, dtype=np.float64)
        self.done += iters
        return np.stack([k, 2 * k, 1 / k], 1)

    def session_positions(self, n):
        return np.full((n, 2), float(self.done), np.float32), self.done


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.5
        return self.t


def test_lines_chunks_and_numbering():
    g = _FakeGraph(7)
    buf = io.StringIO()
    xy = metrics.run_logged(g, 0, None, 23, np.zeros((7, 2)), buf, chunk=10, clock=_Clock())
    recs = [json.loads(s) for s in buf.getvalue().splitlines()]
    assert g.calls == [10, 10, 3]
    assert [r["iter"] for r in recs] == list(range(1, 24))
    for r in recs:
        k = r["iter"]
        assert (r["swing"], r["traction"], r["s_G"]) == (k, 2 * k, 1 / k)
        assert r["component"] == 0 and r["n"] == 7
    # each chunk's 0.5 s split evenly among its iterations
    assert [r["ms"] for r in recs] == [50.0] * 20 + [500.0 / 3] * 3
    assert [r["chunk"] for r in recs] == [10] * 20 + [3] * 3
    assert np.all(xy == 23)


def test_resume_numbers_on_and_zero_iterations(tmp_path):
    g = _FakeGraph(4)
    path = str(tmp_path / "m.jsonl")
    metrics.run_logged(g, 1, None, 5, np.zeros((4, 2)), path, chunk=1)
    assert g.calls == [1] * 5
    xy = metrics.run_logged(g, 1, None, 4, None, str(tmp_path / "m2.jsonl"), chunk=3, resume=True)
    assert xy.shape == (4, 2)                      # n of component 1, from the component offsets
    assert [r["iter"] for r in metrics.read(path)] == [1, 2, 3, 4, 5]
    recs = metrics.read(str(tmp_path / "m2.jsonl"))
    assert [r["iter"] for r in recs] == [6, 7, 8, 9] and all(r["n"] == 4 and r["component"] == 1 for r in recs)
    assert metrics.run_logged(g, 1, None, 0, np.zeros((4, 2)), None).shape == (4, 2)
    with pytest.raises(ValueError):
        metrics.run_logged(g, 1, None, 3, np.zeros((4, 2)), None, chunk=0)
    with pytest.raises(ValueError):
        metrics.run_logged(g, 1, None, -1, np.zeros((4, 2)), None)
    with pytest.raises(ValueError):
        metrics.run_logged(g, 1, None, 3, None, None)


@pytest.mark.gpu
@pytest.mark.parametrize("rep", ["exact", "fmm"])
def test_logged_run_is_bitwise_one_step_call(tmp_path, rep):
    import paper_2403_03504_gb300 as bgl

    ctx = bgl.Context(0)
    tx = synth.tx_lists(**synth.C1)

    def graph():
        g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
        g.components(labels=False)
        return g

    g = graph()
    coff, _, _ = g.component_nodes()
    n = int(coff[1] - coff[0])
    xy0 = np.random.default_rng(3).uniform(-2, 2, (n, 2)).astype(np.float32)
    p = bgl.params(repulsion=bgl.REP_EXACT if rep == "exact" else bgl.REP_FMM, fmm_p=8, leaf_size=32)
    want, wstats = g.fa2_step(0, p, 30, xy0)
    path = str(tmp_path / "run.jsonl")
    got = metrics.run_logged(g, 0, p, 12, xy0, path, chunk=5)
    blob = g.state_save()
    g.destroy()
    g2 = graph()                                  # resumed in a rebuilt graph
    g2.state_load(blob)
    path2 = str(tmp_path / "run2.jsonl")
    got = metrics.run_logged(g2, 0, p, 18, None, path2, chunk=7, resume=True)
    recs = metrics.read(path) + metrics.read(path2)
    assert [r["iter"] for r in recs] == list(range(1, 31))
    assert np.array_equal(got, want)
    assert np.array_equal(np.array([[r["swing"], r["traction"], r["s_G"]] for r in recs]), wstats)
    assert all(r["ms"] > 0 and r["n"] == n for r in recs)
    g2.destroy()
    ctx.close()
