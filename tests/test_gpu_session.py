"""Resumable ForceAtlas2 runs and their checkpoints (the state entry points
of the C ABI).  The iteration of Section 3.2 carries F_{t-1} and the global
speed s_G from one iteration to the next, so a run split into pieces, or
saved and reloaded into a graph rebuilt from the same transactions, must
continue exactly as one uninterrupted run: every comparison here is bitwise."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

EINVAL, ESTATE = -1, -6


def _bgl():
    import paper_2403_03504_gb300 as bgl
    return bgl


@pytest.fixture(scope="module")
def ctx():
    c = _bgl().Context(0)
    yield c
    c.close()


def _graph(ctx, cfg):
    bgl = _bgl()
    tx = synth.tx_lists(**cfg)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    return g


def _start(g, c=0):
    coff, _, _ = g.component_nodes()
    n = int(coff[c + 1] - coff[c])
    return np.random.default_rng(9).uniform(-3, 3, (n, 2)).astype(np.float32)


@pytest.mark.parametrize("rep", ["exact", "fmm"])
def test_session_pieces_equal_one_run(ctx, rep):
    bgl = _bgl()
    g = _graph(ctx, synth.C1)
    p = bgl.params(repulsion=bgl.REP_EXACT if rep == "exact" else bgl.REP_FMM, fmm_p=8, leaf_size=16)
    xy0 = _start(g)
    want, wstats = g.fa2_step(0, p, 20, xy0)
    g.session_begin(0, p, xy0)
    s1 = g.session_advance(7)
    s2 = g.session_advance(13)
    got, done = g.session_positions(len(xy0))
    assert done == 20
    assert np.array_equal(got, want)
    assert np.array_equal(np.concatenate([s1, s2]), wstats)
    g.destroy()


@pytest.mark.parametrize("rep", ["exact", "fmm"])
def test_checkpoint_resumes_bitwise_in_a_rebuilt_graph(ctx, rep):
    bgl = _bgl()
    p = bgl.params(repulsion=bgl.REP_EXACT if rep == "exact" else bgl.REP_FMM, fmm_p=8, leaf_size=16)
    g = _graph(ctx, synth.C1)
    xy0 = _start(g)
    want, _ = g.fa2_step(0, p, 25, xy0)
    g.session_begin(0, p, xy0)
    g.session_advance(12)
    blob = g.state_save()
    g.destroy()
    h = _graph(ctx, synth.C1)                       # same transactions, new graph
    h.state_load(blob)
    mid, done = h.session_positions(len(xy0))
    assert done == 12
    h.session_advance(13)
    got, done = h.session_positions(len(xy0))
    assert done == 25
    assert np.array_equal(got, want)
    # saving again after the load reproduces the checkpoint format and size
    assert len(h.state_save()) == len(blob)
    h.destroy()


def test_checkpoint_errors(ctx):
    bgl = _bgl()
    p = bgl.params(repulsion=bgl.REP_EXACT)
    g = _graph(ctx, synth.C1)
    with pytest.raises(bgl.BglError) as e:
        g.session_advance(1)
    assert e.value.status == ESTATE
    with pytest.raises(bgl.BglError) as e:
        g.state_save()
    assert e.value.status == ESTATE
    xy0 = _start(g)
    g.session_begin(0, p, xy0)
    g.session_advance(3)
    blob = g.state_save()
    before, _ = g.session_positions(len(xy0))
    # truncated, foreign format, another graph: refused, and the session is kept
    for bad in (blob[:40], blob[:-8], b"NOTSTATE" + blob[8:]):
        with pytest.raises(bgl.BglError) as e:
            g.state_load(bad)
        assert e.value.status == EINVAL
    other = _graph(ctx, dict(synth.C1, seed=synth.C1["seed"] + 100))
    with pytest.raises(bgl.BglError) as e:
        other.state_load(blob)
    assert e.value.status == EINVAL
    after, done = g.session_positions(len(xy0))
    assert done == 3 and np.array_equal(before, after)
    # recomputing the components ends the session
    g.components(labels=False)
    with pytest.raises(bgl.BglError) as e:
        g.session_advance(1)
    assert e.value.status == ESTATE
    other.destroy()
    g.destroy()
