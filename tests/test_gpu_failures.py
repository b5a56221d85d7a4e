"""Failure paths of the C ABI, made to fire without faulting the GPU.

* BGL_ENUMERIC: a non-finite input position spreads through the forces;
  the update kernel's finiteness check reports it (exact and FMM
  repulsion), and the context keeps working.
* BGL_ENOMEM: the context's allocator is told (bgl_debug_fail_alloc, a host
  hook) to refuse a device allocation partway through a graph build or a
  layout; the call returns BGL_ENOMEM, leaves its host output untouched, and
  the next call on the same context gives the same layout as before.
* BGL_ETIMEOUT: with BGL_TEST_SORT_STALL=1 in the environment when an FMM
  plan is made, the first tile of each radix pass withholds its counts and
  the bounded waits on it give up after 4,096 polls (no wait is endless and
  every write stays inside the arrays); the evaluation's later kernels
  return at once, the call reports BGL_ETIMEOUT, and the next call without
  the switch gives the same result as a fresh context."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2403_03504_gb300 as bgl
    c = bgl.Context(0)
    yield c
    c.close()


def _c1(ctx):
    import paper_2403_03504_gb300 as bgl
    tx = synth.tx_lists(**synth.C1)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    return tx, g


@pytest.mark.parametrize("rep", ["exact", "fmm"])
def test_non_finite_position_reports_enumeric(ctx, rep):
    import paper_2403_03504_gb300 as bgl
    _, g = _c1(ctx)
    coff, _, nodes = g.component_nodes()
    vs = nodes[coff[0]:coff[1]]
    x, y = oracle.init_positions(0, vs)
    xy = np.stack([x, y], 1).astype(np.float32)
    p = bgl.params(repulsion=bgl.REP_EXACT if rep == "exact" else bgl.REP_FMM, fmm_p=8, leaf_size=32)
    bad = xy.copy()
    bad[7, 1] = np.inf
    with pytest.raises(bgl.BglError) as e:
        g.fa2_step(0, p, 2, bad)
    assert e.value.status == -5
    out, _ = g.fa2_step(0, p, 2, xy)                 # the context and the graph still work
    assert np.all(np.isfinite(out))
    g.destroy()


def test_refused_allocation_reports_enomem_and_leaves_outputs(ctx):
    import paper_2403_03504_gb300 as bgl
    tx, g = _c1(ctx)
    p = bgl.params(seed=1, fa2_iters=5, kk_sweeps=20, repulsion=bgl.REP_AUTO)
    want = g.layout(p)
    refused = 0
    for after in (0, 1, 2, 4, 8):
        out = np.full_like(want, 7.5)
        ctx.debug_fail_alloc(after)
        try:
            g.layout(p, out=out)
        except bgl.BglError as e:
            assert e.status == -2, (after, e)
            assert np.all(out == 7.5), after          # nothing written on failure
            refused += 1
        else:
            assert np.array_equal(out, want)
        ctx.debug_fail_alloc(-1)
        assert np.array_equal(g.layout(p), want), after   # the same context recovers
    assert refused >= 3
    # a graph build that cannot allocate returns no graph, and the next one works
    ctx.debug_fail_alloc(1)
    with pytest.raises(bgl.BglError) as e:
        bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    assert e.value.status == -2
    ctx.debug_fail_alloc(-1)
    g2 = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g2.components(labels=False)
    assert np.array_equal(g2.layout(p), want)
    g2.destroy()
    g.destroy()


def test_bounded_sort_wait_reports_etimeout(ctx, monkeypatch):
    import paper_2403_03504_gb300 as bgl
    n = 30000                                         # several radix tiles of 4,096 keys
    g = bgl.Graph.from_edges(ctx, n, np.arange(n - 1), np.arange(1, n))
    g.components(labels=False)
    x, y = oracle.init_positions(3, np.arange(n))
    xy = np.stack([x, y], 1).astype(np.float32)
    p = bgl.params(repulsion=bgl.REP_FMM, fmm_p=8, leaf_size=16)
    want, wstats = g.fa2_step(0, p, 3, xy)
    monkeypatch.setenv("BGL_TEST_SORT_STALL", "1")
    with pytest.raises(bgl.BglError) as e:
        g.fa2_repulsion(0, p, xy)
    assert e.value.status == -4
    with pytest.raises(bgl.BglError) as e:
        g.fa2_step(0, p, 3, xy)
    assert e.value.status == -4
    monkeypatch.delenv("BGL_TEST_SORT_STALL")
    got, stats = g.fa2_step(0, p, 3, xy)             # the context and the graph still work
    assert np.array_equal(got, want) and np.array_equal(stats, wstats)
    g.destroy()
