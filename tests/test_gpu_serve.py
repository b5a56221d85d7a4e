"""Serving layouts of k-hop neighbourhoods of a resident graph.

The neighbourhood extraction is compared bit-exact with a plain
breadth-first search; the server's results are compared bitwise with the
same requests served alone and with the direct layout of the extracted
subgraph (every kernel is deterministic and each request's state private to
its worker); admission keeps the estimated in-flight footprint within the
budget, and the estimate bounds the measured device memory of a request."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

EINVAL = -1


def _bgl():
    import paper_2403_03504_gb300 as bgl
    return bgl


@pytest.fixture(scope="module")
def ctx():
    c = _bgl().Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def c1(ctx):
    bgl = _bgl()
    tx = synth.tx_lists(**synth.C1)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    return g, og


def test_khop_matches_breadth_first_search(c1):
    g, og = c1
    rng = np.random.default_rng(4)
    for seed in rng.choice(og.n_nodes, 12, replace=False):
        for k in (0, 1, 2, 3):
            got = g.khop(int(seed), k, 1 << 30)
            ids, edges = oracle.khop(og.off, og.adj, int(seed), k)
            assert got is not None
            assert np.array_equal(got[0], ids), (seed, k)
            pairs = sorted(zip(np.minimum(got[1], got[2]).tolist(), np.maximum(got[1], got[2]).tolist()))
            assert pairs == edges, (seed, k)
    # a cap below the size refuses
    seed = int(np.argmax(np.diff(og.off)))
    assert g.khop(seed, 2, 10) is None


def _requests(og):
    deg = np.diff(og.off)
    hub = int(np.argmax(deg))
    rng = np.random.default_rng(6)
    small = [int(s) for s in rng.choice(np.flatnonzero(deg == 1), 3, replace=False)]
    return [(hub, 1), (hub, 2), (small[0], 3), (small[1], 1), (small[2], 4), (hub, 3)]


def _params():
    bgl = _bgl()
    return bgl.params(fa2_iters=30, fmm_min_nodes=400, kk_max_nodes=50)


def test_results_are_the_same_alone_and_in_the_mix(ctx, c1):
    bgl = _bgl()
    g, og = c1
    reqs = _requests(og)
    p = _params()
    mix = bgl.Server(g, slots=3, hbm_budget=8 << 30)
    ids = [mix.submit(s, k, p) for s, k in reqs]
    got = []
    for rid in ids:
        st, n, t, b = mix.wait(rid)
        assert st == 0
        assert t[0] <= t[1] <= t[2]
        assert b[1] <= b[0], "footprint estimate below the measured peak"
        got.append(mix.fetch(rid, n))
    mix.close()
    alone = bgl.Server(g, slots=1, hbm_budget=8 << 30)
    for (s, k), (gids, gxy) in zip(reqs, got):
        rid = alone.submit(s, k, p)
        st, n, _, _ = alone.wait(rid)
        ids1, xy1 = alone.fetch(rid, n)
        assert np.array_equal(ids1, gids) and np.array_equal(xy1, gxy), (s, k)
    alone.close()
    # the direct layout of the extracted subgraph
    s, k = reqs[1]
    nodes, u, v = g.khop(s, k, 1 << 30)
    sub = bgl.Graph.from_edges(ctx, len(nodes), u, v)
    sub.components(labels=False)
    direct = sub.layout(p)
    assert np.array_equal(direct, got[1][1])
    sub.destroy()


def test_admission_by_footprint(ctx, c1):
    bgl = _bgl()
    g, og = c1
    reqs = _requests(og)
    p = _params()
    srv = bgl.Server(g, slots=3, hbm_budget=1)          # no two requests fit together
    ids = [srv.submit(s, k, p) for s, k in reqs]
    fps = []
    for rid in ids:
        st, n, t, b = srv.wait(rid)
        assert st == 0
        fps.append(int(b[0]))
        srv.fetch(rid, n)
    assert srv.inflight_max() == max(fps)                 # one request at a time
    srv.close()
    # oversize requests fail alone, the others are unaffected
    srv = bgl.Server(g, slots=2, hbm_budget=8 << 30)
    bad = srv.submit(reqs[1][0], 2, p, max_nodes=5)
    ok = srv.submit(reqs[3][0], 1, p)
    assert srv.wait(bad)[0] == EINVAL
    assert srv.wait(ok)[0] == 0
    srv.close()


def _direct(ctx, g, seed, hops, p):
    bgl = _bgl()
    nodes, u, v = g.khop(seed, hops, 1 << 30)
    sub = bgl.Graph.from_edges(ctx, len(nodes), u, v)
    sub.components(labels=False)
    xy = sub.layout(p)
    sub.destroy()
    return nodes, xy


def test_batched_requests_are_bitwise_their_own_layouts(ctx, c1):
    """With batching on and one slot, the requests queued behind the one in
    progress with equal parameters share one layout (the disjoint union of
    their neighbourhoods); each result equals the direct layout of its own
    neighbourhood bit for bit: KK-sized and exact ForceAtlas2 neighbourhoods
    (batched), FMM ones (alone, or batched when KK-sized), two parameter
    sets in runs (only equal neighbours join), an assembled request (alone)
    and an oversize one (fails alone)."""
    bgl = _bgl()
    g, og = c1
    deg = np.diff(og.off)
    rng = np.random.default_rng(8)
    seeds = [int(s) for s in rng.choice(og.n_nodes, 24, replace=False)]
    p_ex = bgl.params(fa2_iters=30, kk_max_nodes=20, repulsion=bgl.REP_EXACT)
    p_fmm = bgl.params(fa2_iters=30, kk_max_nodes=20, repulsion=bgl.REP_FMM, fmm_p=8, leaf_size=16)
    p_asm = bgl.params(fa2_iters=30, kk_max_nodes=20, assemble=1)
    hub = int(np.argmax(deg))
    reqs = [(hub, 3, p_ex)]                          # keeps the worker busy while the rest queue
    for i, s in enumerate(seeds):
        reqs.append((s, 1 + i % 3, p_ex if (i // 5) % 2 == 0 else p_fmm))
    reqs.append((seeds[0], 2, p_asm))
    srv = bgl.Server(g, slots=1, hbm_budget=8 << 30)
    srv.batching(8, 1 << 20)
    ids = [srv.submit(s, k, p) for s, k, p in reqs]
    bad = srv.submit(hub, 3, p_ex, max_nodes=3)
    sizes = []
    for (s, k, p), rid in zip(reqs, ids):
        st, n, t, b = srv.wait(rid)
        assert st == 0, (s, k)
        gids, gxy = srv.fetch(rid, n)
        nodes, xy = _direct(ctx, g, s, k, p)
        assert np.array_equal(gids, nodes) and np.array_equal(gxy, xy), (s, k, n)
        sizes.append(n)
    assert srv.wait(bad)[0] == EINVAL
    batches, batched = srv.batch_stats()
    assert batches >= 2 and batched >= 8, (batches, batched)
    assert max(sizes) > 20 and min(sizes) <= 20          # both KK and ForceAtlas2 requests
    srv.close()
    srv = bgl.Server(g, slots=1)
    with pytest.raises(bgl.BglError):
        srv.batching(0, 10)
    srv.close()
