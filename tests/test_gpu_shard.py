"""Components sharded across ranks (Section 4), on the CUDA path.

The ranks' shares are laid out one after another on this GPU (each share
graph keeps every node id and only its components' edges) and merged on the
host; the result must be bitwise the one-rank layout of the whole graph,
for the 1,000-transaction graph (ForceAtlas2 giant + Kamada-Kawai
components) and for a forest with several ForceAtlas2 components."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["c1", "forest"])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_layout_is_bitwise_the_one_rank_layout(which, world):
    import paper_2403_03504_gb300 as bgl
    from paper_2403_03504_gb300 import shard
    ctx = bgl.Context(0)
    if which == "c1":
        tx = synth.tx_lists(**synth.C1)
        g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    else:
        sizes, u, v = synth.forest(29, 400, 3.0, 600.0)
        g = bgl.Graph.from_edges(ctx, int(sizes.sum()), u, v)
    g.components(labels=False)
    p = bgl.params(seed=1, fa2_iters=20, kk_sweeps=30, kk_max_nodes=50, repulsion=bgl.REP_AUTO, fmm_min_nodes=400)
    want = g.layout(p)
    n = g.sizes()["n_nodes"]
    src, dst = g.edges()
    comp_off, _, nodes = g.component_nodes()
    costs = shard.component_costs(np.diff(comp_off), p.kk_max_nodes, p.fa2_iters, p.kk_sweeps, p.repulsion,
                                  p.fmm_min_nodes)

    def layout_fn(nn, s, d):
        gs = bgl.Graph.from_edges(ctx, nn, s, d)
        gs.components(labels=False)
        xy = gs.layout(p)
        gs.destroy()
        return xy

    pieces = []
    for r in range(world):
        _, piece, owner = shard.layout_sharded(n, src, dst, comp_off, nodes, costs, r, world, layout_fn)
        pieces.append(piece)
    assert len(set(owner.tolist())) == world
    merged = shard.merge(n, pieces)
    assert np.array_equal(merged, want)
    g.destroy()
    ctx.close()
