"""GPU parity of the assembly of component layouts into one frame (Section 4):
density rescale, random order, largest-previous meta-tree, weighted
Kamada-Kawai in runs of at most kk_max_nodes, composition.  Integer results
(order, tree) are compared bit-exact with the oracle; the rescale to 1e-5;
the weighted Kamada-Kawai, chaotic like the unweighted one, one sweep from
the same start (1e-3 of the run's largest distance) and by converged energy."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _bgl():
    import paper_2403_03504_gb300 as bgl
    return bgl


@pytest.fixture(scope="module")
def ctx():
    c = _bgl().Context(0)
    yield c
    c.close()


class Forest:
    def __init__(self, ctx, seed, n_comp, lo, hi):
        bgl = _bgl()
        sizes, u, v = synth.forest(seed, n_comp, lo, hi)
        self.n = int(sizes.sum())
        self.g = bgl.Graph.from_edges(ctx, self.n, u, v)
        self.g.components(labels=False)
        self.og = oracle.graph_from_edges(self.n, u, v)
        label, _ = oracle.components(self.og.off, self.og.adj)
        self.comp_off, _, self.nodes = oracle.component_order(label)
        self.xy = np.random.default_rng(seed).normal(0, 5, (self.n, 2)).astype(np.float32)


@pytest.fixture(scope="module")
def forest(ctx):
    return Forest(ctx, 31, 40, 1.0, 25.0)


def test_order_tree_and_rescale_match_oracle(forest):
    bgl = _bgl()
    p = bgl.params(kk_max_nodes=8, kk_sweeps=1, seed=3)
    out, info = forest.g.assemble(p, forest.xy)
    ref = oracle.assemble(forest.og.off, forest.og.adj, forest.comp_off, forest.nodes, forest.xy.astype(np.float64),
                          K=8, seed=3, sweeps=1)
    assert np.array_equal(info["rank"], ref["rank"])
    assert np.array_equal(info["parent"], ref["parent0"])
    assert np.allclose(info["scale"], ref["scale"], rtol=1e-5)
    assert np.allclose(info["radius"], ref["radius"], rtol=1e-5, atol=1e-6)
    # one Kamada-Kawai sweep of every run from the same start
    ctr = ref["levels"][0]["centres"]
    for a in range(0, len(ctr), 8):
        b = min(len(ctr), a + 8)
        span = max(1.0, float(np.max(np.hypot(*(ctr[a:b] - ctr[a]).T))))
        err = float(np.max(np.hypot(*(info["centre"][a:b] - ctr[a:b]).T)))
        assert err <= 1e-3 * span, (a, err, span)
    # every component is its rescaled layout, translated
    for c in range(len(forest.comp_off) - 1):
        vs = forest.nodes[forest.comp_off[c]:forest.comp_off[c + 1]]
        d_in = (forest.xy[vs] - forest.xy[vs[0]]).astype(np.float64) * ref["scale"][c]
        d_out = (out[vs] - out[vs[0]]).astype(np.float64)
        tol = 1e-5 * max(1.0, float(np.max(np.abs(d_in))))
        assert np.max(np.abs(d_out - d_in)) <= tol, c


def test_converged_runs_reach_oracle_energy(forest):
    bgl = _bgl()
    p = bgl.params(kk_max_nodes=8, kk_sweeps=200, seed=3)
    _, info = forest.g.assemble(p, forest.xy)
    ref = oracle.assemble(forest.og.off, forest.og.adj, forest.comp_off, forest.nodes, forest.xy.astype(np.float64),
                          K=8, seed=3, sweeps=200)
    lv = ref["levels"][0]
    for a in range(0, len(lv["centres"]), 8):
        b = min(len(lv["centres"]), a + 8)
        if b - a < 2:
            continue
        par = lv["parent"][a:b] - a
        par[0] = -1
        d = oracle.tree_distances(par, lv["length"][a:b])
        eo = oracle.kkw_energy(lv["centres"][a:b, 0], lv["centres"][a:b, 1], d)
        c = info["centre"][a:b].astype(np.float64)
        eg = oracle.kkw_energy(c[:, 0], c[:, 1], d)
        assert eg <= 1.02 * eo + 1e-6, (a, eg, eo)


def test_two_components_sit_at_the_meta_edge_length(ctx):
    bgl = _bgl()
    u = np.array([0, 1, 3, 4, 5]); v = np.array([1, 2, 4, 5, 3])
    g = bgl.Graph.from_edges(ctx, 6, u, v)
    g.components(labels=False)
    xy = np.random.default_rng(2).normal(0, 1, (6, 2)).astype(np.float32)
    out, info = g.assemble(bgl.params(kk_sweeps=200), xy)
    coff, _, nodes = g.component_nodes()
    cen = [out[nodes[coff[c]:coff[c + 1]]].mean(0) for c in range(2)]
    want = float(info["radius"][0] + info["radius"][1] + oracle.KAPPA)
    assert abs(float(np.hypot(*(cen[0] - cen[1]))) - want) <= 1e-4 * want
    g.destroy()


def test_layout_with_assembly_is_layout_then_assemble(ctx):
    bgl = _bgl()
    tx = synth.tx_lists(**synth.C1)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    p = bgl.params(fa2_iters=20)
    local = g.layout(p)
    p.assemble = 1
    whole = g.layout(p)
    again, _ = g.assemble(p, local)
    assert np.all(np.isfinite(whole))
    assert np.array_equal(whole, again)
    g.destroy()
