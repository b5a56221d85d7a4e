"""GPU parity of the path the benchmark times (Sections 3.2, 3.2.1, 4).

* Long runs: bgl_layout with the benchmark's parameters (ForceAtlas2, FMM
  repulsion chosen automatically for components of at least 8,192 nodes,
  p = 8, leaf 64, 500 iterations) on three synthetic transaction graphs
  whose giant component is just above that size, against the oracle's exact
  FP64 iteration from the same start.  The iteration is chaotic, so the
  runs are compared by the layout energy E_FA2 (within 1 %) and by the mean,
  median and 90th percentile of the edge lengths (within 2 %).
* FMM forces at the final layout of the 200,000-transaction graph's giant
  component (a clustered, deep tree): normalised errors e_i of 2,000
  sampled nodes against the oracle's exact sum, within the truncation
  ceiling of p = 8 and p = 16.
* Batched components: 20 components of 200-2,000 nodes laid out together
  by one bgl_layout call (one ForceAtlas2 iteration graph for all of them,
  each with its own global speed, the larger ones with FMM repulsion),
  each compared on its own against the oracle after three iterations."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

RHO = math.sqrt(2) / (4 - math.sqrt(2))


def ceiling(p):
    return max(2 * (1 + RHO) * RHO ** (p + 1) / (1 - RHO), 2e-5)


@pytest.fixture(scope="module")
def ctx():
    import paper_2403_03504_gb300 as bgl
    c = bgl.Context(0)
    yield c
    c.close()


def _bgl():
    import paper_2403_03504_gb300 as bgl
    return bgl


def _component(og, nodes, coff, c):
    vs = nodes[coff[c]:coff[c + 1]]
    loff, ladj = oracle.subgraph(og.off, og.adj, vs)
    return vs, loff, ladj, np.diff(loff) + 1.0


def _edge_lengths(x, y, loff, ladj):
    src = np.repeat(np.arange(len(loff) - 1), np.diff(loff))
    keep = src < ladj
    a, b = src[keep], ladj[keep]
    d = np.hypot(x[a] - x[b], y[a] - y[b])
    return np.array([d.mean(), np.percentile(d, 50), np.percentile(d, 90)])


@pytest.mark.parametrize("graph_seed,pos_seed", [(11, 0), (12, 1), (13, 2)])
def test_fmm_layout_long_run_matches_oracle(ctx, graph_seed, pos_seed):
    bgl = _bgl()
    tx = synth.tx_lists(n_tx=3000, seed=graph_seed)
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    p = bgl.params(seed=pos_seed, fa2_iters=500, repulsion=bgl.REP_AUTO, fmm_p=8, leaf_size=64, kk_max_nodes=50,
                   fmm_min_nodes=8192)
    n_kk, n_fa2 = g.split(50)
    assert n_fa2 == 1 and coff[1] - coff[0] >= 8192          # one ForceAtlas2 component, on the FMM path
    xy = g.layout(p).astype(np.float64)
    # AUTO took the FMM: the same layout with the FMM forced is bitwise equal
    p_fmm = bgl.params(seed=pos_seed, fa2_iters=500, repulsion=bgl.REP_FMM, fmm_p=8, leaf_size=64, kk_max_nodes=50)
    assert np.array_equal(xy, g.layout(p_fmm).astype(np.float64))
    vs, loff, ladj, mass = _component(og, nodes, coff, 0)
    x0, y0 = oracle.init_positions(pos_seed, vs)
    st, _ = oracle.fa2_run(x0, y0, mass, loff, ladj, 500)
    eg = oracle.fa2_energy(xy[vs, 0], xy[vs, 1], mass, loff, ladj)
    eo = oracle.fa2_energy(st.x, st.y, mass, loff, ladj)
    assert abs(eg - eo) <= 0.01 * abs(eo), (eg, eo)
    lg = _edge_lengths(xy[vs, 0], xy[vs, 1], loff, ladj)
    lo = _edge_lengths(st.x, st.y, loff, ladj)
    assert np.all(np.abs(lg - lo) <= 0.02 * lo), (lg, lo)
    g.destroy()


def test_fmm_forces_at_the_c2_final_layout(ctx):
    bgl = _bgl()
    tx = synth.tx_lists(**synth.C2)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    p = bgl.params(seed=0, fa2_iters=500, repulsion=bgl.REP_AUTO, fmm_p=8, leaf_size=64, kk_max_nodes=50)
    xy_all = g.layout(p)
    vs = nodes[coff[0]:coff[1]]
    xy = np.ascontiguousarray(xy_all[vs])
    off, adj = g.csr()
    pos = np.full(len(off) - 1, -1, np.int64)
    pos[vs] = np.arange(len(vs))
    loff = np.zeros(len(vs) + 1, np.int64)
    loff[1:] = np.cumsum(np.diff(off)[vs])
    ladj = pos[np.concatenate([adj[off[v]:off[v + 1]] for v in vs])].astype(np.int32)
    mass = np.diff(loff) + 1.0
    sample = np.sort(np.random.default_rng(2).choice(len(vs), 2000, replace=False))
    o = oracle.fa2_forces(xy[:, 0], xy[:, 1], mass, loff, ladj, 1.0, 1.0, targets=sample)
    stats = g.fmm_stats(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=8), xy, reps=1)
    assert stats["depth"] >= 6, stats                     # a clustered layout, not a shallow random cloud
    for pp in (8, 16):
        f = g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=pp, leaf_size=64), xy)
        e = np.hypot(*(f[sample] - o["frep"]).T) / o["srep"]
        assert e.max() <= ceiling(pp), (pp, e.max())
    g.destroy()


def test_batched_fa2_components_each_match_oracle(ctx):
    bgl = _bgl()
    sizes, u, v = synth.forest(23, 20, 200.0, 2000.0)
    n = int(sizes.sum())
    og = oracle.graph_from_edges(n, u, v)
    g = bgl.Graph.from_edges(ctx, n, u, v)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    sz = np.diff(coff)
    assert len(sz) == 20 and sz.min() >= 200
    assert np.sum(sz >= 1000) >= 3 and np.sum(sz < 1000) >= 3   # both repulsion kinds in the batch
    p = bgl.params(seed=3, fa2_iters=3, repulsion=bgl.REP_AUTO, fmm_min_nodes=1000, fmm_p=24, leaf_size=64,
                   kk_max_nodes=50)
    xy = g.layout(p).astype(np.float64)
    for c in range(len(sz)):
        vs, loff, ladj, mass = _component(og, nodes, coff, c)
        x0, y0 = oracle.init_positions(3, vs)
        st, _ = oracle.fa2_run(x0, y0, mass, loff, ladj, 3)
        diag = math.hypot(np.ptp(st.x), np.ptp(st.y))
        err = np.max(np.hypot(xy[vs, 0] - st.x, xy[vs, 1] - st.y))
        assert err <= 1e-3 * diag, (c, len(vs), err, diag)
    g.destroy()


def test_measured_crossover_picks_exact_or_fmm_per_component(ctx):
    """fmm_min_nodes = -1: components below 2,048 nodes take the exact sum,
    those of 131,072 or more the FMM, the ones in between whichever was
    faster when timed; each component equals, bitwise, its layout under the
    kind it was given (components are independent)."""
    bgl = _bgl()
    small, _, _ = synth.forest(41, 3, 300.0, 300.0)
    mid, _, _ = synth.forest(42, 1, 6000.0, 6000.0)
    sizes = [140000, int(mid[0])] + [int(x) for x in small]
    u, v, base = [], [], 0
    for k, n in enumerate(sizes):
        if k == 0:                                    # a long path
            u.append(np.arange(base, base + n - 1))
            v.append(np.arange(base + 1, base + n))
        else:
            s2, uu, vv = synth.forest(41 + k, 1, float(n), float(n))
            assert int(s2[0]) == n
            u.append(uu + base)
            v.append(vv + base)
        base += n
    u = np.concatenate(u).astype(np.int32)
    v = np.concatenate(v).astype(np.int32)
    g = bgl.Graph.from_edges(ctx, base, u, v)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    common = dict(seed=5, fa2_iters=3, kk_max_nodes=50, fmm_p=8, leaf_size=64)
    tuned = g.layout(bgl.params(repulsion=bgl.REP_AUTO, fmm_min_nodes=-1, **common))
    exact = g.layout(bgl.params(repulsion=bgl.REP_EXACT, **common))
    fmm = g.layout(bgl.params(repulsion=bgl.REP_FMM, **common))
    for c in range(len(coff) - 1):
        vs = nodes[coff[c]:coff[c + 1]]
        n = len(vs)
        is_exact = np.array_equal(tuned[vs], exact[vs])
        is_fmm = np.array_equal(tuned[vs], fmm[vs])
        if n < 2048:
            assert is_exact, (c, n)
        elif n >= 131072:
            assert is_fmm, (c, n)
        else:
            assert is_exact or is_fmm, (c, n)
    g.destroy()


def test_fused_iteration_is_bitwise_the_unfused_one(ctx, monkeypatch):
    """A run whose only component is on the FMM iterates fused (swing and
    traction sums and s_G in the combine pass, the next root square in the
    update); the unfused iteration, taken when a run has several components,
    sums in the same order, so a component's layout does not depend on what
    shares its run (sharding and batched serving rely on it)."""
    bgl = _bgl()
    tx = synth.tx_lists(n_tx=3000, seed=11)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    vs = nodes[coff[0]:coff[1]]
    x, y = oracle.init_positions(4, vs)
    xy0 = np.stack([x, y], 1).astype(np.float32)
    for variant in (0, 1):
        p = bgl.params(seed=4, fa2_iters=60, repulsion=bgl.REP_FMM, fmm_p=8, leaf_size=64, kk_max_nodes=50,
                       swing_variant=variant)
        fused = g.layout(p)
        fxy, fstats = g.fa2_step(0, p, 40, xy0)
        monkeypatch.setenv("BGL_FUSED_ITERATION", "0")
        assert np.array_equal(fused, g.layout(p)), variant
        uxy, ustats = g.fa2_step(0, p, 40, xy0)
        assert np.array_equal(fxy, uxy) and np.array_equal(fstats, ustats), variant
        monkeypatch.delenv("BGL_FUSED_ITERATION")
    g.destroy()
