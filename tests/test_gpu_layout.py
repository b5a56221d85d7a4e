"""GPU parity of the layout kernels against the FP64 oracle.

Kamada-Kawai (Section 3.1): BFS distances bit-exact; ten sweeps of Newton
steps within 1e-3 of the component diameter; ten sweeps from the oracle's
minimum stay there; 200 sweeps from random starts end stationary and at the
oracle's energy.  A component may differ only where the oracle itself,
started from one-ulp moves of the same FP32 start, ends that far away too
(tests/kk_sensitivity.py).  ForceAtlas2 (Section 3.2): forces within 1e-5 of
the sum of contribution magnitudes (FP32 direct sum), positions within 1e-3
of the bounding-box diagonal after 10 iterations, and long runs compared by
layout energy and edge-length statistics (the iteration is chaotic)."""
import json
import math
import os

import numpy as np
import pytest

import kk_sensitivity
import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    import paper_2403_03504_gb300 as bgl
    c = bgl.Context(0)
    yield c
    c.close()


def _bgl():
    import paper_2403_03504_gb300 as bgl
    return bgl


class Built:
    """A graph on both sides plus per-component local data."""

    def __init__(self, ctx, og, g):
        self.og = og
        self.g = g
        self.lab, _ = g.components()
        self.coff, _, self.nodes = g.component_nodes()

    def comp(self, c):
        vs = self.nodes[self.coff[c]:self.coff[c + 1]]
        loff, ladj = oracle.subgraph(self.og.off, self.og.adj, vs)
        return vs, loff, ladj, np.diff(loff) + 1.0


@pytest.fixture(scope="module")
def c1(ctx):
    bgl = _bgl()
    tx = synth.tx_lists(**synth.C1)
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    return Built(ctx, og, g)


@pytest.fixture(scope="module")
def forest(ctx):
    bgl = _bgl()
    sizes, u, v = synth.forest(17, 300, 3.0, 200.0)
    n = int(sizes.sum())
    og = oracle.graph_from_edges(n, u, v)
    g = bgl.Graph.from_edges(ctx, n, u, v)
    return Built(ctx, og, g)


# ------------------------------------------------------------------ KK

def test_kk_distances_bit_exact(c1, forest):
    for b in (c1, forest):
        sizes = np.diff(b.coff)
        for c in range(len(sizes)):
            if sizes[c] > 255:
                continue
            vs, loff, ladj, _ = b.comp(c)
            d = b.g.kk_distances(c, len(vs))
            assert np.array_equal(d, oracle.bfs_apsp(loff, ladj)), c


def _kk_start(seed, vs, d, l=1.0):
    x, y = oracle.init_positions(seed, vs)
    sc = l * d.max() / 2 if len(vs) > 1 else 0.0
    return x * sc, y * sc


def _kk_components(b, lo=2, hi=255, step=1):
    sizes = np.diff(b.coff)
    return np.flatnonzero((sizes >= lo) & (sizes <= hi))[::step]


def test_kk_ten_sweeps_match_oracle(c1, forest):
    """Ten Gauss-Seidel sweeps from the same FP32 start: positions within
    1e-3 of the diameter for every component, unless the oracle itself,
    started from one-ulp moves of that start, ends farther than 1e-4 of the
    diameter from its unperturbed run (the early sweeps from random starts
    amplify rounding a thousandfold there), or the oracle's trajectory meets
    a Hessian whose small curvature is below 1e-4 of the large one (a path
    straightening: FP32 cannot resolve that curvature, and the energy is
    flat along it), where the KK energies must still agree."""
    bgl = _bgl()
    p = bgl.params(kk_sweeps=10)
    checked, excused = 0, []
    for b in (c1, forest):
        for c in _kk_components(b, step=2):
            checked += 1
            if _kk_ten_sweeps_excused(b, int(c), p):
                excused.append(int(c))
    assert checked > 200 and len(excused) < checked // 2, (checked, excused)


def _kk_ten_sweeps_excused(b, c, p):
    """Ten sweeps of component c from the seeded start against the oracle's:
    False when within 1e-3 of the diameter; True when the oracle's own
    sensitivity excuses the difference (asserting what the excuse needs)."""
    vs, loff, ladj, _ = b.comp(c)
    d = oracle.bfs_apsp(loff, ladj)
    x, y = _kk_start(5, vs, d)
    xy = np.stack([x, y], 1).astype(np.float32)
    got = b.g.kk_run(c, p, xy)
    ox, oy, _, _, _ = oracle.kk_run(xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64), d, 1.0, 10)
    assert np.all(np.isfinite(got)), c
    diam = max(1, int(d.max()))
    err = np.max(np.hypot(got[:, 0] - ox, got[:, 1] - oy)) / diam
    if err <= 1e-3:
        return False
    _, spread, _ = kk_sensitivity.oracle_spread(xy[:, 0], xy[:, 1], d, 10)
    if spread / diam <= 1e-4:
        flat, rx, ry = kk_sensitivity.min_curvature_ratio(xy[:, 0], xy[:, 1], d, 10)
        assert np.array_equal(rx, ox) and np.array_equal(ry, oy)
        eg = oracle.kk_energy(got[:, 0].astype(np.float64), got[:, 1].astype(np.float64), d, 1.0)
        eo = oracle.kk_energy(ox, oy, d, 1.0)
        assert flat < 1e-4 and kk_sensitivity.energy_close(eg, eo), (c, len(vs), err, spread / diam, flat, eg, eo)
    return True


# every edge of the KK size classes (lanes x nodes per lane: 4 x 1 up to 4
# nodes, 4 x 2 up to 8, 4 x 4 up to 16, 8 x 4 up to 32, 16 x 4 up to 64,
# 16 x 8 up to 128, 16 x 16 up to 255), the default KK split (50 / 51) and
# the largest component the byte distances take
KK_EDGE_SIZES = [1, 2, 3, 4, 5, 8, 9, 16, 17, 32, 33, 50, 51, 64, 65, 128, 129, 200, 254, 255]


@pytest.fixture(scope="module")
def kk_edges(ctx):
    """Forests of the KK_EDGE_SIZES plus a 255-node path, whose diameter 254
    is the largest distance a byte holds beside the unreachable mark."""
    bgl = _bgl()
    sizes, u, v = synth.forest_of_sizes(23, KK_EDGE_SIZES)
    n0 = int(sizes.sum())
    pu = np.arange(n0, n0 + 254, dtype=np.int32)
    u, v = np.concatenate([u, pu]), np.concatenate([v, pu + 1])
    n = n0 + 255
    og = oracle.graph_from_edges(n, u, v)
    g = bgl.Graph.from_edges(ctx, n, u, v)
    return Built(ctx, og, g)


def test_kk_size_class_edges(kk_edges):
    """At every size-class edge: distances bit-exact (the path's 254
    included), ten sweeps against the oracle as above, and a 200-sweep run
    that ends finite and stationary."""
    bgl = _bgl()
    sizes = np.diff(kk_edges.coff)
    assert sorted(sizes.tolist()) == sorted(KK_EDGE_SIZES + [255])
    p10, p200 = bgl.params(kk_sweeps=10), bgl.params(kk_sweeps=200)
    excused = []
    for c in range(len(sizes)):
        vs, loff, ladj, _ = kk_edges.comp(c)
        d = oracle.bfs_apsp(loff, ladj)
        assert np.array_equal(kk_edges.g.kk_distances(c, len(vs)), d), (c, len(vs))
        if _kk_ten_sweeps_excused(kk_edges, c, p10):
            excused.append(len(vs))
        x, y = _kk_start(5, vs, d)
        got = kk_edges.g.kk_run(c, p200, np.stack([x, y], 1).astype(np.float32)).astype(np.float64)
        assert np.all(np.isfinite(got)), (c, len(vs))
        e = oracle.kk_energy(got[:, 0], got[:, 1], d, 1.0)
        gmax = max(np.hypot(*oracle.kk_grad_hess(got[:, 0], got[:, 1], d, 1.0, m)[:2]) for m in range(len(vs)))
        assert gmax <= 1e-3 * max(1.0, e), (c, len(vs), gmax)
    assert max(sizes) == 255 and len(excused) <= len(sizes) // 2, excused


def test_kk_stays_at_the_oracle_minimum(forest):
    """From the oracle's converged layout, ten GPU sweeps stay within 1e-3 of the diameter."""
    bgl = _bgl()
    p = bgl.params(kk_sweeps=10)
    for c in _kk_components(forest, lo=3, hi=120, step=5):
        vs, loff, ladj, _ = forest.comp(c)
        d = oracle.bfs_apsp(loff, ladj)
        x, y = _kk_start(5, vs, d)
        ox, oy, _, _, _ = oracle.kk_run(x, y, d, 1.0, 200)
        xy = np.stack([ox, oy], 1).astype(np.float32)
        got = forest.g.kk_run(int(c), p, xy)
        err = np.max(np.hypot(got[:, 0] - ox, got[:, 1] - oy)) / d.max()
        assert err <= 1e-3, (c, err)


def test_kk_full_run_reaches_the_oracle_minimum(forest):
    """200 sweeps from the same start: the GPU run is stationary and ends at
    the oracle's energy (1e-4 relative) on every component, unless the
    oracle itself, from one-ulp moves of the start, ends at another local
    minimum -- another energy, or a layout more than 1e-3 of the diameter
    away (the larger components, where rounding decides which minimum the
    early sweeps fall into)."""
    bgl = _bgl()
    p = bgl.params(kk_sweeps=200)
    checked, excused = 0, []
    for c in _kk_components(forest, lo=3, hi=255, step=4):
        vs, loff, ladj, _ = forest.comp(c)
        d = oracle.bfs_apsp(loff, ladj)
        x, y = _kk_start(5, vs, d)
        xy = np.stack([x, y], 1).astype(np.float32)
        got = forest.g.kk_run(int(c), p, xy).astype(np.float64)
        ox, oy, e, _, _ = oracle.kk_run(xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64), d, 1.0, 200)
        eg = oracle.kk_energy(got[:, 0], got[:, 1], d, 1.0)
        gmax = max(np.hypot(*oracle.kk_grad_hess(got[:, 0], got[:, 1], d, 1.0, m)[:2]) for m in range(len(vs)))
        assert gmax <= 1e-3 * max(1.0, e[-1]), (c, gmax)
        checked += 1
        if kk_sensitivity.energy_close(eg, e[-1]):
            continue
        _, spread, other = kk_sensitivity.oracle_spread(xy[:, 0], xy[:, 1], d, 200)
        assert other or spread / max(1, int(d.max())) > 1e-3, (int(c), len(vs), eg, e[-1], spread)
        excused.append(int(c))
    assert checked > 60 and len(excused) <= checked // 4, (checked, excused)


# ------------------------------------------------------------------ FA2 forces

def _rel_force_err(f_gpu, f_ref, scale):
    return np.max(np.hypot(*(f_gpu - f_ref).T) / scale)


@pytest.mark.parametrize("seed", [1, 2])
def test_fa2_exact_forces_c1(c1, seed):
    bgl = _bgl()
    vs, loff, ladj, mass = c1.comp(0)
    x, y = oracle.init_positions(seed, vs)
    xy = np.stack([x, y], 1).astype(np.float32)
    for kr, kg in ((1.0, 1.0), (3.0, 0.2)):
        p = bgl.params(repulsion=bgl.REP_EXACT, kr=kr, kg=kg)
        f = c1.g.fa2_forces(0, p, xy)
        o = oracle.fa2_forces(xy[:, 0], xy[:, 1], mass, loff, ladj, kr, kg)
        ref = o["frep"] + o["fatt"] + o["fgrav"]
        assert _rel_force_err(f, ref, o["sabs"]) <= 1e-5
        fr = c1.g.fa2_repulsion(0, p, xy)
        assert _rel_force_err(fr, o["frep"], o["srep"]) <= 1e-5


def test_fa2_three_iterations_from_random_start(c1):
    # from random positions the iteration amplifies differences about tenfold
    # per iteration (the oracle against itself: 1e-7 -> 3e-5 of the diagonal
    # in 3 iterations, 4e-2 in 10), so positions are compared after 3
    bgl = _bgl()
    vs, loff, ladj, mass = c1.comp(0)
    x, y = oracle.init_positions(0, vs)
    xy = np.stack([x, y], 1).astype(np.float32)
    got, stats = c1.g.fa2_step(0, bgl.params(repulsion=bgl.REP_EXACT), 3, xy)
    st, ostats = oracle.fa2_run(xy[:, 0], xy[:, 1], mass, loff, ladj, 3)
    diag = math.hypot(np.ptp(st.x), np.ptp(st.y))
    assert np.max(np.hypot(got[:, 0] - st.x, got[:, 1] - st.y)) <= 1e-3 * diag
    assert np.allclose(stats, ostats, rtol=1e-4)


def test_fa2_host_loop_equals_device_loop(c1, monkeypatch):
    """BGL_HOST_LOOP=1 launches the captured iteration once per iteration from
    the host instead of the device-side loop; positions and statistics are
    bitwise the same (exact and FMM repulsion)."""
    bgl = _bgl()
    vs, loff, ladj, mass = c1.comp(0)
    x, y = oracle.init_positions(0, vs)
    xy = np.stack([x, y], 1).astype(np.float32)
    for p in (bgl.params(repulsion=bgl.REP_EXACT), bgl.params(repulsion=bgl.REP_FMM, fmm_p=8, leaf_size=16)):
        monkeypatch.delenv("BGL_HOST_LOOP", raising=False)
        a, sa = c1.g.fa2_step(0, p, 7, xy)
        monkeypatch.setenv("BGL_HOST_LOOP", "1")
        b, sb = c1.g.fa2_step(0, p, 7, xy)
        monkeypatch.delenv("BGL_HOST_LOOP", raising=False)
        assert np.array_equal(a, b) and np.array_equal(sa, sb)


def test_fa2_ten_iterations_match_oracle(c1):
    # ten fresh iterations (F_-1 = 0, s_G = 1) from a relaxed layout: the
    # oracle's 50-iteration result, rounded to FP32
    bgl = _bgl()
    vs, loff, ladj, mass = c1.comp(0)
    x, y = oracle.init_positions(0, vs)
    st0, _ = oracle.fa2_run(x, y, mass, loff, ladj, 50)
    xy = np.stack([st0.x, st0.y], 1).astype(np.float32)
    for variant in (0, 1):
        p = bgl.params(repulsion=bgl.REP_EXACT, swing_variant=variant)
        got, stats = c1.g.fa2_step(0, p, 10, xy)
        st, ostats = oracle.fa2_run(xy[:, 0], xy[:, 1], mass, loff, ladj, 10, variant=variant)
        diag = math.hypot(np.ptp(st.x), np.ptp(st.y))
        err = np.max(np.hypot(got[:, 0] - st.x, got[:, 1] - st.y))
        assert err <= 1e-3 * diag, (variant, err, diag)
        assert np.allclose(stats, ostats, rtol=1e-3)


def test_fa2_two_node_golden(ctx):
    bgl = _bgl()
    gold = json.load(open(os.path.join(GOLDEN, "fa2_two_node.json")))
    s, e = gold["setup"], gold["expected"]
    g = bgl.Graph.from_edges(ctx, 2, [0], [1])
    g.components()
    p = bgl.params(repulsion=bgl.REP_EXACT, kr=s["kr"], kg=s["kg"], ks=s["ks"], ksmax=s["ksmax"], tau=s["tau"])
    xy = np.array([s["p0"], s["p1"]], np.float32)
    got, stats = g.fa2_step(0, p, 1, xy)
    assert got[0, 0] == pytest.approx(e["x0_after_1"], rel=1e-6)
    assert got[1, 0] == pytest.approx(e["x1_after_1"], rel=1e-6)
    assert np.allclose(stats[0], e["stats_1"], rtol=1e-6)
    got, stats = g.fa2_step(0, p, 2, xy)
    assert got[0, 0] == pytest.approx(e["x0_after_2"], rel=1e-5)
    assert np.allclose(stats[1], e["stats_2"], rtol=1e-5)
    g.destroy()


def test_fa2_exact_forces_c2_sampled(ctx):
    """Full-size giant component (~5.5e5 nodes): forces on 2000 sampled nodes."""
    bgl = _bgl()
    tx = synth.tx_lists(**synth.C2)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    off, adj = g.csr()
    vs = nodes[coff[0]:coff[1]]
    pos = np.full(len(off) - 1, -1, np.int64)
    pos[vs] = np.arange(len(vs))
    loff = np.zeros(len(vs) + 1, np.int64)
    loff[1:] = np.cumsum(np.diff(off)[vs])
    ladj = pos[np.concatenate([adj[off[v]:off[v + 1]] for v in vs])].astype(np.int32)
    mass = np.diff(loff) + 1.0
    x, y = oracle.init_positions(2, vs)
    xy = np.stack([x, y], 1).astype(np.float32)
    p = bgl.params(repulsion=bgl.REP_EXACT)
    f = g.fa2_forces(0, p, xy)
    tg = np.random.default_rng(2).choice(len(vs), 2000, replace=False)
    o = oracle.fa2_forces(xy[:, 0], xy[:, 1], mass, loff, ladj, 1.0, 1.0, targets=tg)
    ref = o["frep"] + o["fatt"] + o["fgrav"]
    assert _rel_force_err(f[tg], ref, o["sabs"]) <= 1e-5
    g.destroy()


# ------------------------------------------------------------------ whole layout

def _edge_stats(xy, og):
    e = og.src, og.dst
    d = np.hypot(xy[e[0], 0] - xy[e[1], 0], xy[e[0], 1] - xy[e[1], 1])
    return d.mean(), np.percentile(d, 50), np.percentile(d, 90)


def test_layout_c1_against_oracle(c1):
    bgl = _bgl()
    p = bgl.params(seed=1, repulsion=bgl.REP_EXACT)
    xy = c1.g.layout(p).astype(np.float64)
    again = c1.g.layout(p).astype(np.float64)
    assert np.array_equal(xy, again)                   # bitwise reproducible
    oxy = oracle.layout(c1.og, seed=1)
    sizes = np.diff(c1.coff)
    # singletons at the origin
    for c in np.flatnonzero(sizes == 1):
        assert np.all(xy[c1.nodes[c1.coff[c]]] == 0)
    # ForceAtlas2 component: energy within 1%, edge lengths within 2%
    vs, loff, ladj, mass = c1.comp(0)
    eg = oracle.fa2_energy(xy[vs, 0], xy[vs, 1], mass, loff, ladj)
    eo = oracle.fa2_energy(oxy[vs, 0], oxy[vs, 1], mass, loff, ladj)
    assert abs(eg - eo) <= 0.01 * abs(eo)
    sub = np.isin(c1.og.src, vs)

    class E:
        src, dst = c1.og.src[sub], c1.og.dst[sub]
    for a, b in zip(_edge_stats(xy, E), _edge_stats(oxy, E)):
        assert abs(a - b) <= 0.02 * b
    # KK components (at most 50 nodes, where the oracle's minimum does not
    # depend on rounding of the start): stationary and at the oracle's
    # energy, every one of them
    for c in np.flatnonzero((sizes >= 2) & (sizes <= 50)):
        vs, loff, ladj, _ = c1.comp(c)
        d = oracle.bfs_apsp(loff, ladj)
        eg = oracle.kk_energy(xy[vs, 0], xy[vs, 1], d)
        eo = oracle.kk_energy(oxy[vs, 0], oxy[vs, 1], d)
        gmax = max(np.hypot(*oracle.kk_grad_hess(xy[vs, 0], xy[vs, 1], d, 1.0, m)[:2]) for m in range(len(vs)))
        assert gmax <= 1e-3 * max(1.0, eo), (c, gmax)
        assert kk_sensitivity.energy_close(eg, eo), (int(c), len(vs), eg, eo)


def test_layout_host_loop_equals_device_loop(c1, monkeypatch):
    """A whole layout with KK and ForceAtlas2 components: the KK size
    classes run beside the iterations (in the same graph with the device
    loop, on a side stream with the host loop); both give the same bits."""
    bgl = _bgl()
    for p in (bgl.params(seed=2, fa2_iters=12, kk_sweeps=40, repulsion=bgl.REP_EXACT),
              bgl.params(seed=2, fa2_iters=12, kk_sweeps=40, repulsion=bgl.REP_FMM, fmm_p=8, leaf_size=32)):
        monkeypatch.delenv("BGL_HOST_LOOP", raising=False)
        a = c1.g.layout(p)
        monkeypatch.setenv("BGL_HOST_LOOP", "1")
        b = c1.g.layout(p)
        monkeypatch.delenv("BGL_HOST_LOOP", raising=False)
        assert np.array_equal(a, b)
