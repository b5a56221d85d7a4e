"""Pins for the FP64 oracle: each check ties it to something other than itself.

Sources of truth: hand-worked examples from the paper's definitions
(tests/golden/), published test vectors, closed forms, invariants
(antisymmetry, scaling, rotation), finite-difference gradients, library
routines (scipy shortest paths, networkx components) and brute force.
"""
import json
import math
import os

import numpy as np
import pytest

import kk_sensitivity
import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------- initial positions

def test_splitmix64_published_vectors():
    g = _golden("splitmix64.json")
    for vec in g["vectors"]:
        out = oracle.splitmix64_stream(vec["seed"], 3)
        if "outputs_hex" in vec:
            want = [int(h, 16) for h in vec["outputs_hex"]]
        else:
            want = [int(d) for d in vec["outputs_dec"]]
        assert [int(v) for v in out] == want


def test_init_positions_from_published_stream():
    # node id 0 under seed 0 starts the stream at state 0: outputs are the
    # published seed-0 vector, so x, y follow from its top 24 bits.
    x, y = oracle.init_positions(0, [0])
    assert x[0] == (0xE220A8 / 2.0 ** 24) * 2 - 1
    assert y[0] == (0x6E789E / 2.0 ** 24) * 2 - 1
    xs, ys = oracle.init_positions(7, np.arange(10000))
    for v in (xs, ys):
        assert v.min() >= -1.0 and v.max() < 1.0
        assert np.all(v.astype(np.float32).astype(np.float64) == v)   # exact in float32
        assert abs(v.mean()) < 0.03


# ------------------------------------------------------------- Section 2 graph build

def _tx_from_case(case):
    names = {}
    keys = {}
    for nm in sorted({a for t in case["tx"] for a in t["in"] + t["out"]}):
        # opaque keys in an order unrelated to first appearance
        keys[nm] = (hash(nm) * 0 + (1 << 63)) - 7919 * (ord(nm) * 104729 % 1009)
        names[keys[nm]] = nm
    in_off = [0]
    out_off = [0]
    in_addr = []
    out_addr = []
    for t in case["tx"]:
        in_addr += [keys[a] for a in t["in"]]
        out_addr += [keys[a] for a in t["out"]]
        in_off.append(len(in_addr))
        out_off.append(len(out_addr))
    return (np.array(in_off), np.array(in_addr, np.uint64), np.array(out_off),
            np.array(out_addr, np.uint64), keys)


@pytest.mark.parametrize("idx", [0, 1])
def test_graph_build_golden(idx):
    case = _golden("txgraph_small.json")["cases"][idx]
    in_off, in_addr, out_off, out_addr, keys = _tx_from_case(case)
    g = oracle.graph_build(in_off, in_addr, out_off, out_addr)
    T = len(case["tx"])
    for nm, id_ in case["addr_ids"].items():
        assert int(g.addr[id_ - T]) == keys[nm]
    assert np.stack([g.src, g.dst], 1).tolist() == case["edges"]
    und = sorted({(min(a, b), max(a, b)) for a, b in case["edges"] if a != b})
    assert [list(p) for p in und] == case["undirected"]
    assert g.deg.tolist() == case["deg"]
    label, nc = oracle.components(g.off, g.adj)
    assert label.tolist() == case["label"]
    comp_off, comp_label, nodes = oracle.component_order(label)
    got = [nodes[comp_off[c]:comp_off[c + 1]].tolist() for c in range(len(comp_off) - 1)]
    assert got == case["comp_nodes"]
    assert nc == len(case["comp_nodes"])


def test_graph_build_invariants_c1():
    tx = synth.tx_lists(**synth.C1)
    g = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    T = tx.n_tx
    # every edge joins a transaction and an address (bipartite, Section 2)
    assert np.all((g.src < T) != (g.dst < T))
    # inputs point address -> tx, outputs tx -> address; count before dedupe
    assert len(g.src) <= len(tx.in_addr) + len(tx.out_addr)
    # directed edges unique and sorted
    key = g.src.astype(np.int64) << 32 | g.dst.astype(np.int64)
    assert np.all(np.diff(key) > 0)
    # sum of degrees = 2E; rows sorted, symmetric
    assert int(g.deg.sum()) == 2 * g.n_undirected
    for v in range(0, g.n_nodes, 37):
        row = g.adj[g.off[v]:g.off[v + 1]]
        assert np.all(np.diff(row) > 0)
        for w in row:
            assert v in g.adj[g.off[w]:g.off[w + 1]]
    # first-appearance order of address ids: brute-force scan
    seen = {}
    for t in range(T):
        for a in list(tx.in_addr[tx.in_off[t]:tx.in_off[t + 1]]) + list(tx.out_addr[tx.out_off[t]:tx.out_off[t + 1]]):
            seen.setdefault(int(a), len(seen))
    assert len(seen) == len(g.addr) == tx.n_addr_created
    assert all(seen[int(a)] == k for k, a in enumerate(g.addr))


# ------------------------------------------------------------- Section 4 components

def test_components_vs_networkx():
    nx = pytest.importorskip("networkx")
    tx = synth.tx_lists(**synth.C1)
    g = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    label, nc = oracle.components(g.off, g.adj)
    G = nx.Graph()
    G.add_nodes_from(range(g.n_nodes))
    G.add_edges_from(zip(g.src.tolist(), g.dst.tolist()))
    comps = list(nx.connected_components(G))
    assert nc == len(comps)
    for c in comps:
        m = min(c)
        assert all(label[v] == m for v in c)
    comp_off, comp_label, nodes = oracle.component_order(label)
    sizes = np.diff(comp_off)
    assert np.all(sizes[:-1] >= sizes[1:])
    assert sorted(sizes.tolist(), reverse=True) == sorted((len(c) for c in comps), reverse=True)
    for c in range(len(sizes)):
        vs = nodes[comp_off[c]:comp_off[c + 1]]
        assert np.all(np.diff(vs) > 0) and np.all(label[vs] == comp_label[c])
        if c + 1 < len(sizes) and sizes[c] == sizes[c + 1]:
            assert comp_label[c] < comp_label[c + 1]


def _bfs_labels(n, off, adj):
    label = np.full(n, -1)
    for s in range(n):
        if label[s] >= 0:
            continue
        stack = [s]
        label[s] = s
        while stack:
            v = stack.pop()
            for w in adj[off[v]:off[v + 1]]:
                if label[w] < 0:
                    label[w] = s
                    stack.append(w)
    return label


def test_components_vs_bfs_forest():
    sizes, u, v = synth.forest(11, 300, 1.0, 40.0)
    n = int(sizes.sum())
    g = oracle.graph_from_edges(n, u, v)
    label, nc = oracle.components(g.off, g.adj)
    assert nc == len(sizes)
    assert np.array_equal(label, _bfs_labels(n, g.off, g.adj))


# ------------------------------------------------------------- Section 3.1 distances

def _random_connected(rng, n, extra):
    u = [int(rng.integers(0, k)) for k in range(1, n)]
    v = list(range(1, n))
    for _ in range(extra):
        a, b = rng.integers(0, n, 2)
        u.append(int(a))
        v.append(int(b))
    return oracle.graph_from_edges(n, u, v)


def test_bfs_vs_floyd_warshall_and_scipy():
    csg = pytest.importorskip("scipy.sparse.csgraph")
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(1, 31))
        g = _random_connected(rng, n, int(rng.integers(0, n + 1)))
        d = oracle.bfs_apsp(g.off, g.adj)
        assert np.array_equal(d, oracle.floyd_warshall(g.off, g.adj))
        if n > 1:
            A = sp.csr_matrix((np.ones(len(g.adj)), g.adj, g.off), shape=(n, n))
            ds = csg.shortest_path(A, unweighted=True, directed=False)
            assert np.array_equal(d, ds.astype(np.int32))
        assert np.array_equal(d, d.T) and np.all(np.diag(d) == 0)
        for a in range(n):
            for b in g.adj[g.off[a]:g.off[a + 1]]:
                assert np.all(np.abs(d[a] - d[b]) <= 1)


def test_bfs_unreachable_marked():
    g = oracle.graph_from_edges(4, [0], [1])
    d = oracle.bfs_apsp(g.off, g.adj)
    assert d[0, 1] == 1 and d[0, 2] == -1 and d[2, 3] == -1 and d[3, 3] == 0


def test_floyd_warshall_marks_unreachable_pairs_as_bfs_does():
    """Two paths 0-1-2 and 3-4 plus the isolated node 5: distances inside a
    part are path lengths, every pair across parts is -1 (both methods)."""
    g = oracle.graph_from_edges(6, [0, 1, 3], [1, 2, 4])
    want = np.full((6, 6), -1, np.int32)
    for part in ([0, 1, 2], [3, 4], [5]):
        for a in part:
            for b in part:
                want[a, b] = abs(a - b)
    assert np.array_equal(oracle.floyd_warshall(g.off, g.adj), want)
    assert np.array_equal(oracle.bfs_apsp(g.off, g.adj), want)


# ------------------------------------------------------------- Section 3.2 forces

def _two_node():
    off = np.array([0, 1, 2])
    adj = np.array([1, 0], np.int32)
    return off, adj


def test_fa2_two_node_closed_form():
    off, adj = _two_node()
    for d in (0.5, 1.0, 3.0):
        for kr, kg in ((1.0, 1.0), (2.5, 0.3)):
            f = oracle.fa2_forces([0.0, d], [0.0, 0.0], [2.0, 2.0], off, adj, kr, kg)
            assert np.allclose(f["frep"][0], [-4 * kr / d, 0], rtol=1e-15, atol=0)
            assert np.allclose(f["fatt"][0], [d, 0], rtol=1e-15, atol=0)
            assert np.allclose(f["fgrav"][0], [0, 0], atol=0)
            assert np.allclose(f["frep"][1], [4 * kr / d, 0], rtol=1e-15)
            assert np.allclose(f["fgrav"][1], [-2 * kg * d, 0], rtol=1e-15)
            # error scales: repulsion terms kr m_i m_j / d; all terms adds |p_i - p_j| and |kg m_i p_i|
            assert np.allclose(f["srep"], [4 * kr / d, 4 * kr / d], rtol=1e-15, atol=0)
            assert np.allclose(f["sabs"], [4 * kr / d + d, 4 * kr / d + d + 2 * kg * d], rtol=1e-15, atol=0)
            # E = |p0 - p1|^2 / 2 - kr m0 m1 ln|p0 - p1| + kg (m0 |p0|^2 + m1 |p1|^2) / 2
            e = oracle.fa2_energy([0.0, d], [0.0, 0.0], [2.0, 2.0], off, adj, kr, kg)
            assert e == pytest.approx(d * d / 2 - 4 * kr * math.log(d) + kg * d * d, rel=1e-14, abs=1e-15)


def _comp_c1(kind="largest"):
    tx = synth.tx_lists(**synth.C1)
    g = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    label, _ = oracle.components(g.off, g.adj)
    comp_off, _, nodes = oracle.component_order(label)
    vs = nodes[comp_off[0]:comp_off[1]]
    loff, ladj = oracle.subgraph(g.off, g.adj, vs)
    mass = np.diff(loff) + 1.0
    return vs, loff, ladj, mass


def test_fa2_antisymmetry_scaling_rotation():
    vs, off, adj, mass = _comp_c1()
    x, y = oracle.init_positions(3, vs)
    f = oracle.fa2_forces(x, y, mass, off, adj, 1.0, 1.0)
    for key in ("frep", "fatt"):
        tot = np.abs(f[key]).sum()
        assert np.all(np.abs(f[key].sum(0)) <= 1e-12 * tot)
    a = 3.7
    fa = oracle.fa2_forces(a * x, a * y, mass, off, adj, 1.0, 1.0)
    assert np.allclose(fa["frep"], f["frep"] / a, rtol=1e-10, atol=1e-12 * np.abs(f["frep"]).max())
    assert np.allclose(fa["fatt"], f["fatt"] * a, rtol=1e-10, atol=1e-12 * np.abs(fa["fatt"]).max())
    assert np.allclose(fa["fgrav"], f["fgrav"] * a, rtol=1e-12)
    th = 0.61
    c, s = math.cos(th), math.sin(th)
    fr = oracle.fa2_forces(c * x - s * y, s * x + c * y, mass, off, adj, 1.0, 1.0)
    for key in ("frep", "fatt", "fgrav"):
        want = np.stack([c * f[key][:, 0] - s * f[key][:, 1], s * f[key][:, 0] + c * f[key][:, 1]], 1)
        assert np.allclose(fr[key], want, rtol=1e-9, atol=1e-10 * np.abs(want).max())


def test_fa2_force_is_negative_energy_gradient():
    vs, off, adj, mass = _comp_c1()
    vs, off, adj, mass = vs, off, adj, mass
    x, y = oracle.init_positions(9, vs)
    kr, kg = 1.3, 0.7
    f = oracle.fa2_forces(x, y, mass, off, adj, kr, kg)
    ftot = f["frep"] + f["fatt"] + f["fgrav"]
    h = 1e-6
    rng = np.random.default_rng(0)
    for i in rng.choice(len(vs), 12, replace=False):
        for ax in (0, 1):
            xp, yp, xm, ym = x.copy(), y.copy(), x.copy(), y.copy()
            if ax == 0:
                xp[i] += h
                xm[i] -= h
            else:
                yp[i] += h
                ym[i] -= h
            g = (oracle.fa2_energy(xp, yp, mass, off, adj, kr, kg)
                 - oracle.fa2_energy(xm, ym, mass, off, adj, kr, kg)) / (2 * h)
            assert abs(-g - ftot[i, ax]) <= 1e-5 * (1 + f["sabs"][i])


def test_fa2_coincident_pair_contributes_nothing():
    off = np.array([0, 0, 0, 0])
    adj = np.zeros(0, np.int32)
    f = oracle.fa2_forces([1.0, 1.0, 2.0], [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], off, adj, 1.0, 0.0)
    assert np.allclose(f["frep"][0], [-1.0, 0.0]) and np.all(np.isfinite(f["frep"]))
    assert f["srep"][0] == 1.0 and f["srep"][2] == 2.0
    # the energy omits the coincident pair: -ln 2 - ln 2 from the pairs with node 2 at distance 2
    e = oracle.fa2_energy([1.0, 1.0, 3.0], [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], off, adj, 1.0, 0.0)
    assert e == pytest.approx(-2 * math.log(2.0), rel=1e-15)


def test_fa2_two_node_iterations_golden():
    g = _golden("fa2_two_node.json")
    s, e = g["setup"], g["expected"]
    off, adj = _two_node()
    x = [s["p0"][0], s["p1"][0]]
    y = [s["p0"][1], s["p1"][1]]
    st, stats = oracle.fa2_run(x, y, s["mass"], off, adj, 1, s["kr"], s["kg"], s["ks"], s["ksmax"], s["tau"])
    assert st.x[0] == pytest.approx(e["x0_after_1"], rel=1e-14)
    assert st.x[1] == pytest.approx(e["x1_after_1"], rel=1e-14)
    assert np.allclose(stats[0], e["stats_1"], rtol=1e-14)
    st, stats = oracle.fa2_run(None, None, s["mass"], off, adj, 1, s["kr"], s["kg"], s["ks"], s["ksmax"],
                               s["tau"], state=st)
    assert np.allclose(stats[0], e["stats_2"], rtol=1e-13)
    assert st.x[0] == pytest.approx(e["x0_after_2"], rel=1e-13)
    assert st.fpx[0] == pytest.approx(e["F0_iter2"], rel=1e-13)
    assert np.all(st.y == 0)


@pytest.mark.parametrize("variant", [0, 1])
def test_fa2_swing_variants_golden(variant):
    """One iteration of a three-node path with unequal masses from a given
    F_{t-1} and s_G, worked by hand: pins the printed (unweighted) sums and
    ForceAtlas2's mass-weighted sums with halved traction."""
    gd = _golden("fa2_swing_variants.json")
    s, e = gd["setup"], gd["expected"]
    g = oracle.graph_from_edges(3, [a for a, _ in s["edges"]], [b for _, b in s["edges"]])
    assert np.array_equal(np.diff(g.off) + 1.0, s["mass"])
    st = oracle.FA2State(np.array(s["x"]), np.array(s["y"]), np.array(s["fprev_x"], float),
                         np.array(s["fprev_y"], float), s["sg"])
    st, stats = oracle.fa2_run(None, None, s["mass"], g.off, g.adj, 1, s["kr"], s["kg"], s["ks"], s["ksmax"],
                               s["tau"], variant=variant, state=st)
    ev = e[f"variant{variant}"]
    assert np.allclose(stats[0], ev["stats"], rtol=1e-14, atol=0)
    assert np.allclose(st.x, ev["x"], rtol=1e-14, atol=0)
    assert np.allclose(st.fpx, e["F_x"], rtol=1e-14, atol=0)
    assert np.all(st.y == 0) and np.all(st.fpy == 0)


@pytest.mark.parametrize("case", range(len(_golden("fa2_iteration_2d.json")["cases"])))
def test_fa2_iteration_2d_golden(case):
    """One iteration of one edge off the axes, worked by hand: tau != 1,
    s_G != 1 with the 1.5 s_G cap binding and not, the ksmax cap binding for
    one node only and for forces shorter than 1/2, variant 1, a small swing
    with a large s_G, and F_t = F_{t-1} (swg = 0)."""
    gd = _golden("fa2_iteration_2d.json")
    cm, c = gd["common"], gd["cases"][case]
    g = oracle.graph_from_edges(2, [0], [1])
    assert np.array_equal(np.diff(g.off) + 1.0, cm["mass"])
    st = oracle.FA2State(np.array(c.get("x0", cm["x"])), np.array(c.get("y0", cm["y"])), np.array(c["fprev_x"]),
                         np.array(c["fprev_y"]), c["sg"])
    st, stats = oracle.fa2_run(None, None, cm["mass"], g.off, g.adj, 1, c["kr"], c["kg"], cm["ks"], c["ksmax"],
                               c["tau"], variant=c["variant"], state=st)
    assert np.allclose(stats[0], c["stats"], rtol=1e-14, atol=1e-15), c["name"]
    assert np.allclose(st.x, c["x"], rtol=1e-14, atol=1e-15), c["name"]
    assert np.allclose(st.y, c["y"], rtol=1e-14, atol=1e-15), c["name"]
    assert np.allclose(st.fpx, c["F_x"], rtol=1e-14, atol=1e-15) and np.allclose(st.fpy, c["F_y"], rtol=1e-14,
                                                                                 atol=1e-15)
    assert st.sg == pytest.approx(c["stats"][2], rel=1e-14)


def test_fa2_speed_cap_limits_displacement():
    # with ksmax = 0.01 every node moves exactly 0.01 in the first iteration
    vs, off, adj, mass = _comp_c1()
    x, y = oracle.init_positions(1, vs)
    st, _ = oracle.fa2_run(x, y, mass, off, adj, 1, ks=1e6, ksmax=0.01)
    disp = np.hypot(st.x - x, st.y - y)
    assert np.allclose(disp, 0.01, rtol=1e-12)


def test_fa2_energy_decreases_early():
    vs, off, adj, mass = _comp_c1()
    x, y = oracle.init_positions(1, vs)
    e0 = oracle.fa2_energy(x, y, mass, off, adj)
    st, stats = oracle.fa2_run(x, y, mass, off, adj, 20)
    e1 = oracle.fa2_energy(st.x, st.y, mass, off, adj)
    assert e1 < e0
    assert np.all(stats[:, 2] > 0) and np.all(stats[1:, 2] <= 1.5 * stats[:-1, 2] * (1 + 1e-15))


# ------------------------------------------------------------- Section 3.1 Kamada-Kawai

def test_kk_gradient_hessian_finite_differences():
    rng = np.random.default_rng(2)
    g = _random_connected(rng, 12, 4)
    d = oracle.bfs_apsp(g.off, g.adj)
    x = rng.normal(size=12) * 2
    y = rng.normal(size=12) * 2
    l = 1.3
    h = 1e-5
    for m in range(12):
        o = oracle.kk_grad_hess(x, y, d, l, m)

        def E(dx, dy):
            xx, yy = x.copy(), y.copy()
            xx[m] += dx
            yy[m] += dy
            return oracle.kk_energy(xx, yy, d, l)

        gx = (E(h, 0) - E(-h, 0)) / (2 * h) / 2
        gy = (E(0, h) - E(0, -h)) / (2 * h) / 2
        k = 2e-3   # second differences: larger step keeps cancellation small
        hxx = (E(k, 0) - 2 * E(0, 0) + E(-k, 0)) / k ** 2 / 2
        hyy = (E(0, k) - 2 * E(0, 0) + E(0, -k)) / k ** 2 / 2
        hxy = (E(k, k) - E(k, -k) - E(-k, k) + E(-k, -k)) / (4 * k * k) / 2
        assert np.allclose(o[:2], [gx, gy], rtol=1e-6, atol=1e-8)
        assert np.allclose(o[2:], [hxx, hxy, hyy], rtol=1e-4, atol=1e-5)


def test_kk_coincident_pair_contributes_nothing():
    """A node at the same place as p_m adds no term to p_m's gradient and
    Hessian (r = 0 has no direction); the other terms are the textbook sums:
    with p_m = (0, 0), a coincident node and a node at (2, 0) at graph
    distance 1 (k = 1, l_mi = l = 1): g = (dx - l dx / r, 0) = (-1, 0),
    H_xx = 1 - l dy^2 / r^3 = 1, H_yy = 1 - l dx^2 / r^3 = 1 / 2, H_xy = 0."""
    g = oracle.graph_from_edges(3, [0, 0], [1, 2])
    d = oracle.bfs_apsp(g.off, g.adj)
    o = oracle.kk_grad_hess(np.array([0.0, 0.0, 2.0]), np.array([0.0, 0.0, 0.0]), d, 1.0, 0)
    assert np.allclose(o, [-1.0, 0.0, 1.0, 0.0, 0.5], rtol=1e-15, atol=0)
    assert np.isfinite(oracle.kk_energy(np.array([0.0, 0.0, 2.0]), np.zeros(3), d, 1.0))


@pytest.mark.parametrize("case", range(len(_golden("kk_newton_step.json")["cases"])))
def test_kk_newton_step_golden(case):
    """The safeguarded 2x2 Newton step against hand-worked cases: the plain
    step, the step shortened to l, eigenvalues replaced where H is
    indefinite, the floor at 0.1 max|l|, and no step for H = 0."""
    c = _golden("kk_newton_step.json")["cases"][case]
    step, moved = oracle.kk_step(c["g"], c["H"], c["l"])
    assert moved == c["moved"], c["name"]
    if moved:
        assert np.allclose(step, c["step"], rtol=1e-14, atol=1e-16), (c["name"], step)


def test_kk_two_nodes_reach_distance_l():
    g = oracle.graph_from_edges(2, [0], [1])
    d = oracle.bfs_apsp(g.off, g.adj)
    for l in (1.0, 2.5):
        x, y, e, _, _ = oracle.kk_run([0.3, -0.1], [0.2, 0.4], d, l, 50)
        assert math.hypot(x[0] - x[1], y[0] - y[1]) == pytest.approx(l, rel=1e-12)


def test_kk_run_energy_trace_skips_and_tolerance_stop():
    """The run's outputs by their definitions: energy[s] is the energy after
    sweep s + 1 (a run of s + 1 sweeps from the same start ends there); a
    node whose Hessian is zero is skipped and counted, once per sweep; with
    tol > 0 the run ends after the first sweep in which no node saw a
    gradient of length tol or more."""
    rng = np.random.default_rng(8)
    g = _random_connected(rng, 7, 3)
    d = oracle.bfs_apsp(g.off, g.adj)
    x0, y0 = rng.normal(size=7), rng.normal(size=7)
    _, _, e, skipped, done = oracle.kk_run(x0, y0, d, 1.0, 6)
    assert done == 6 and skipped == 0 and len(e) == 6
    for s in range(6):
        xs, ys, _, _, _ = oracle.kk_run(x0, y0, d, 1.0, s + 1)
        assert e[s] == oracle.kk_energy(xs, ys, d, 1.0)
    # two coincident nodes: r = 0 leaves both Hessians zero, both skipped
    g2 = oracle.graph_from_edges(2, [0], [1])
    d2 = oracle.bfs_apsp(g2.off, g2.adj)
    x, y, e2, skipped, done = oracle.kk_run([0.5, 0.5], [1.0, 1.0], d2, 1.0, 3)
    assert (skipped, done) == (6, 3) and list(x) == [0.5, 0.5] and list(y) == [1.0, 1.0]
    # already at the minimum: the first sweep sees g = 0 and ends the run
    x, y, _, _, done = oracle.kk_run([0.0, 1.0], [0.0, 0.0], d2, 1.0, 50, tol=1e-9)
    assert done == 1
    # from 3 l apart the first sweep sees |g| > tol, so at least two sweeps
    # run, and the run ends well before 50 once the distance is l
    x, y, _, _, done = oracle.kk_run([0.0, 3.0], [0.0, 0.0], d2, 1.0, 50, tol=1e-9)
    assert 2 <= done < 50
    assert math.hypot(x[0] - x[1], y[0] - y[1]) == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_kk_path_becomes_straight(n):
    g = oracle.graph_from_edges(n, list(range(n - 1)), list(range(1, n)))
    d = oracle.bfs_apsp(g.off, g.adj)
    x, y = oracle.init_positions(4, np.arange(n))
    x, y = x * (n - 1) / 2, y * (n - 1) / 2
    x, y, e, _, _ = oracle.kk_run(x, y, d, 1.0, 300)
    # the straight path is the exact minimum (E = 0)
    assert e[-1] < 1e-16
    for i in range(n):
        for j in range(n):
            assert math.hypot(x[i] - x[j], y[i] - y[j]) == pytest.approx(abs(i - j), abs=1e-7)


def test_kk_triangle_is_equilateral():
    g = oracle.graph_from_edges(3, [0, 1, 2], [1, 2, 0])
    d = oracle.bfs_apsp(g.off, g.adj)
    x, y, e, _, _ = oracle.kk_run([0.0, 0.5, 0.1], [0.0, 0.05, 0.7], d, 2.0, 100)
    for i, j in ((0, 1), (1, 2), (0, 2)):
        assert math.hypot(x[i] - x[j], y[i] - y[j]) == pytest.approx(2.0, rel=1e-10)
    assert e[-1] < 1e-20


def test_kk_stationary_and_monotone_on_small_components():
    sizes, u, v = synth.forest(21, 40, 3.0, 50.0)
    n = int(sizes.sum())
    g = oracle.graph_from_edges(n, u, v)
    label, _ = oracle.components(g.off, g.adj)
    comp_off, _, nodes = oracle.component_order(label)
    for c in range(len(comp_off) - 1):
        vs = nodes[comp_off[c]:comp_off[c + 1]]
        loff, ladj = oracle.subgraph(g.off, g.adj, vs)
        d = oracle.bfs_apsp(loff, ladj)
        x, y = oracle.init_positions(1, vs)
        sc = d.max() / 2
        x, y, e, skipped, _ = oracle.kk_run(x * sc, y * sc, d, 1.0, 200)
        gmax = max(np.hypot(*oracle.kk_grad_hess(x, y, d, 1.0, m)[:2]) for m in range(len(vs)))
        assert gmax <= 1e-6, (c, len(vs), gmax)
        # Newton-Raphson on an indefinite Hessian may climb for a few sweeps
        # (monitored, not assumed); the run must still end below its start
        # and stay at the minimum once there.
        x0, y0 = oracle.init_positions(1, vs)
        e0 = oracle.kk_energy(x0 * sc, y0 * sc, d, 1.0)
        assert e[-1] <= e0
        assert np.all(np.abs(np.diff(e[-20:])) <= 1e-9 * e[-1] + 1e-12)


def _kk_fp32_start(seed, vs, d):
    x, y = oracle.init_positions(seed, vs)
    sc = np.float32(d.max() / 2)
    return (x.astype(np.float32) * sc).astype(np.float32), (y.astype(np.float32) * sc).astype(np.float32)


def test_kk_small_components_do_not_hinge_on_rounding():
    """On the KK components of the 1,000-transaction graph (at most 50 nodes),
    200 oracle sweeps from one-ulp moves of the FP32 start end at the same
    energy as from the start itself: a GPU run must match every one."""
    tx = synth.tx_lists(**synth.C1)
    g = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    label, _ = oracle.components(g.off, g.adj)
    comp_off, _, nodes = oracle.component_order(label)
    sizes = np.diff(comp_off)
    comps = np.flatnonzero((sizes >= 2) & (sizes <= 50))
    assert len(comps) > 100
    for c in comps:
        vs = nodes[comp_off[c]:comp_off[c + 1]]
        loff, ladj = oracle.subgraph(g.off, g.adj, vs)
        d = oracle.bfs_apsp(loff, ladj)
        x, y = _kk_fp32_start(1, vs, d)
        _, _, other = kk_sensitivity.oracle_spread(x, y, d, 200)
        assert not other, (int(c), len(vs))


def test_kk_large_components_hinge_on_rounding():
    """The reading that KK from random starts is chaotic, shown on the oracle
    alone: among forest components of 150-200 nodes, a one-ulp move of the
    FP32 start sends at least a quarter of the 200-sweep runs to another
    energy minimum (so an FP32 run cannot be held to the oracle's minimum
    there), while the small ones above never move."""
    sizes, u, v = synth.forest(17, 300, 3.0, 200.0)
    g = oracle.graph_from_edges(int(sizes.sum()), u, v)
    label, _ = oracle.components(g.off, g.adj)
    comp_off, _, nodes = oracle.component_order(label)
    sz = np.diff(comp_off)
    comps = np.flatnonzero(sz >= 150)[::2]
    assert len(comps) >= 8
    moved = 0
    for c in comps:
        vs = nodes[comp_off[c]:comp_off[c + 1]]
        loff, ladj = oracle.subgraph(g.off, g.adj, vs)
        d = oracle.bfs_apsp(loff, ladj)
        x, y = _kk_fp32_start(5, vs, d)
        _, _, other = kk_sensitivity.oracle_spread(x, y, d, 200)
        moved += other
    assert moved >= len(comps) / 4, (moved, len(comps))


# ------------------------------------------------------------- Section 4 whole layout

def test_layout_c1_shapes():
    tx = synth.tx_lists(**synth.C1)
    g = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    xy = oracle.layout(g, fa2_iters=2, kk_sweeps=5, seed=1)
    assert xy.shape == (g.n_nodes, 2) and np.all(np.isfinite(xy))
    label, _ = oracle.components(g.off, g.adj)
    iso = np.diff(g.off) == 0
    assert np.all(xy[iso] == 0)


# ------------------------------------------------------------- Section 4 assembly

def test_meta_tree_golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "meta_tree.json")) as f:
        gold = json.load(f)
    assert oracle.meta_tree(np.array(gold["sizes"])).tolist() == gold["parents"]


def test_meta_tree_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(50):
        sizes = rng.integers(1, 6, rng.integers(1, 12))
        par = oracle.meta_tree(sizes)
        for k in range(1, len(sizes)):
            best = max(sizes[:k])
            assert par[k] == min(j for j in range(k) if sizes[j] == best)


def test_tree_distances_vs_scipy():
    sp = pytest.importorskip("scipy.sparse.csgraph")
    from scipy.sparse import coo_matrix
    rng = np.random.default_rng(5)
    for m in (1, 2, 7, 30):
        parent = np.array([-1] + [int(rng.integers(0, k)) for k in range(1, m)])
        length = np.concatenate([[0.0], rng.uniform(0.5, 4.0, m - 1)])
        d = oracle.tree_distances(parent, length)
        if m > 1:
            a = coo_matrix((length[1:], (np.arange(1, m), parent[1:])), shape=(m, m)).tocsr()
            ref = sp.shortest_path(a, directed=False)
        else:
            ref = np.zeros((1, 1))
        assert np.allclose(d, ref, rtol=1e-12, atol=1e-12)


def test_kkw_equals_kk_on_integer_distances():
    # with l = 1 and hop distances the weighted energy is the Section 3.1 energy
    sizes, u, v = synth.forest(23, 3, 6.0, 30.0)
    g = oracle.graph_from_edges(int(sizes.sum()), u, v)
    label, _ = oracle.components(g.off, g.adj)
    comp_off, _, nodes = oracle.component_order(label)
    vs = nodes[comp_off[0]:comp_off[1]]
    loff, ladj = oracle.subgraph(g.off, g.adj, vs)
    d = oracle.bfs_apsp(loff, ladj)
    x, y = oracle.init_positions(2, vs)
    sc = d.max() / 2
    a = oracle.kk_run(x * sc, y * sc, d, 1.0, 15)
    b = oracle.kkw_run(x * sc, y * sc, d.astype(np.float64), 1.0, 15)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_kkw_gradient_vs_finite_differences():
    rng = np.random.default_rng(8)
    parent = np.array([-1, 0, 0, 1, 1, 2])
    length = np.array([0.0, 2.0, 3.5, 1.0, 4.0, 2.5])
    d = oracle.tree_distances(parent, length)
    x, y = rng.normal(0, 3, 6), rng.normal(0, 3, 6)
    h = 1e-6
    for m in range(6):
        g = oracle.kkw_grad_hess(x, y, d, m)
        for axis, gi in ((x, 0), (y, 1)):
            axis[m] += h
            ep = oracle.kkw_energy(x, y, d)
            axis[m] -= 2 * h
            em = oracle.kkw_energy(x, y, d)
            axis[m] += h
            # g is half the gradient
            assert abs((ep - em) / (2 * h) / 2 - g[gi]) <= 1e-5 * (1 + abs(g[gi]))


def test_kkw_weighted_path_is_realised_exactly():
    parent = np.array([-1, 0, 1, 2])
    length = np.array([0.0, 2.0, 3.0, 0.5])
    d = oracle.tree_distances(parent, length)
    x, y = oracle.init_positions(4, np.arange(4))
    x, y, e = oracle.kkw_run(x * 3, y * 3, d, length[1:].mean(), 300)
    assert e[-1] <= 1e-18 + 1e-12 * e[0]
    assert e[-1] == oracle.kkw_energy(x, y, d)             # the trace is the energy after each sweep
    r = np.hypot(x[:, None] - x[None], y[:, None] - y[None])
    assert np.allclose(r, d, rtol=1e-6, atol=1e-8)


def _forest_layout(seed, n_comp, lo, hi):
    sizes, u, v = synth.forest(seed, n_comp, lo, hi)
    g = oracle.graph_from_edges(int(sizes.sum()), u, v)
    label, _ = oracle.components(g.off, g.adj)
    comp_off, _, nodes = oracle.component_order(label)
    xy = np.random.default_rng(seed).normal(0, 5, (g.n_nodes, 2))
    return g, comp_off, nodes, xy


def test_assembly_keeps_component_shapes_at_unit_mean_edge():
    g, comp_off, nodes, xy = _forest_layout(31, 40, 1.0, 25.0)
    out = oracle.assemble(g.off, g.adj, comp_off, nodes, xy, K=8, sweeps=50)
    for c in range(len(comp_off) - 1):
        vs = nodes[comp_off[c]:comp_off[c + 1]]
        # a translation of the rescaled component: differences scale exactly
        diff_in = xy[vs] - xy[vs[0]]
        diff_out = out["xy"][vs] - out["xy"][vs[0]]
        assert np.allclose(diff_out, diff_in * out["scale"][c], rtol=1e-9, atol=1e-9)
        lens = [np.hypot(*(out["xy"][a] - out["xy"][b])) for a in vs for b in g.adj[g.off[a]:g.off[a + 1]] if b > a]
        if lens:
            assert abs(np.mean(lens) - 1.0) <= 1e-12
    # the order is a permutation sorted by the keys
    keys = oracle.meta_keys(0, len(comp_off) - 1)
    order = np.argsort(out["rank"])
    assert sorted(out["rank"].tolist()) == list(range(len(comp_off) - 1))
    assert np.all(np.diff(keys[order].astype(np.float64)) >= 0)
    assert len(out["levels"]) >= 2           # 40 components in chunks of 8: more than one level


def test_assembly_of_two_components_places_them_at_the_edge_length():
    # two components: one meta-edge, KK on two nodes reaches its length exactly
    u = np.array([0, 1, 3, 4, 5]); v = np.array([1, 2, 4, 5, 3])
    g = oracle.graph_from_edges(6, u, v)
    label, _ = oracle.components(g.off, g.adj)
    comp_off, _, nodes = oracle.component_order(label)
    xy = np.random.default_rng(2).normal(0, 1, (6, 2))
    out = oracle.assemble(g.off, g.adj, comp_off, nodes, xy, K=50, sweeps=100)
    cen = [out["xy"][nodes[comp_off[c]:comp_off[c + 1]]].mean(0) for c in range(2)]
    want = out["radius"][0] + out["radius"][1] + oracle.KAPPA
    assert abs(np.hypot(*(cen[0] - cen[1])) - want) <= 1e-9 * want


def test_khop_vs_scipy_distances():
    sp = pytest.importorskip("scipy.sparse.csgraph")
    from scipy.sparse import csr_matrix
    tx = synth.tx_lists(**synth.C1)
    g = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    a = csr_matrix((np.ones(len(g.adj)), g.adj, g.off), shape=(g.n_nodes, g.n_nodes))
    rng = np.random.default_rng(1)
    for seed in rng.choice(g.n_nodes, 5, replace=False):
        dist = sp.shortest_path(a, unweighted=True, indices=int(seed))
        for k in (0, 1, 2, 3):
            ids, edges = oracle.khop(g.off, g.adj, int(seed), k)
            assert np.array_equal(ids, np.flatnonzero(dist <= k))
            inside = set(ids.tolist())
            m = sum(1 for x in ids for w in g.adj[g.off[x]:g.off[x + 1]] if int(w) in inside and int(w) != int(x)) // 2
            assert len(edges) == m
