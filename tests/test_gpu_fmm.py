"""GPU parity of the Fast Multipole repulsion (Section 3.2.1).

The FMM approximates the exact all-pairs repulsion; its reference is the
oracle's FP64 exact sum (and the GPU's FP32 exact sum for whole-component
RMS errors).  Error measure per node:
  e_i = |F_fmm(i) - F_exact(i)| / (kr m_i sum_j m_j / |p_i - p_j|),
bounded by the truncation ceiling 2 (1 + rho) rho^(p+1) / (1 - rho) of the
interaction-list geometry, rho = sqrt(2) / (4 - sqrt(2)) (well-separated
boxes are at least two box widths apart), and never asked to beat the
FP32 floor of the direct sum."""
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


class Path:
    """A path graph on n nodes: one component whose local order is the id order."""

    def __init__(self, ctx, n):
        bgl = _bgl()
        self.n = n
        self.g = bgl.Graph.from_edges(ctx, n, np.arange(n - 1), np.arange(1, n))
        self.g.components(labels=False)
        self.og = oracle.graph_from_edges(n, np.arange(n - 1), np.arange(1, n))
        self.mass = np.diff(self.og.off) + 1.0


@pytest.fixture(scope="module")
def path30k(ctx):
    return Path(ctx, 30000)


def _errors(fmm, exact, xy, pth, sample, kr=1.0):
    o = oracle.fa2_forces(xy[:, 0], xy[:, 1], pth.mass, pth.og.off, pth.og.adj, kr, 1.0, targets=sample)
    e = np.hypot(*(fmm[sample] - o["frep"]).T) / o["srep"]
    rms = np.sqrt(np.mean(np.sum((fmm - exact) ** 2, 1)) / np.mean(np.sum(exact ** 2, 1)))
    return e, rms


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_fmm_error_within_ceiling_and_decreasing(path30k, kind):
    bgl = _bgl()
    xy = synth.points(7, path30k.n, kind, scale=50.0)
    exact = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy)
    sample = np.random.default_rng(1).choice(path30k.n, 400, replace=False)
    prev = None
    for p in (4, 8, 12, 16, 24):
        f = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=p), xy)
        e, rms = _errors(f, exact, xy, path30k, sample)
        assert np.all(np.isfinite(f))
        assert e.max() <= ceiling(p), (kind, p, e.max(), ceiling(p))
        if prev is not None and p <= 16:
            assert rms < prev, (kind, p, rms, prev)          # geometric decrease in p
        prev = rms
    assert rms <= 1e-5, rms                                   # p = 24 reaches the FP32 direct-sum level


@pytest.mark.parametrize("p", [8, 16])
def test_fmm_force_sum_vanishes(path30k, p):
    """The exact repulsion is antisymmetric, so its sum over the component is
    0; the FMM's residual |sum_i F(i)| / sum_i |F(i)| stays within its error
    ceiling (and the exact sum's own residual is at the FP32 level)."""
    bgl = _bgl()
    xy = synth.points(9, path30k.n, "clustered", scale=30.0)
    exact = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy).astype(np.float64)
    f = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=p), xy).astype(np.float64)
    res = np.hypot(*f.sum(0)) / np.sum(np.hypot(*f.T))
    res_exact = np.hypot(*exact.sum(0)) / np.sum(np.hypot(*exact.T))
    assert res_exact <= 1e-5, res_exact
    assert res <= ceiling(p), (p, res)


def test_fmm_is_bitwise_reproducible(path30k):
    bgl = _bgl()
    xy = synth.points(3, path30k.n, "clustered", scale=10.0)
    p = bgl.params(repulsion=bgl.REP_FMM, fmm_p=8)
    a = path30k.g.fa2_repulsion(0, p, xy)
    b = path30k.g.fa2_repulsion(0, p, xy)
    assert np.array_equal(a, b)


def test_fmm_sort_passes_follow_tree_depth(path30k):
    """When a tree is at most 8 levels deep, the next evaluation of the same
    plan sorts the Morton keys on their top 16 bits only (two radix passes
    skipped): the tree is the same, only the order of points inside a leaf
    differs, so the forces agree to rounding.  Deeper trees keep the full
    sort, and then repeated evaluations are bitwise equal."""
    bgl = _bgl()
    p = bgl.params(repulsion=bgl.REP_FMM, fmm_p=8)
    shallow = path30k.g.fmm_stats(0, p, synth.points(7, path30k.n, "uniform", scale=50.0), reps=2)
    assert shallow["depth"] <= 8 and shallow["sort_skip"] == 2
    assert shallow["sortmode_rel_diff"] <= 1e-5
    deep = path30k.g.fmm_stats(0, p, synth.points(5, path30k.n, "clustered", scale=20.0), reps=2)
    assert deep["depth"] > 8 and deep["sort_skip"] == 0
    assert deep["sortmode_rel_diff"] == 0.0


def test_fmm_device_loop_equals_host_loop_across_tree_depths(path30k, monkeypatch):
    """In the device-side loop the sort's two low radix passes sit under a
    graph IF node whose condition the keys kernel sets from the sort-pass
    skip; the host loop launches them and they return at once.  From a
    clustered start (trees deeper than 8 levels: the full sort) and a uniform
    one (shallow trees: two passes skipped after the first evaluation) the
    positions and statistics of both loops are bitwise the same."""
    bgl = _bgl()
    p = bgl.params(repulsion=bgl.REP_FMM, fmm_p=8)
    for xy in (synth.points(5, path30k.n, "clustered", scale=20.0), synth.points(7, path30k.n, "uniform", scale=50.0)):
        monkeypatch.delenv("BGL_HOST_LOOP", raising=False)
        a, sa = path30k.g.fa2_step(0, p, 6, xy)
        monkeypatch.setenv("BGL_HOST_LOOP", "1")
        b, sb = path30k.g.fa2_step(0, p, 6, xy)
        monkeypatch.delenv("BGL_HOST_LOOP", raising=False)
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b) and np.array_equal(sa, sb)


def test_fmm_small_leaf_sizes(path30k):
    bgl = _bgl()
    xy = synth.points(5, path30k.n, "clustered", scale=20.0)
    exact = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy)
    sample = np.random.default_rng(2).choice(path30k.n, 200, replace=False)
    for leaf in (1, 7, 32, 200):
        f = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=12, leaf_size=leaf), xy)
        e, _ = _errors(f, exact, xy, path30k, sample)
        assert e.max() <= ceiling(12), (leaf, e.max())


def test_fmm_long_w_lists(path30k):
    """Coarse leaves next to a finely divided cluster get long W lists (more
    than the 16 entries the far-field kernel stages); their M2P runs in the
    heavy-leaf kernel, sixteen warps per leaf.  The forces of those leaves'
    points stay within the error ceiling, at p = 8 and p = 16."""
    bgl = _bgl()
    rng = np.random.default_rng(12)
    n = path30k.n
    xy = np.empty((n, 2), np.float32)
    xy[:2000] = rng.uniform(0, 100, (2000, 2))                 # sparse: coarse leaves
    xy[2000:] = 50.0 + rng.uniform(0, 1, (n - 2000, 2))          # dense: deep subdivision
    exact = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy)
    sample = np.concatenate([rng.choice(2000, 250, replace=False), 2000 + rng.choice(n - 2000, 50, replace=False)])
    for p in (8, 16):
        prm = bgl.params(repulsion=bgl.REP_FMM, fmm_p=p)
        st = path30k.g.fmm_stats(0, prm, xy, reps=1)
        assert st["w_heavy"] > 0, st
        f = path30k.g.fa2_repulsion(0, prm, xy)
        e, _ = _errors(f, exact, xy, path30k, sample)
        assert e.max() <= ceiling(p), (p, e.max(), ceiling(p))


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_fmm_bf16_m2l_error(path30k, kind):
    """M2L translations in BF16 on the tensor cores (FP32 accumulate, every
    source expansion scaled by its largest component before rounding).  BF16
    keeps 8 significant bits, unit roundoff u = 2^-8; the translated
    expansion of one V entry then carries a relative error of a few u, which
    bounds the far-field part of each force: RMS over the component at most
    1e-2 and the per-node error (in units of the node's total repulsion
    scale) at most 5e-2.  The result differs from the FP32 M2L, is never
    more accurate than it, and is bitwise reproducible (each entry's
    translation and each box's sum in list order are fixed)."""
    bgl = _bgl()
    xy = synth.points(11, path30k.n, kind, scale=50.0)
    exact = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy)
    sample = np.random.default_rng(4).choice(path30k.n, 300, replace=False)
    f32 = path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=12), xy)
    p16 = bgl.params(repulsion=bgl.REP_FMM, fmm_p=12, m2l_bf16=1)
    f16 = path30k.g.fa2_repulsion(0, p16, xy)
    assert np.all(np.isfinite(f16))
    assert not np.array_equal(f16, f32)
    e16, r16 = _errors(f16, exact, xy, path30k, sample)
    _, r32 = _errors(f32, exact, xy, path30k, sample)
    assert r16 <= 1e-2, (kind, r16)
    assert e16.max() <= 5e-2, (kind, e16.max())
    assert r16 >= r32, (kind, r16, r32)
    assert np.array_equal(f16, path30k.g.fa2_repulsion(0, p16, xy))
    with pytest.raises(RuntimeError):
        path30k.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=16, m2l_bf16=1), xy)


@pytest.mark.parametrize("case", ["tiny", "coincident", "collinear", "far_clusters", "wide_range", "edge_line"])
def test_fmm_degenerate_geometries(ctx, case):
    bgl = _bgl()
    rng = np.random.default_rng(11)
    if case == "tiny":
        n = 40                                   # one leaf: pure P2P
        xy = rng.uniform(-1, 1, (n, 2))
    elif case == "coincident":
        n = 3000                                 # every point at the same place: no force
        xy = np.tile([[0.25, -3.0]], (n, 1))
    elif case == "collinear":
        n = 5000
        xy = np.stack([rng.uniform(-10, 10, n), np.full(n, 2.0)], 1)
    elif case == "far_clusters":
        n = 6000                                 # deep tree around two tight clusters
        xy = np.concatenate([rng.normal(0, 1e-3, (n // 2, 2)), rng.normal(0, 1e-3, (n // 2, 2)) + [100.0, 40.0]])
    elif case == "edge_line":
        # two coarse leaves (the left half of the root) against a line of
        # 40,000 points just right of the midline, refined to ~1,000 leaves:
        # each coarse leaf touches over 500 fine ones (long U and W lists)
        left = np.stack([rng.uniform(0.05, 0.45, 20), rng.uniform(0.0, 1.0, 20)], 1)
        line = np.stack([np.full(40000, 0.5001), rng.uniform(0.0, 1.0, 40000)], 1)
        xy = np.concatenate([[[0.0, 0.0], [1.0, 1.0]], left, line])
        n = len(xy)
    else:
        n = 6000                                 # scales from 1e-3 to 1e3
        r = 10 ** rng.uniform(-3, 3, n)
        t = rng.uniform(0, 2 * np.pi, n)
        xy = np.stack([r * np.cos(t), r * np.sin(t)], 1)
    xy = xy.astype(np.float32)
    pth = Path(ctx, n)
    exact = pth.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy)
    f = pth.g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=16), xy)
    assert np.all(np.isfinite(f))
    if case == "coincident":
        assert np.all(f == 0) and np.all(exact == 0)
        return
    sample = np.arange(n) if n <= 500 else np.random.default_rng(3).choice(n, 300, replace=False)
    e, _ = _errors(f, exact, xy, pth, sample)
    assert e.max() <= ceiling(16), (case, e.max())
    pth.g.destroy()


def test_fmm_forces_c2_giant(ctx):
    """The full-size giant component: FMM against the GPU exact sum on every
    node and against the oracle on 2000 sampled nodes."""
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
    xy = np.stack([x, y], 1).astype(np.float32) * 300.0
    exact = g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_EXACT), xy)
    sample = np.random.default_rng(2).choice(len(vs), 2000, replace=False)
    o = oracle.fa2_forces(xy[:, 0], xy[:, 1], mass, loff, ladj, 1.0, 1.0, targets=sample)
    for p in (8, 16):
        f = g.fa2_repulsion(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=p), xy)
        e = np.hypot(*(f[sample] - o["frep"]).T) / o["srep"]
        rms = np.sqrt(np.mean(np.sum((f - exact) ** 2, 1)) / np.mean(np.sum(exact ** 2, 1)))
        assert e.max() <= ceiling(p), (p, e.max())
        assert rms <= ceiling(p), (p, rms)
    g.destroy()


def test_fmm_fa2_iterations_track_exact(ctx):
    """Two ForceAtlas2 iterations with FMM repulsion (p = 16) stay with the
    exact-repulsion iterations on the C1 giant component."""
    bgl = _bgl()
    tx = synth.tx_lists(**synth.C1)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    vs = nodes[coff[0]:coff[1]]
    x, y = oracle.init_positions(0, vs)
    xy = np.stack([x, y], 1).astype(np.float32)
    a, sa = g.fa2_step(0, bgl.params(repulsion=bgl.REP_EXACT), 2, xy)
    b, sb = g.fa2_step(0, bgl.params(repulsion=bgl.REP_FMM, fmm_p=16, leaf_size=32), 2, xy)
    diag = math.hypot(np.ptp(a[:, 0]), np.ptp(a[:, 1]))
    assert np.max(np.hypot(*(a - b).T)) <= 1e-3 * diag
    assert np.allclose(sa, sb, rtol=1e-3)
    g.destroy()
