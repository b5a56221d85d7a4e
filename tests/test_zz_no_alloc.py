"""The allocation-free ForceAtlas2 iteration (bgl_fa2_iteration_noalloc).

Callers whose device memory is all reserved by their own pool, or that
cannot take the synchronisation of cudaMalloc/cudaFree in their loop, run
ForceAtlas2 iterations through this entry point: they pass every array, and
the reduction scratch sits in a fixed static device array.  These tests call
it through the C ABI, two calls in a row, and check each result against the
allocating entry point bgl_fa2_step with the same number of iterations and
against the FP64 oracle, at the tolerance of the other ForceAtlas2 trajectory
tests (positions within 1e-3 of the layout's bounding-box diagonal, s_G
within 1e-4): on the 1,000-transaction graph's giant component (two
reduction tiles) and on a 5,000-node component (a partial last tile), with
both swing/traction variants; at the size limit (2^20 nodes, every tile of
the scratch in use) against an FP64 recomputation of the sums; and with a
non-finite position, which bgl_ctx_sync reports."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _local(g, c):
    coff, _, nodes = g.component_nodes()
    off, adj = g.csr()
    vs = nodes[coff[c]:coff[c + 1]]
    n = len(vs)
    pos = np.full(len(off) - 1, -1, np.int64)
    pos[vs] = np.arange(n)
    loff = np.zeros(n + 1, np.int64)
    loff[1:] = np.cumsum(np.diff(off)[vs])
    ladj = pos[np.concatenate([adj[off[v]:off[v + 1]] for v in vs])].astype(np.int32)
    return n, loff, ladj


def _graph(ctx, which):
    import paper_2403_03504_gb300 as bgl
    if which == "c1-giant":
        tx = synth.tx_lists(**synth.C1)
        return bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    sizes, u, v = synth.forest(71, 1, 5000.0, 5000.0)
    return bgl.Graph.from_edges(ctx, int(sizes.sum()), u, v)


class _Dev:
    """Caller-owned device arrays of one component."""

    def __init__(self, loff, ladj, xy0):
        import torch
        dev = torch.device("cuda", 0)
        n = len(loff) - 1
        self.n = n
        self.off = torch.from_numpy(loff).to(dev)
        self.adj = torch.from_numpy(ladj).to(dev)
        self.mass = torch.from_numpy((np.diff(loff) + 1).astype(np.float32)).to(dev)
        self.xy = torch.from_numpy(xy0.copy()).to(dev)
        self.fprev = torch.zeros((n, 2), dtype=torch.float32, device=dev)
        self.f = torch.zeros((n, 2), dtype=torch.float32, device=dev)
        self.sg = torch.ones(1, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()

    def step(self, ctx, p):
        ctx.fa2_iteration_noalloc(self.n, self.off, self.adj, self.mass, self.xy, self.fprev, self.f, self.sg, p)


@pytest.mark.parametrize("which", ["c1-giant", "forest-5000"])
@pytest.mark.parametrize("variant", [0, 1])
def test_noalloc_iterations_match_fa2_step_and_oracle(which, variant):
    import paper_2403_03504_gb300 as bgl

    ctx = bgl.Context(0)
    g = _graph(ctx, which)
    g.components(labels=False)
    n, loff, ladj = _local(g, 0)
    assert n > 2048 and n % 2048 != 0          # several reduction tiles, the last one partial
    xy0 = np.random.default_rng(4).uniform(-1, 1, (n, 2)).astype(np.float32)
    p = bgl.params(repulsion=bgl.REP_EXACT, swing_variant=variant)
    d = _Dev(loff, ladj, xy0)
    mass = np.diff(loff) + 1.0
    for it in (1, 2):
        d.step(ctx, p)
        ctx.sync()
        got = d.xy.cpu().numpy()
        sg = float(d.sg.cpu()[0])
        want, stats = g.fa2_step(0, p, it, xy0)
        st, ostats = oracle.fa2_run(xy0[:, 0].astype(np.float64), xy0[:, 1].astype(np.float64), mass, loff, ladj,
                                    it, variant=variant)
        for ref, ref_sg in ((want, stats[-1, 2]), (np.stack([st.x, st.y], 1), ostats[-1, 2])):
            diag = math.hypot(np.ptp(ref[:, 0]), np.ptp(ref[:, 1]))
            err = float(np.max(np.hypot(*(got - ref).T)))
            assert err <= 1e-3 * diag, (which, variant, it, err, diag)
            assert sg == pytest.approx(ref_sg, rel=1e-4), (which, variant, it)
    g.destroy()
    ctx.close()


def test_noalloc_at_the_size_limit():
    """n = 2^20 (a path): all 512 tiles of the scratch hold partial sums;
    s_G of the second call equals the FP64 sums of the GPU's own forces."""
    import paper_2403_03504_gb300 as bgl

    n = 1 << 20
    loff = np.zeros(n + 1, np.int64)
    deg = np.full(n, 2, np.int64)
    deg[0] = deg[-1] = 1
    loff[1:] = np.cumsum(deg)
    ladj = np.empty(loff[-1], np.int32)
    ladj[loff[:-1][1:] - 0] = np.arange(0, n - 1)            # left neighbour of nodes 1..n-1
    ladj[loff[1:][:-1] - 1] = np.arange(1, n)                # right neighbour of nodes 0..n-2
    xy0 = np.random.default_rng(7).uniform(-1, 1, (n, 2)).astype(np.float32)
    ctx = bgl.Context(0)
    d = _Dev(loff, ladj, xy0)
    p = bgl.params(repulsion=bgl.REP_EXACT)
    d.step(ctx, p)
    ctx.sync()
    f1 = d.f.cpu().numpy().astype(np.float64)
    assert float(d.sg.cpu()[0]) == 1.0                      # swg = trc when F_{-1} = 0
    d.step(ctx, p)
    ctx.sync()
    f2 = d.f.cpu().numpy().astype(np.float64)
    swg = np.sum(np.hypot(*(f2 - f1).T))
    trc = np.sum(np.hypot(*(f2 + f1).T))
    assert np.all(np.isfinite(d.xy.cpu().numpy()))
    assert float(d.sg.cpu()[0]) == pytest.approx(min(trc / swg, 1.5), rel=1e-5)
    # one node more than the scratch holds is refused before any work
    with pytest.raises(bgl.BglError) as e:
        ctx.fa2_iteration_noalloc(n + 1, d.off, d.adj, d.mass, d.xy, d.fprev, d.f, d.sg, p)
    assert e.value.status == -1
    ctx.close()


def test_noalloc_non_finite_position_is_reported():
    """A NaN position spreads through the forces; bgl_ctx_sync reports it
    once (BGL_ENUMERIC) and the context stays usable."""
    import paper_2403_03504_gb300 as bgl

    ctx = bgl.Context(0)
    g = _graph(ctx, "c1-giant")
    g.components(labels=False)
    n, loff, ladj = _local(g, 0)
    xy0 = np.random.default_rng(4).uniform(-1, 1, (n, 2)).astype(np.float32)
    xy0[5, 0] = np.nan
    d = _Dev(loff, ladj, xy0)
    p = bgl.params(repulsion=bgl.REP_EXACT)
    d.step(ctx, p)
    with pytest.raises(bgl.BglError) as e:
        ctx.sync()
    assert e.value.status == -5
    ctx.sync()                                               # the record was cleared
    d2 = _Dev(loff, ladj, np.nan_to_num(xy0, nan=0.25))
    d2.step(ctx, p)
    ctx.sync()
    assert np.all(np.isfinite(d2.xy.cpu().numpy()))
    g.destroy()
    ctx.close()
