"""The allocation-free ForceAtlas2 iteration (bgl_fa2_iteration_noalloc).

Callers whose device memory is all reserved by their own pool, or that
cannot take the synchronisation of cudaMalloc/cudaFree in their loop, run
ForceAtlas2 iterations through this entry point: they pass every array, and
the reduction scratch sits in a fixed static device array.  This test calls
it twice in a row through the C ABI on the 1,000-transaction graph's giant
component and checks each result against the allocating entry point
bgl_fa2_step with the same number of iterations, at the tolerance of the
other ForceAtlas2 trajectory tests (positions within 1e-3 of the layout's
bounding-box diagonal, speeds within 1e-4)."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_iterations_match_fa2_step():
    import torch
    import paper_2403_03504_gb300 as bgl

    ctx = bgl.Context(0)
    tx = synth.tx_lists(**synth.C1)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g.components(labels=False)
    coff, _, nodes = g.component_nodes()
    off, adj = g.csr()
    vs = nodes[coff[0]:coff[1]]
    n = len(vs)
    pos = np.full(len(off) - 1, -1, np.int64)
    pos[vs] = np.arange(n)
    loff = np.zeros(n + 1, np.int64)
    loff[1:] = np.cumsum(np.diff(off)[vs])
    ladj = pos[np.concatenate([adj[off[v]:off[v + 1]] for v in vs])].astype(np.int32)
    mass = (np.diff(loff) + 1).astype(np.float32)
    xy0 = np.random.default_rng(4).uniform(-1, 1, (n, 2)).astype(np.float32)
    p = bgl.params(repulsion=bgl.REP_EXACT)

    dev = torch.device("cuda", 0)
    d_off = torch.from_numpy(loff).to(dev)
    d_adj = torch.from_numpy(ladj).to(dev)
    d_mass = torch.from_numpy(mass).to(dev)
    d_xy = torch.from_numpy(xy0.copy()).to(dev)
    d_fprev = torch.zeros((n, 2), dtype=torch.float32, device=dev)
    d_f = torch.zeros((n, 2), dtype=torch.float32, device=dev)
    d_sg = torch.ones(1, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    for it in (1, 2):
        ctx.fa2_iteration_noalloc(n, d_off, d_adj, d_mass, d_xy, d_fprev, d_f, d_sg, p)
        ctx.sync()
        got = d_xy.cpu().numpy()
        want, stats = g.fa2_step(0, p, it, xy0)
        diag = math.hypot(np.ptp(want[:, 0]), np.ptp(want[:, 1]))
        err = float(np.max(np.hypot(*(got - want).T)))
        assert err <= 1e-3 * diag, (it, err, diag)
        assert float(d_sg.cpu()[0]) == pytest.approx(stats[-1, 2], rel=1e-4)

    # sizes above the static scratch capacity are refused without touching the device
    with pytest.raises(bgl.BglError) as e:
        ctx.fa2_iteration_noalloc((1 << 20) + 1, d_off, d_adj, d_mass, d_xy, d_fprev, d_f, d_sg, p)
    assert e.value.status == -1
    g.destroy()
    ctx.close()
