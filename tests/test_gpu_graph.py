"""GPU parity of graph construction (Section 2), components and the size
split (Section 4): bit-exact against the oracle and the hand-worked cases."""
import json
import os

import numpy as np
import pytest

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


def _check_graph(g, og):
    s = g.sizes()
    assert s["n_nodes"] == og.n_nodes
    assert s["n_addr"] == len(og.addr)
    assert np.array_equal(g.addresses(), og.addr)
    src, dst = g.edges()
    assert np.array_equal(src, og.src) and np.array_equal(dst, og.dst)
    off, adj = g.csr()
    assert np.array_equal(off, og.off) and np.array_equal(adj, og.adj)
    assert np.array_equal(g.degrees(), og.deg)
    lab, nc = g.components()
    olab, onc = oracle.components(og.off, og.adj)
    assert nc == onc and np.array_equal(lab, olab)
    coff, clab, nodes = g.component_nodes()
    ooff, olabc, onodes = oracle.component_order(olab)
    assert np.array_equal(coff, ooff) and np.array_equal(clab, olabc) and np.array_equal(nodes, onodes)


def _tx_case(case):
    keys = {nm: (1 << 63) - 7919 * (ord(nm) * 104729 % 1009) for nm in
            sorted({a for t in case["tx"] for a in t["in"] + t["out"]})}
    in_off, out_off, ia, oa = [0], [0], [], []
    for t in case["tx"]:
        ia += [keys[a] for a in t["in"]]
        oa += [keys[a] for a in t["out"]]
        in_off.append(len(ia))
        out_off.append(len(oa))
    return np.array(in_off), np.array(ia, np.uint64), np.array(out_off), np.array(oa, np.uint64)


@pytest.mark.parametrize("idx", [0, 1])
def test_golden_tx_graphs(ctx, idx):
    bgl = _bgl()
    case = json.load(open(os.path.join(GOLDEN, "txgraph_small.json")))["cases"][idx]
    io, ia, oo, oa = _tx_case(case)
    g = bgl.Graph.build(ctx, io, ia, oo, oa)
    src, dst = g.edges()
    assert np.stack([src, dst], 1).tolist() == case["edges"]
    assert g.degrees().tolist() == case["deg"]
    lab, nc = g.components()
    assert lab.tolist() == case["label"]
    coff, _, nodes = g.component_nodes()
    assert [nodes[coff[c]:coff[c + 1]].tolist() for c in range(nc)] == case["comp_nodes"]
    _check_graph(g, oracle.graph_build(io, ia, oo, oa))
    g.destroy()


@pytest.mark.parametrize("cfg", ["C1", "C2"])
def test_tx_graph_bit_exact(ctx, cfg):
    bgl = _bgl()
    tx = synth.tx_lists(**getattr(synth, cfg))
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    g = bgl.Graph.build(ctx, tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    _check_graph(g, og)
    n_kk, n_fa2 = g.split(50)
    sizes = np.diff(g.component_nodes()[0])
    assert n_fa2 == int((sizes > 50).sum()) and n_kk == int((sizes <= 50).sum())
    g.destroy()


def test_build_from_device_arrays_matches_host(ctx):
    bgl = _bgl()
    import torch
    tx = synth.tx_lists(**synth.C1)
    dev = torch.device("cuda", 0)
    t = [torch.from_numpy(a).to(dev) for a in (tx.in_off, tx.in_addr.view(np.int64), tx.out_off,
                                               tx.out_addr.view(np.int64))]
    torch.cuda.synchronize()
    g = bgl.Graph.build_dev(ctx, tx.n_tx, len(tx.in_addr), len(tx.out_addr), *t)
    og = oracle.graph_build(tx.in_off, tx.in_addr, tx.out_off, tx.out_addr)
    _check_graph(g, og)
    g.destroy()
    # inconsistent sizes are caught on the device
    with pytest.raises(bgl.BglError) as e:
        bgl.Graph.build_dev(ctx, tx.n_tx, len(tx.in_addr) + 1, len(tx.out_addr), *t)
    assert e.value.status == -1


def test_edge_list_graph_with_duplicates_and_self_loops(ctx):
    bgl = _bgl()
    sizes, u, v = synth.forest(7, 500, 1.0, 200.0)
    n = int(sizes.sum())
    u = np.concatenate([u, u[:50], [3, 3]]).astype(np.int32)       # duplicates and a self-loop
    v = np.concatenate([v, v[:50], [3, 3]]).astype(np.int32)
    g = bgl.Graph.from_edges(ctx, n, u, v)
    og = oracle.graph_from_edges(n, u, v)
    _check_graph(g, og)
    lab, nc = g.components()
    assert nc == len(sizes)
    g.destroy()


def test_empty_and_degenerate_inputs(ctx):
    bgl = _bgl()
    g = bgl.Graph.build(ctx, [0], np.zeros(0, np.uint64), [0], np.zeros(0, np.uint64))
    assert g.sizes()["n_nodes"] == 0
    assert g.components(labels=False) == 0
    assert g.layout().shape == (0, 2)
    g.destroy()
    # transactions without endpoints are isolated nodes
    g = bgl.Graph.build(ctx, [0, 0, 0], np.zeros(0, np.uint64), [0, 0, 0], np.zeros(0, np.uint64))
    lab, nc = g.components()
    assert nc == 2 and lab.tolist() == [0, 1]
    assert np.all(g.layout() == 0)
    g.destroy()
    with pytest.raises(bgl.BglError) as e:
        bgl.Graph.build(ctx, [0, 2, 1], np.zeros(2, np.uint64), [0, 0, 0], np.zeros(0, np.uint64))
    assert e.value.status == -1
    with pytest.raises(bgl.BglError) as e:
        bgl.Graph.from_edges(ctx, 3, [0, 5], [1, 2])
    assert e.value.status == -1
    g = bgl.Graph.from_edges(ctx, 4, [0], [1])
    with pytest.raises(bgl.BglError) as e:
        g.layout()
    assert e.value.status == -6          # components not labelled yet
    g.destroy()
