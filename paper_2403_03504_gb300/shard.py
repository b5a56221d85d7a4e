"""Components of one graph laid out on several GPUs (Section 4: every
connected component is laid out on its own).

The components are split among the ranks of a job by longest-processing-time
bin packing on an estimated cost, each rank lays out its share, and the
coordinates are gathered on the host.  A rank lays out its share on a graph
with every node id of the whole graph but only the edges of its own
components: a component's layout depends only on its node ids (initial
positions are drawn per id), its adjacency and the parameters, so each one
comes out exactly as in a one-rank layout, while the nodes of the other
components are isolated nodes that sit at the origin at no cost.  Nothing is
exchanged while the layouts run; the gather of the coordinates is the only
collective.

Cost model (work units per component of n nodes):
  Kamada-Kawai (2 <= n <= kk_max_nodes)   n^2 * kk_sweeps      (pairs per sweep)
  ForceAtlas2, exact repulsion            n^2 * fa2_iters      (pairs per iteration)
  ForceAtlas2, FMM repulsion              FMM_PAIRS_PER_NODE * n * fa2_iters
                                          (near-field pairs per target, about
                                           nine leaves of ~40 points)
  single nodes                            0
"""
from __future__ import annotations

import numpy as np

FMM_PAIRS_PER_NODE = 400.0
REP_EXACT, REP_FMM, REP_AUTO = 0, 1, 2


def component_costs(sizes, kk_max_nodes=50, fa2_iters=50, kk_sweeps=200, repulsion=REP_AUTO,
                    fmm_min_nodes=8192) -> np.ndarray:
    """Estimated work of each component (sizes in component order)."""
    n = np.asarray(sizes, np.float64)
    cost = np.zeros_like(n)
    kk = (n >= 2) & (n <= kk_max_nodes)
    cost[kk] = n[kk] ** 2 * kk_sweeps
    fa2 = n > kk_max_nodes
    if repulsion == REP_FMM:
        fmm = fa2
    elif repulsion == REP_EXACT:
        fmm = np.zeros_like(fa2)
    else:
        fmm = fa2 & (n >= fmm_min_nodes)
    exact = fa2 & ~fmm
    cost[exact] = n[exact] ** 2 * fa2_iters
    cost[fmm] = FMM_PAIRS_PER_NODE * n[fmm] * fa2_iters
    return cost


def lpt_assign(costs, world: int):
    """Longest processing time first: items by cost descending (ties by
    index) go one by one to the least-loaded rank (ties to the lowest rank).
    Returns (rank of each item, load of each rank).  The largest load is at
    most (4/3 - 1/(3 world)) times the best possible (Graham, 1969)."""
    costs = np.asarray(costs, np.float64)
    owner = np.zeros(len(costs), np.int32)
    load = np.zeros(world, np.float64)
    for i in np.lexsort((np.arange(len(costs)), -costs)):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return owner, load


def node_owner(comp_off, nodes, comp_owner, n_nodes) -> np.ndarray:
    """Rank of every node: the rank of its component."""
    own = np.empty(n_nodes, np.int32)
    sizes = np.diff(np.asarray(comp_off))
    own[np.asarray(nodes)] = np.repeat(np.asarray(comp_owner, np.int32), sizes)
    return own


def share_edges(src, dst, owner_of_node, rank: int):
    """The directed edges of the rank's components (both ends in one component)."""
    src = np.asarray(src)
    dst = np.asarray(dst)
    keep = owner_of_node[src] == rank
    return src[keep], dst[keep]


def merge(n_nodes: int, pieces) -> np.ndarray:
    """Coordinates of the whole graph from (node ids, xy) pieces, one per rank."""
    xy = np.zeros((n_nodes, 2), np.float32)
    seen = np.zeros(n_nodes, bool)
    for ids, part in pieces:
        ids = np.asarray(ids)
        if np.any(seen[ids]):
            raise ValueError("a node was laid out by two ranks")
        seen[ids] = True
        xy[ids] = part
    return xy


def layout_sharded(n_nodes, src, dst, comp_off, nodes, costs, rank: int, world: int, layout_fn, dist=None):
    """Lays out this rank's share and gathers every rank's coordinates.

    layout_fn(n_nodes, src, dst) -> xy[n_nodes, 2] lays out the graph on all
    n_nodes ids with the given directed edges.  With a process group `dist`
    the pieces are exchanged by all_gather_object, and every rank returns
    the merged coordinates; without one (world ranks run one after another
    in this process) the caller merges the pieces.  Returns (merged xy or
    None, this rank's piece, the assignment of components to ranks)."""
    comp_owner, _ = lpt_assign(costs, world)
    own = node_owner(comp_off, nodes, comp_owner, n_nodes)
    s, d = share_edges(src, dst, own, rank)
    xy = np.asarray(layout_fn(n_nodes, s, d), np.float32)
    ids = np.flatnonzero(own == rank)
    piece = (ids, xy[ids])
    if dist is None:
        return None, piece, comp_owner
    pieces = [None] * world
    dist.all_gather_object(pieces, piece)
    return merge(n_nodes, pieces), piece, comp_owner
