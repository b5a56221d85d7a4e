/*
 * bgl.h -- C ABI of the GB300 (sm_103a) layout library for large graphs.
 *
 * The library lays out the bipartite address/transaction graph of "Graph
 * Visualization for Blockchain Data" (Dietl et al., 2024): it builds the
 * graph from per-transaction input/output address lists (Section 2), labels
 * its connected components ignoring edge directions (Section 4), splits them
 * by node count (Section 4), lays out small components with Kamada-Kawai
 * (Section 3.1) and large ones with ForceAtlas2 whose all-pairs repulsion is
 * summed exactly or by a 2-D Fast Multipole Method (Sections 3.2, 3.2.1),
 * and returns coordinates in each component's own frame.
 *
 * Conventions shared by every call:
 *  - Every call returns a bgl_status; nothing is thrown or aborted across the
 *    ABI.  On failure the call leaves its outputs untouched where it can and
 *    bgl_last_error() describes the failure.
 *  - Pointers without a `d_` prefix are HOST memory owned by the caller;
 *    inputs are copied in, outputs must be preallocated by the caller at the
 *    sizes given by bgl_graph_sizes() / bgl_components().
 *  - Pointers with a `d_` prefix are DEVICE memory on the context's device,
 *    owned by the caller, read or written in stream order on the context's
 *    stream (bgl_ctx_set_stream).  These calls do not synchronise the
 *    stream except where stated.
 *  - Handles are opaque and owned by the library; release them with the
 *    matching destroy call.  A context is used by one host thread at a time.
 *  - Node ids: transaction t has id t (0 <= t < n_tx); an address has id
 *    n_tx + (rank of its first appearance when scanning tx 0 inputs, tx 0
 *    outputs, tx 1 inputs, tx 1 outputs, ...).
 *  - Edges (Section 2): address -> tx for every input, tx -> address for
 *    every output; exact duplicate directed edges are kept once.  The
 *    undirected graph has one edge per unordered pair {u, v} with u != v; the
 *    degree of a node is its number of distinct undirected neighbours.
 *  - Components are indexed c = 0 .. n_comp-1 by node count descending, then
 *    by label (the smallest node id in the component) ascending; the nodes
 *    of a component are listed in ascending id.  "Local" arrays of a
 *    component follow that node order.
 */
#ifndef BGL_H
#define BGL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BGL_OK = 0,
    BGL_EINVAL = -1,   /* an argument is out of range or inconsistent */
    BGL_ENOMEM = -2,   /* a device or host allocation failed */
    BGL_ECUDA = -3,    /* a CUDA runtime call failed */
    BGL_ETIMEOUT = -4, /* a bounded device-side wait gave up */
    BGL_ENUMERIC = -5, /* a non-finite position or force appeared */
    BGL_ESTATE = -6    /* the call needs a step that has not been run */
} bgl_status;

typedef struct bgl_ctx bgl_ctx;
typedef struct bgl_graph bgl_graph;

enum { BGL_REP_EXACT = 0, BGL_REP_FMM = 1, BGL_REP_AUTO = 2 };

/*
 * Parameters of the layout (defaults from bgl_params_default()).
 *  ForceAtlas2 (Section 3.2): per iteration each node feels
 *    repulsion  kr * m_i * sum_j m_j (p_i - p_j) / |p_i - p_j|^2, m = degree + 1,
 *    attraction -sum_{j adjacent} (p_i - p_j),
 *    gravity    -kg * m_i * p_i;
 *  swing and traction (Section 3.2) set the global speed
 *    s_G = min(tau * trc / swg, 1.5 * s_G) (s_G = 1 and F_{-1} = 0 at the start),
 *  and node n moves by s_n F_t(n) with
 *    s_n = ks * s_G / (1 + s_G * sqrt(|F_t(n) - F_{t-1}(n)|)), capped at ksmax / |F_t(n)|.
 *  swing_variant 0 uses the unweighted sums printed in Section 3.2;
 *  1 uses ForceAtlas2's (degree+1)-weighted sums with traction halved.
 *  Kamada-Kawai (Section 3.1): energy sum_{i<j} d_ij^-2 (|p_i - p_j| - kk_l d_ij)^2,
 *  kk_sweeps Gauss-Seidel sweeps of per-node 2x2 Newton-Raphson steps in
 *  ascending local order; kk_tol > 0 stops after a sweep whose largest
 *  gradient norm is below kk_tol.
 */
typedef struct bgl_params {
    uint64_t seed;          /* initial positions (SplitMix64 per node id)      default 0 */
    int32_t kk_max_nodes;   /* components with <= this many nodes use KK        default 50 */
    int32_t fa2_iters;      /* ForceAtlas2 iterations                           default 50 */
    double kr;              /* repulsion constant                               default 1 */
    double kg;              /* gravity constant                                 default 1 */
    double ks;              /* node speed constant                              default 0.1 */
    double ksmax;           /* largest displacement of a node per iteration     default 10 */
    double tau;             /* traction/swing tolerance                         default 1 */
    int32_t repulsion;      /* BGL_REP_EXACT, BGL_REP_FMM or BGL_REP_AUTO        default AUTO */
    int32_t fmm_p;          /* multipole expansion order, 1..24                 default 8 */
    int32_t leaf_size;      /* quadtree leaf capacity, 1..256                   default 64 */
    int32_t fmm_min_nodes;  /* AUTO uses the FMM for components at least this big  default 8192;
                               -1: by measurement (below 2048 nodes exact, from 131072 FMM, in
                               between the faster of the two, timed once per context and size
                               octave; the choice may differ between processes) */
    int32_t swing_variant;  /* 0 as printed (Section 3.2), 1 ForceAtlas2 weights default 0 */
    int32_t kk_sweeps;      /* KK sweeps                                         default 200 */
    double kk_l;            /* KK edge length l                                  default 1 */
    double kk_tol;          /* KK early-stop gradient norm, 0 = fixed sweeps     default 0 */
    int32_t assemble;       /* 1: bgl_layout assembles the component layouts into one frame
                               (Section 4, see bgl_assemble); 0: each in its own frame default 0 */
    int32_t m2l_bf16;       /* 1: FMM M2L translations in BF16 on the tensor cores (FP32
                               accumulate, per-box scaling; fmm_p <= 15)          default 0 */
} bgl_params;

/* ---------------------------------------------------------------- context */
/* The context calls are the library's own plumbing (device, stream, memory
 * pool, error text, defaults); the paper has no counterpart for them. */

/* Create a context on CUDA device `device`, with its own non-blocking
 * stream and device memory pool.  *out receives the handle. */
bgl_status bgl_ctx_create(int device, bgl_ctx **out);

/* Destroy a context (after its graphs).  NULL is ignored. */
void bgl_ctx_destroy(bgl_ctx *ctx);

/* Run all later work on `cuda_stream` (a cudaStream_t of the context's
 * device); NULL restores the context's own stream. */
bgl_status bgl_ctx_set_stream(bgl_ctx *ctx, void *cuda_stream);

/* Block until all work queued by the context has finished.  Returns
 * BGL_ENUMERIC (once) if a bgl_fa2_iteration_noalloc call on this context
 * produced a non-finite position since the last bgl_ctx_sync. */
bgl_status bgl_ctx_sync(bgl_ctx *ctx);

/* Message of the last failure on this context ("" if none).  Valid until
 * the next call on the context. */
const char *bgl_last_error(const bgl_ctx *ctx);

/* Fill *p with the defaults listed above. */
void bgl_params_default(bgl_params *p);

/* --------------------------------------------------------- graph (Section 2) */

/*
 * Build the bipartite transaction graph of Section 2 from host arrays:
 * in_off[n_tx+1] / in_addr[in_off[n_tx]] list the input addresses of each
 * transaction, out_off / out_addr the outputs (CSR form; addresses are
 * opaque 64-bit keys).  Offsets must start at 0 and never decrease
 * (BGL_EINVAL otherwise).  The graph stays on the device; *out receives it.
 */
bgl_status bgl_graph_build(bgl_ctx *ctx, int64_t n_tx, const int64_t *in_off, const uint64_t *in_addr,
                           const int64_t *out_off, const uint64_t *out_addr, bgl_graph **out);

/* As bgl_graph_build (Section 2), from device arrays; n_in = in_off[n_tx] and
 * n_out = out_off[n_tx] are passed by the caller.  Offsets are validated on
 * the device (BGL_EINVAL if inconsistent).  Synchronises the stream once. */
bgl_status bgl_graph_build_dev(bgl_ctx *ctx, int64_t n_tx, int64_t n_in, int64_t n_out,
                               const int64_t *d_in_off, const uint64_t *d_in_addr,
                               const int64_t *d_out_off, const uint64_t *d_out_addr, bgl_graph **out);

/* Graph on nodes 0..n-1 from m directed edges u[k] -> v[k] (host arrays),
 * for graphs of other domains (Section 5).  Duplicates are kept once;
 * self-loops are kept as directed edges but add no undirected neighbour.
 * There are no addresses (n_addr = 0, n_tx = 0). */
bgl_status bgl_graph_from_edges(bgl_ctx *ctx, int64_t n, int64_t m, const int32_t *u, const int32_t *v,
                                bgl_graph **out);

/* Sizes of a built graph of Section 2 (any pointer may be NULL). */
bgl_status bgl_graph_sizes(const bgl_graph *g, int64_t *n_nodes, int64_t *n_addr, int64_t *n_dir_edges,
                           int64_t *n_undir_edges);

/* Address keys in id order (the address nodes of Section 2): key_out[k] is
 * the key of node n_tx + k (n_addr entries). */
bgl_status bgl_graph_addresses(const bgl_graph *g, uint64_t *key_out);

/* Directed edges of Section 2 sorted by (src, dst): n_dir_edges entries each. */
bgl_status bgl_graph_edges(const bgl_graph *g, int32_t *src, int32_t *dst);

/* Undirected adjacency in CSR form (the graph of Section 2 with directions
 * ignored, as Sections 3 and 4 use it): off[n_nodes+1], adj[2 n_undir_edges],
 * neighbours of each node in ascending id. */
bgl_status bgl_graph_csr(const bgl_graph *g, int64_t *off, int32_t *adj);

/* deg_out[n_nodes]: number of distinct undirected neighbours (the degree
 * that sets ForceAtlas2's mass, Section 3.2). */
bgl_status bgl_degrees(const bgl_graph *g, int32_t *deg_out);

/* Release a graph and its device memory (plumbing, no counterpart in the
 * paper).  NULL is ignored. */
bgl_status bgl_graph_destroy(bgl_graph *g);

/* ------------------------------------------------- components (Section 4) */

/* Label connected components ignoring directions (Section 4).
 * label_out[n_nodes] (may be NULL) receives the smallest node id of each
 * node's component; *n_comp the number of components. */
bgl_status bgl_components(bgl_graph *g, int32_t *label_out, int64_t *n_comp);

/* Component order of Section 4's split (needs bgl_components; BGL_ESTATE
 * otherwise): comp_off[n_comp+1] node offsets,
 * comp_label[n_comp], nodes[n_nodes] node ids grouped by component.  Any
 * pointer may be NULL. */
bgl_status bgl_component_nodes(const bgl_graph *g, int64_t *comp_off, int32_t *comp_label, int32_t *nodes);

/* Size split (Section 4): components with at most kk_max_nodes nodes are
 * laid out by Kamada-Kawai, the others by ForceAtlas2.  Because components
 * are ordered by size, the ForceAtlas2 ones are c = 0 .. n_fa2-1. */
bgl_status bgl_split(bgl_graph *g, int32_t kk_max_nodes, int64_t *n_kk, int64_t *n_fa2);

/* ------------------------------------------------------ layout (Section 4) */

/*
 * Lay out every component (Section 4: Kamada-Kawai, Section 3.1, for the
 * small ones, ForceAtlas2, Section 3.2, for the rest; needs bgl_components,
 * BGL_ESTATE otherwise; runs the split with p->kk_max_nodes).  Initial positions: node id v starts at
 * (x, y) = ((h1 >> 40) 2^-24 * 2 - 1, (h2 >> 40) 2^-24 * 2 - 1), where h1, h2
 * are the first two outputs of SplitMix64 seeded with
 * p->seed XOR (v * 0x9E3779B97F4A7C15); Kamada-Kawai components scale these
 * by kk_l * diameter / 2.  Components with one node sit at the origin.
 * xy_out[2 n_nodes] (host) receives x, y of node v at [2v], [2v+1], each in
 * its component's own frame.  Synchronises the stream.
 */
bgl_status bgl_layout(bgl_graph *g, const bgl_params *p, float *xy_out);

/* As bgl_layout (Section 4), writing the device array d_xy_out[2 n_nodes]; does not
 * synchronise the stream after the last kernel. */
bgl_status bgl_layout_dev(bgl_graph *g, const bgl_params *p, float *d_xy_out);

/* ---------------------------------------- per-component parity entry points */

/* Hop distances of component c (Section 3.1): d_out[n_c * n_c], row-major in
 * local order.  Components of up to 255 nodes. */
bgl_status bgl_kk_distances(bgl_graph *g, int64_t c, int32_t *d_out);

/* Kamada-Kawai (Section 3.1) on component c (at most 255 nodes, BGL_EINVAL
 * above) from the caller's local
 * positions xy_inout[2 n_c] (x, y interleaved), p->kk_sweeps sweeps. */
bgl_status bgl_kk_run(bgl_graph *g, int64_t c, const bgl_params *p, float *xy_inout);

/* One ForceAtlas2 force evaluation (Section 3.2; repulsion by Section
 * 3.2.1's FMM when chosen) on component c at local positions
 * xy_in[2 n_c]: f_out[2 n_c] receives the total force (repulsion + attraction
 * + gravity).  p->repulsion selects the exact sum or the FMM (AUTO follows
 * p->fmm_min_nodes). */
bgl_status bgl_fa2_forces(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in, float *f_out);

/* As bgl_fa2_forces, repulsion only (Section 3.2, or 3.2.1 with the FMM). */
bgl_status bgl_fa2_repulsion(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in, float *f_out);

/* `iters` ForceAtlas2 iterations (Section 3.2) on component c from local positions
 * xy_inout[2 n_c], starting from F_{-1} = 0 and s_G = 1.  stats_out
 * (3 * iters doubles, may be NULL) receives swing, traction and s_G of every
 * iteration. */
bgl_status bgl_fa2_step(bgl_graph *g, int64_t c, const bgl_params *p, int32_t iters, float *xy_inout,
                        double *stats_out);

/* ---------------------------------------------------------------- assembly */

/*
 * Assembly of per-component layouts into one frame (Section 4): each
 * component is centred on its centroid and rescaled to mean edge length 1
 * (components without edges keep their scale); the components are put in a
 * random order (SplitMix64 key per component index, seed p->seed); in
 * consecutive runs ("pieces") of at most p->kk_max_nodes, each is linked to
 * the largest earlier one of its run (the first of equals), by an edge of
 * length r_a + r_b + 1 (r = largest distance of a node from the centroid
 * after rescaling, i.e. half the diameter); Kamada-Kawai (p->kk_sweeps
 * sweeps of Section 3.1's safeguarded Newton step, with the weighted path
 * lengths as distances, steps capped at the run's mean edge length) places
 * the run's components; each run, centred on the mean of its components'
 * centres, becomes one item of the next level, which repeats until one item
 * is left.  A node's position is its rescaled local position plus the
 * offsets of the items holding it.
 *
 * xy_in[2 n_nodes]: per-component layouts in node-id order (as bgl_layout
 * returns them); xy_out[2 n_nodes]: the assembled frame.  Optional outputs
 * (NULL to skip), per component in component order: rank_out[n_comp] its
 * place in the random order; parent_out[n_comp] (indexed by rank) the rank of
 * the component it is linked to in its run, -1 for a run's first;
 * scale_out, radius_out[n_comp]; centre_out[2 n_comp] (indexed by rank) its
 * centre in its run's Kamada-Kawai layout before centring.  Needs
 * bgl_components.  Synchronises the stream.
 */
bgl_status bgl_assemble(bgl_graph *g, const bgl_params *p, const float *xy_in, float *xy_out, int64_t *rank_out,
                        int64_t *parent_out, float *scale_out, float *radius_out, float *centre_out);

/* ----------------------------------------------------------------- serving */

/*
 * Layouts of neighbourhoods of a resident graph, served with continuous
 * batching.  The paper lays out transaction graphs "for a certain time
 * period" (Section 4); a service answers many such requests for parts of one
 * large graph.  A request (seed node, hops k) asks for the k-hop
 * neighbourhood of the seed -- every node within k undirected hops and every
 * edge among them, node ids renumbered 0..n-1 in ascending resident id --
 * laid out as bgl_layout does with the request's parameters (KK for
 * components of at most kk_max_nodes nodes, ForceAtlas2 otherwise;
 * p->assemble for one frame).
 *
 * bgl_graph_khop: the neighbourhood itself (synchronous, on g's stream):
 *   *n_nodes = its size, or -1 if it has more than max_nodes nodes (then
 *   nothing else is written); node_ids[n] (may be NULL) the resident ids in
 *   ascending order; *n_edges and u, v[m] (may be NULL) the induced edges in
 *   local ids, each once.  Call it with NULL arrays to learn the sizes.
 * bgl_server_create: `slots` workers (1..64), each with its own context on
 *   the resident graph's device; a request enters the layout stage when the
 *   estimated HBM footprint of all requests in that stage, its own included,
 *   is at most hbm_budget bytes (a request alone is always admitted);
 *   waiting requests keep their arrival order.  The resident graph must stay
 *   alive and unchanged until bgl_server_destroy.
 * bgl_server_submit: queues a request (p is copied); *id identifies it.
 * bgl_server_wait: blocks until the request is done; returns its status
 *   (BGL_EINVAL if the neighbourhood exceeds max_nodes); *n_nodes its size;
 *   times[3] (may be NULL) the steady-clock seconds of submission, admission
 *   to the layout stage and completion (coordinates in host memory);
 *   bytes[2] (may be NULL) the estimated footprint and the measured peak of
 *   device memory of its layout stage.
 * bgl_server_fetch: copies the result (node_ids[n] resident ids, xy[2n]) and
 *   forgets the request; NULL arrays only forget it.
 * bgl_server_stats: the largest estimated in-flight footprint so far.
 * bgl_server_batching: from then on, a worker that takes a request also
 *   takes the requests queued right behind it that have equal parameters
 *   (field by field), while they number at most max_requests and their
 *   neighbourhoods at most max_nodes nodes in all, and lays them out with one
 *   layout: the disjoint union of their subgraphs, in which every node seeds
 *   its initial position with its local id in its own request.  A k-hop
 *   neighbourhood is connected, so every request is one component of the
 *   union and its coordinates are bitwise those it gets alone.  Requests
 *   with p->assemble = 1, and requests whose component takes ForceAtlas2
 *   with FMM repulsion (its evaluations share no launches with the others,
 *   so batching would only serialise them), are laid out alone.  The exact
 *   sums of all components of one layout share their launches, which is
 *   where batching gains.  max_requests = 1 (the default)
 *   turns batching off; BGL_EINVAL for max_requests < 1 or max_nodes < 0.
 * bgl_server_batch_stats: *batches layouts that served more than one
 *   request so far, and *batched the requests they served (either may be
 *   NULL).
 * bgl_server_destroy: finishes the queued requests and stops the workers.
 * A request's result does not depend on the other requests in flight.
 */
typedef struct bgl_server bgl_server;
bgl_status bgl_graph_khop(bgl_graph *g, int64_t seed, int32_t hops, int64_t max_nodes, int64_t *n_nodes,
                          int32_t *node_ids, int64_t *n_edges, int32_t *u, int32_t *v);
bgl_status bgl_server_create(bgl_graph *resident, int32_t slots, int64_t hbm_budget, bgl_server **out);
bgl_status bgl_server_submit(bgl_server *srv, int64_t seed, int32_t hops, int64_t max_nodes, const bgl_params *p,
                             int64_t *id);
bgl_status bgl_server_wait(bgl_server *srv, int64_t id, int64_t *n_nodes, double *times, int64_t *bytes);
bgl_status bgl_server_fetch(bgl_server *srv, int64_t id, int32_t *node_ids, float *xy);
bgl_status bgl_server_stats(bgl_server *srv, int64_t *inflight_max_bytes);
bgl_status bgl_server_batching(bgl_server *srv, int32_t max_requests, int64_t max_nodes);
bgl_status bgl_server_batch_stats(bgl_server *srv, int64_t *batches, int64_t *batched);
bgl_status bgl_server_destroy(bgl_server *srv);

/* ------------------------------------------ resumable runs and checkpoints */

/*
 * A ForceAtlas2 run (Section 3.2) that lives on the graph between calls, so
 * that a long layout can be advanced in pieces, inspected, checkpointed and
 * resumed.  The graph holds at most one session; components must have been
 * computed (bgl_components), and recomputing them ends the session.
 *
 * bgl_fa2_session_begin: starts a session on component c from the caller's
 *   local positions xy_in[2 n_c] (x, y interleaved), with F_{-1} = 0,
 *   s_G = 1 and a private copy of *p; replaces any earlier session.
 * bgl_fa2_session_advance: runs `iters` more iterations; stats_out (3 * iters
 *   doubles, may be NULL) receives swing, traction and s_G of each.  Advancing
 *   by a then b iterations gives bitwise the positions of a + b iterations
 *   in one call, and those of bgl_fa2_step with a + b iterations.
 * bgl_fa2_session_positions: copies the current local positions to
 *   xy_out[2 n_c]; iters_done (may be NULL) receives the iterations run.
 * No session: BGL_ESTATE.  All three synchronise the context's stream.
 */
bgl_status bgl_fa2_session_begin(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in);
bgl_status bgl_fa2_session_advance(bgl_graph *g, int32_t iters, double *stats_out);
bgl_status bgl_fa2_session_positions(bgl_graph *g, float *xy_out, int64_t *iters_done);

/*
 * Checkpoint of the graph's session (recovery of a long layout; the paper
 * has no counterpart, what it saves is the state of Section 3.2's
 * iteration): everything the iteration needs to
 * continue -- positions, F_{t-1}, s_G, the iteration count, the parameters
 * and the FMM's choice of radix passes for its next sort -- in a host
 * buffer owned by the caller, plus the identity of
 * the component (graph sizes, component index and size, and a 64-bit hash of
 * its node ids and adjacency).
 * bgl_state_save: with buf = NULL stores the size needed in *len; otherwise
 *   *len must be at least that size, the state is written to buf and *len
 *   set to the bytes written.  No session: BGL_ESTATE.
 * bgl_state_load: replaces the graph's session by the checkpoint in
 *   buf[len].  The graph must be the one the checkpoint came from (rebuilt
 *   from the same input and with components computed): anything else, a
 *   short buffer or a foreign format returns BGL_EINVAL and leaves the
 *   session unchanged.  Advancing a loaded session continues bitwise as the
 *   saved one would have.
 * The format is host-endian and tied to this library version.
 */
bgl_status bgl_state_save(bgl_graph *g, void *buf, size_t *len);
bgl_status bgl_state_load(bgl_graph *g, const void *buf, size_t len);

/* ---------------------------------------------------------------- profiling */

#define BGL_FMM_NSTATS 18

/*
 * Profiling aid for the Fast Multipole repulsion (Section 3.2.1) on
 * component c at local positions xy_in[2 n_c]: runs `reps` evaluations with
 * p->fmm_p and p->leaf_size and fills out[BGL_FMM_NSTATS] with
 *   0 boxes, 1 leaves, 2 depth (deepest level),
 *   3 near-field pairs (targets x sources over the U lists, self pairs included),
 *   4 M2L translations (V entries), 5 M2P terms (W entries x targets),
 *   6 P2L terms (sources of the X entries),
 *   7..13 mean device milliseconds of the phases run one after another:
 *   points (bounding box, Morton keys, radix sort, gather), tree,
 *   neighbour tables and interaction lists, upward pass (P2M, M2M),
 *   downward pass (M2L, P2L, L2L), near field (P2P), far field (L2P, M2P);
 *   14 mean milliseconds of a whole evaluation in the schedule used inside
 *   ForceAtlas2 iterations (upward and downward passes overlapping the near
 *   field on a second stream);
 *   15 largest |F_last - F_first| / largest |F_first| between the first
 *   evaluation (radix sort over all 32 key bits) and the last one, whose sort
 *   skips the two low passes when the previous tree was at most 8 levels
 *   deep (then the trees are the same and only the order of points inside
 *   a leaf differs); 16 the passes skipped by the last evaluation (0 or 2);
 *   17 leaves whose W list is longer than the 16 entries the far-field
 *   kernel stages (their M2P runs on sixteen warps per leaf).
 * Synchronises the stream.
 */
bgl_status bgl_fmm_stats(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in, int32_t reps,
                         double *out);

/* ------------------------------------------------------- allocation-free step */

#define BGL_NOALLOC_MAX_NODES (1 << 20)

/*
 * One ForceAtlas2 iteration with exact repulsion on one component held in
 * caller-owned device arrays, allocating no memory.  The paper has no
 * counterpart: this is a variant of bgl_fa2_step for callers that cannot
 * allocate device memory when they run it -- a process that reserves all of
 * its HBM for its own pool up front, or a latency-bound loop that cannot
 * take the device-wide synchronisation cudaMalloc/cudaFree may cause.
 *
 * Arrays (device memory of the context's device, local ids 0..n-1):
 *   d_off[n+1], d_adj[d_off[n]]  undirected adjacency (CSR)
 *   d_mass[n]                    degree + 1
 *   d_xy[2n]      in/out         positions (x, y interleaved)
 *   d_fprev[2n]   in/out         previous forces; zero before the first iteration
 *   d_f[2n]       out            this iteration's forces
 *   d_sg[1]       in/out         global speed s_G; 1.0 before the first iteration
 * Calling it `iters` times from zero d_fprev and d_sg = 1 applies the force,
 * swing, traction and update rules of bgl_fa2_step with
 * p->repulsion = BGL_REP_EXACT (p->kr, kg, ks, ksmax, tau, swing_variant);
 * its sums are taken in another order and precision, so the two agree within
 * rounding (positions within 1e-3 of the layout's bounding-box diagonal and
 * s_G within 1e-4 relative after two iterations), not bitwise.  A position
 * that becomes non-finite is recorded on the context; the next
 * bgl_ctx_sync reports it as BGL_ENUMERIC and clears the record.
 *
 * Scratch: the per-tile swing/traction sums and a counter live in one
 * fixed array of about 8 KiB per device (room for BGL_NOALLOC_MAX_NODES
 * nodes), held by every GPU that loads the library until exit; the context
 * looks up its device address when it is created.  n above
 * BGL_NOALLOC_MAX_NODES returns BGL_EINVAL.  Every call shares the array
 * and leaves its last contents there: calls whose work overlaps on the GPU
 * (other streams, other host threads, other contexts on the same device)
 * race on it and must be serialised by the caller.  Work is queued on the
 * context's stream; the call does not synchronise it.
 */
bgl_status bgl_fa2_iteration_noalloc(bgl_ctx *ctx, int64_t n, const int64_t *d_off, const int32_t *d_adj,
                                     const float *d_mass, float *d_xy, float *d_fprev, float *d_f, double *d_sg,
                                     const bgl_params *p);

/* Measured ALU throughput behind the roofline of the pair kernels (the
 * all-pairs repulsion of Section 3.2): out[0] FP32 FMA lanes, out[1] MUFU
 * reciprocals (rcp.approx) and out[2] repulsion pairs (7 FP32 operations and
 * one reciprocal, sources in registers), each per SM per clock from the
 * clock64() counts of one 1,024-thread block per SM; out[3] the SM count;
 * out[4] repulsion pairs taken two at a time with packed FP32x2 arithmetic
 * (7 packed operations and two reciprocals per two pairs).  out holds 5
 * doubles.  Synchronises the stream. */
bgl_status bgl_peak_probe(bgl_ctx *ctx, double *out);

/* Number of kernels this process has launched through the library so far
 * (direct launches plus the kernel nodes of every CUDA graph replay); a
 * measurement aid with no counterpart in the paper. */
int64_t bgl_launch_count(void);

/* Test aid for the failure paths (the paper has no counterpart): after
 * `after` more successful device allocations on this context, the next one
 * fails as if the device were out of memory, so the call making it returns
 * BGL_ENOMEM with its outputs untouched; the aid then turns itself off.
 * after = -1 turns it off at once.  No GPU fault is involved. */
bgl_status bgl_debug_fail_alloc(bgl_ctx *ctx, int64_t after);

#ifdef __cplusplus
}
#endif

#endif /* BGL_H */
