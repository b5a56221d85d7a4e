// Serving layouts of neighbourhoods of a resident graph.
//
// A request names a seed node and a hop count k: its subgraph is the
// k-hop neighbourhood of the seed in the resident graph (every node within
// k undirected hops and every edge between two of them), laid out with the
// method of Section 4 (KK for small components, ForceAtlas2 with FMM or exact
// repulsion for large ones).  The server keeps the resident graph in HBM and
// runs `slots` workers, each with its own context (stream, allocator,
// extraction scratch), so the work of several requests overlaps on the
// device.  A request is admitted to the layout stage when the estimated HBM
// footprint of everything in flight, its own included, fits the budget (a
// lone request is always admitted); requests that arrive meanwhile wait in
// arrival order.  Results do not depend on what else runs: every kernel is
// deterministic and per-request state is private to its worker.
//
// k-hop extraction on the device: frontier expansion edge-parallel (a
// thread per frontier edge, its frontier node by binary search over the
// degree prefix sums), visited marks stamped with a per-worker counter (never
// cleared), then the visited nodes sorted by id (local id = rank, so the
// subgraph does not depend on the order of discovery) and the induced edges
// listed per node in adjacency order.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>

#include <atomic>

#include "bgl_internal.cuh"

namespace bgl {

namespace {

constexpr int KH_TPB = 256;

inline unsigned kh_blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + KH_TPB - 1) / KH_TPB); }

// dst[i] = src[i] + add, i < count (a request's edges in the batch's numbering)
__global__ void kh_offset_copy_kernel(const int32_t *__restrict__ src, int32_t *__restrict__ dst, int64_t count,
                                      int32_t add) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = src[i] + add;
}

// dst[i] = i, i < count (a request's local ids, seeding its initial positions)
__global__ void kh_iota_kernel(int32_t *__restrict__ dst, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = (int32_t)i;
}

__global__ void kh_seed_kernel(int32_t *stamp, int32_t *vis, int32_t seed, int32_t epoch) {
    stamp[seed] = epoch;
    vis[0] = seed;
}

__global__ void kh_deg_kernel(const int32_t *__restrict__ front, int64_t nf, const int64_t *__restrict__ off,
                              int64_t *__restrict__ deg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) deg[i] = off[front[i] + 1] - off[front[i]];
}

// one thread per edge of the frontier; new nodes appended to vis[base ..]
__global__ void kh_expand_kernel(const int32_t *__restrict__ front, int64_t nf, const int64_t *__restrict__ dscan,
                                 int64_t E, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                 int32_t *stamp, int32_t epoch, int32_t *vis, int64_t base, int64_t cap,
                                 unsigned long long *cnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int64_t lo = 0, hi = nf;           // largest i with dscan[i] <= e
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (dscan[mid] <= e) lo = mid;
        else hi = mid;
    }
    const int32_t f = front[lo];
    const int32_t w = adj[off[f] + (e - dscan[lo])];
    if (stamp[w] == epoch) return;
    if (atomicExch(&stamp[w], epoch) == epoch) return;
    const unsigned long long idx = atomicAdd(cnt, 1ull);
    if (base + (int64_t)idx < cap) vis[base + idx] = w;
}

__global__ void kh_local_kernel(const int32_t *__restrict__ vis, int64_t n, int32_t *__restrict__ local) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) local[vis[r]] = (int32_t)r;
}

// Induced edges (r, local[w]) with local[w] > r, one thread per adjacency
// entry e of the neighbourhood's nodes (ds: their degree prefix sums), so a
// hub's list is spread over many threads; entries in (node, adjacency)
// order, so each node's edges keep its adjacency order.

// the last r in [lo, hi] with ds[r] <= e (ds non-decreasing, ds[lo] <= e)
__device__ __forceinline__ int64_t kh_owner(const int64_t *__restrict__ ds, int64_t lo, int64_t hi, int64_t e) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (ds[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// node r and neighbour w of entry e = blockIdx.x * blockDim.x + threadIdx.x
// (false past E); the block's node range found once
__device__ __forceinline__ bool kh_entry(const int32_t *__restrict__ vis, int64_t n, const int64_t *__restrict__ ds,
                                         int64_t E, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                         int64_t &r, int32_t &w) {
    __shared__ int64_t rr[2];
    const int64_t k0 = (int64_t)blockIdx.x * blockDim.x;
    if (threadIdx.x < 2) rr[threadIdx.x] = kh_owner(ds, 0, n - 1, threadIdx.x == 0 ? k0 : min(E, k0 + (int64_t)blockDim.x) - 1);
    __syncthreads();
    const int64_t e = k0 + threadIdx.x;
    if (e >= E) return false;
    r = kh_owner(ds, rr[0], rr[1], e);
    w = adj[off[vis[r]] + (e - ds[r])];
    return true;
}

__global__ void kh_edge_flag_kernel(const int32_t *__restrict__ vis, int64_t n, const int64_t *__restrict__ ds,
                                    int64_t E, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                    const int32_t *__restrict__ stamp, int32_t epoch,
                                    const int32_t *__restrict__ local, int32_t *__restrict__ keep) {
    if ((int64_t)blockIdx.x * blockDim.x >= E) return;
    int64_t r;
    int32_t w;
    if (!kh_entry(vis, n, ds, E, off, adj, r, w)) return;
    keep[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = stamp[w] == epoch && local[w] > r ? 1 : 0;
}

__global__ void kh_edge_fill_kernel(const int32_t *__restrict__ vis, int64_t n, const int64_t *__restrict__ ds,
                                    int64_t E, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                    const int32_t *__restrict__ stamp, int32_t epoch,
                                    const int32_t *__restrict__ local, const int32_t *__restrict__ kpos,
                                    int32_t *__restrict__ u, int32_t *__restrict__ v) {
    if ((int64_t)blockIdx.x * blockDim.x >= E) return;
    int64_t r;
    int32_t w;
    if (!kh_entry(vis, n, ds, E, off, adj, r, w)) return;
    if (stamp[w] == epoch && local[w] > r) {
        const int64_t k = kpos[(int64_t)blockIdx.x * blockDim.x + threadIdx.x];
        u[k] = (int32_t)r;
        v[k] = local[w];
    }
}

}  // namespace

// Scratch of one extracting context: visited stamps and local ids over the
// resident graph's nodes, the visit list (at most cap entries).
struct KhopScratch {
    DevBuf<int32_t> stamp, local, vis;
    DevBuf<int64_t> deg, dscan, tot;
    DevBuf<unsigned long long> cnt;
    int32_t epoch = 0;
    int64_t cap = 0;
    void reserve(bgl_ctx *c, int64_t n_res, int64_t cap_) {
        if (stamp.n < (size_t)n_res) {
            stamp.reset(c->alloc, n_res);
            local.reset(c->alloc, n_res);
            BGL_CUDA(cudaMemsetAsync(stamp.p, 0, sizeof(int32_t) * n_res, c->stream));
            epoch = 0;
        }
        if (cap < cap_) {
            vis.reset(c->alloc, cap_ + 1);
            deg.reset(c->alloc, cap_ + 1);
            dscan.reset(c->alloc, cap_ + 1);
            cap = cap_;
        }
        if (!tot.p) tot.reset(c->alloc, 1);
        if (!cnt.p) cnt.reset(c->alloc, 1);
    }
};

// k-hop neighbourhood of `seed` in R (undirected CSR R->off, R->adj) on the
// stream of ctx.  Returns its node count, or -1 if it has more than cap
// nodes; on success vis[0 .. n) holds the node ids in ascending order and
// (u, v)[0 .. m) the induced edges in local ids.
static int64_t khop_extract(bgl_ctx *ctx, const bgl_graph *R, KhopScratch &ws, int64_t seed, int hops, int64_t cap,
                            DevBuf<int32_t> &u, DevBuf<int32_t> &v, int64_t &m) {
    BGL_REQUIRE(seed >= 0 && seed < R->n, "khop: seed out of range");
    BGL_REQUIRE(hops >= 0, "khop: hops must be >= 0");
    BGL_REQUIRE(cap >= 1, "khop: max_nodes must be >= 1");
    cudaStream_t s = ctx->stream;
    ws.reserve(ctx, R->n, cap);
    const int32_t epoch = ++ws.epoch;
    kh_seed_kernel<<<1, 1, 0, s>>>(ws.stamp.p, ws.vis.p, (int32_t)seed, epoch);
    BGL_LAUNCH_CHECK();
    int64_t total = 1, f0 = 0, nf = 1;
    for (int h = 0; h < hops && nf > 0; ++h) {
        kh_deg_kernel<<<kh_blocks(nf), KH_TPB, 0, s>>>(ws.vis.p + f0, nf, R->off.p, ws.deg.p);
        BGL_LAUNCH_CHECK();
        scan_exclusive_i64(ctx, ws.deg.p, ws.dscan.p, nf, ws.tot.p);
        int64_t E = 0;
        BGL_CUDA(cudaMemcpyAsync(&E, ws.tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaMemsetAsync(ws.cnt.p, 0, sizeof(unsigned long long), s));
        BGL_CUDA(cudaStreamSynchronize(s));
        if (E == 0) break;
        kh_expand_kernel<<<kh_blocks(E), KH_TPB, 0, s>>>(ws.vis.p + f0, nf, ws.dscan.p, E, R->off.p, R->adj.p,
                                                         ws.stamp.p, epoch, ws.vis.p, total, cap, ws.cnt.p);
        BGL_LAUNCH_CHECK();
        unsigned long long add = 0;
        BGL_CUDA(cudaMemcpyAsync(&add, ws.cnt.p, sizeof(add), cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaStreamSynchronize(s));
        if (total + (int64_t)add > cap) return -1;
        f0 = total;
        nf = (int64_t)add;
        total += nf;
    }
    const int64_t n = total;
    // ascending node ids: local id = rank
    DevBuf<uint32_t> keys(ctx->alloc, n);
    BGL_CUDA(cudaMemcpyAsync(keys.p, ws.vis.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    radix_sort_u32(ctx, keys.p, nullptr, n, std::max(1, bits_for((uint64_t)R->n)));
    BGL_CUDA(cudaMemcpyAsync(ws.vis.p, keys.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    kh_local_kernel<<<kh_blocks(n), KH_TPB, 0, s>>>(ws.vis.p, n, ws.local.p);
    BGL_LAUNCH_CHECK();
    // adjacency entries of the neighbourhood's nodes: degree prefix sums
    kh_deg_kernel<<<kh_blocks(n), KH_TPB, 0, s>>>(ws.vis.p, n, R->off.p, ws.deg.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i64(ctx, ws.deg.p, ws.dscan.p, n, ws.tot.p);
    int64_t E = 0;
    BGL_CUDA(cudaMemcpyAsync(&E, ws.tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    BGL_REQUIRE(E < (int64_t(1) << 31), "khop: more than 2^31 adjacency entries in the neighbourhood");
    m = 0;
    DevBuf<int32_t> keep(ctx->alloc, std::max<int64_t>(E, 1)), kpos(ctx->alloc, std::max<int64_t>(E, 1));
    DevBuf<int32_t> ktot(ctx->alloc, 1);
    if (E > 0) {
        kh_edge_flag_kernel<<<kh_blocks(E), KH_TPB, 0, s>>>(ws.vis.p, n, ws.dscan.p, E, R->off.p, R->adj.p,
                                                            ws.stamp.p, epoch, ws.local.p, keep.p);
        BGL_LAUNCH_CHECK();
        scan_exclusive_i32(ctx, keep.p, kpos.p, E, ktot.p);
        int32_t m32 = 0;
        BGL_CUDA(cudaMemcpyAsync(&m32, ktot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaStreamSynchronize(s));
        m = m32;
    }
    u.reset(ctx->alloc, std::max<int64_t>(m, 1));
    v.reset(ctx->alloc, std::max<int64_t>(m, 1));
    if (m > 0) {
        kh_edge_fill_kernel<<<kh_blocks(E), KH_TPB, 0, s>>>(ws.vis.p, n, ws.dscan.p, E, R->off.p, R->adj.p,
                                                            ws.stamp.p, epoch, ws.local.p, kpos.p, u.p, v.p);
        BGL_LAUNCH_CHECK();
    }
    return n;
}

// HBM footprint of laying out a subgraph of n nodes and m undirected edges:
// graph and component arrays, layout state, FMM plan (boxes, lists,
// expansions, sort workspace) and the caching allocator's slack
int64_t serve_footprint(int64_t n, int64_t m) { return 768 * n + 96 * m + (int64_t(16) << 20); }

struct ServeRequest {
    int64_t seed = 0, cap = 0;
    int hops = 0;
    bgl_params p;
    bgl_status status = BGL_OK;
    std::string error;
    bool done = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int64_t footprint = 0, peak = 0;
    std::vector<int32_t> nodes;
    std::vector<float> xy;
};

struct Server {
    bgl_graph *R = nullptr;
    int64_t budget = 0;
    // batching: up to batch_max queued requests with equal parameters whose
    // neighbourhoods total at most batch_nodes nodes share one layout
    std::atomic<int> batch_max{1};
    std::atomic<int64_t> batch_nodes{0};
    std::mutex mu;
    std::condition_variable cv_work, cv_mem, cv_done;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<ServeRequest>> reqs;
    int64_t next_id = 1, inflight = 0, inflight_max = 0;
    int64_t batches = 0, batched = 0;     // layouts of more than one request, and their requests
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<bgl_ctx *> ctxs;
    std::string init_error;
};

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static bool params_equal(const bgl_params &a, const bgl_params &b) {
    return a.seed == b.seed && a.kk_max_nodes == b.kk_max_nodes && a.fa2_iters == b.fa2_iters && a.kr == b.kr &&
           a.kg == b.kg && a.ks == b.ks && a.ksmax == b.ksmax && a.tau == b.tau && a.repulsion == b.repulsion &&
           a.fmm_p == b.fmm_p && a.leaf_size == b.leaf_size && a.fmm_min_nodes == b.fmm_min_nodes &&
           a.swing_variant == b.swing_variant && a.kk_sweeps == b.kk_sweeps && a.kk_l == b.kk_l &&
           a.kk_tol == b.kk_tol && a.assemble == b.assemble && a.m2l_bf16 == b.m2l_bf16;
}

// A request's neighbourhood: node ids on the host (ascending), induced edges
// in local ids on the device
struct Extracted {
    ServeRequest *r = nullptr;
    int64_t n = 0, m = 0;
    DevBuf<int32_t> u, v;
};

static void extract(Server *S, bgl_ctx *ctx, KhopScratch &ws, Extracted &x) {
    BGL_RANGE("serving: k-hop extraction");
    ServeRequest *r = x.r;
    x.n = khop_extract(ctx, S->R, ws, r->seed, r->hops, r->cap, x.u, x.v, x.m);
    if (x.n < 0) fail(BGL_EINVAL, "neighbourhood larger than max_nodes");
    r->nodes.resize(x.n);
    // the visit list is the next extraction's scratch: copy it out now
    BGL_CUDA(cudaMemcpyAsync(r->nodes.data(), ws.vis.p, sizeof(int32_t) * x.n, cudaMemcpyDeviceToHost, ctx->stream));
    BGL_CUDA(cudaStreamSynchronize(ctx->stream));
}

// Lays out one or several extracted neighbourhoods with one bgl_layout.
// Several go in as one graph, the disjoint union of the requests' subgraphs
// (request k's nodes numbered from the sum of the earlier sizes), whose
// nodes keep their own local ids as the ids that seed their initial
// positions.  A k-hop neighbourhood is connected, so each request is one
// component of the union, and a component's layout depends only on its
// seed ids, adjacency and the parameters: every request's coordinates are
// bitwise those of its own layout.
static void layout_group(Server *S, bgl_ctx *ctx, std::vector<Extracted> &grp) {
    BGL_RANGE("serving: layout of a request group");
    int64_t n = 0, m = 0;
    for (auto &x : grp) {
        n += x.n;
        m += x.m;
    }
    const int64_t fp = serve_footprint(n, m);
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_mem.wait(lk, [&] { return S->inflight == 0 || S->inflight + fp <= S->budget || S->stop; });
        S->inflight += fp;
        S->inflight_max = std::max(S->inflight_max, S->inflight);
    }
    const double t_admit = now_s();
    for (auto &x : grp) {
        x.r->footprint = fp;
        x.r->t_admit = t_admit;
    }
    ctx->alloc->reset_peak();
    const size_t live0 = ctx->alloc->live_bytes();
    cudaStream_t s = ctx->stream;
    try {
        std::unique_ptr<bgl_graph> sub(new bgl_graph());
        sub->ctx = ctx;
        if (grp.size() == 1) {
            graph_from_edges_device(sub.get(), n, m, grp[0].u.p, grp[0].v.p);
        } else {
            DevBuf<int32_t> u(ctx->alloc, std::max<int64_t>(m, 1)), v(ctx->alloc, std::max<int64_t>(m, 1));
            sub->seed_id.reset(ctx->alloc, std::max<int64_t>(n, 1));
            int64_t no = 0, mo = 0;
            for (auto &x : grp) {
                if (x.m > 0) {
                    kh_offset_copy_kernel<<<kh_blocks(x.m), KH_TPB, 0, s>>>(x.u.p, u.p + mo, x.m, (int32_t)no);
                    BGL_LAUNCH_CHECK();
                    kh_offset_copy_kernel<<<kh_blocks(x.m), KH_TPB, 0, s>>>(x.v.p, v.p + mo, x.m, (int32_t)no);
                    BGL_LAUNCH_CHECK();
                }
                kh_iota_kernel<<<kh_blocks(x.n), KH_TPB, 0, s>>>(sub->seed_id.p + no, x.n);
                BGL_LAUNCH_CHECK();
                no += x.n;
                mo += x.m;
            }
            graph_from_edges_device(sub.get(), n, m, u.p, v.p);
        }
        for (auto &x : grp) {
            x.u.release();
            x.v.release();
        }
        components_device(sub.get());
        DevBuf<float2> xy(ctx->alloc, std::max<int64_t>(n, 1));
        layout_device(sub.get(), &grp[0].r->p, reinterpret_cast<float *>(xy.p));
        int64_t no = 0;
        for (auto &x : grp) {
            x.r->xy.resize(2 * x.n);
            BGL_CUDA(cudaMemcpyAsync(x.r->xy.data(), xy.p + no, sizeof(float2) * x.n, cudaMemcpyDeviceToHost, s));
            no += x.n;
        }
        BGL_CUDA(cudaStreamSynchronize(s));
        const int64_t peak = (int64_t)(ctx->alloc->peak_bytes() - std::min(live0, ctx->alloc->peak_bytes()));
        for (auto &x : grp) x.r->peak = peak;
    } catch (...) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->inflight -= fp;
        S->cv_mem.notify_all();
        throw;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->inflight -= fp;
    if (grp.size() > 1) {
        ++S->batches;
        S->batched += (int64_t)grp.size();
    }
    S->cv_mem.notify_all();
}

static void finish(Server *S, ServeRequest *r, bgl_status st, const std::string &msg) {
    std::lock_guard<std::mutex> lk(S->mu);
    r->status = st;
    r->error = msg;
    r->t_done = now_s();
    r->done = true;
    S->cv_done.notify_all();
}

// runs f, returning its failure as a status and message
template <class F>
static bgl_status guarded(F &&f, std::string &msg) {
    try {
        f();
        return BGL_OK;
    } catch (const Error &e) {
        msg = e.what();
        return e.status;
    } catch (const std::exception &e) {
        msg = e.what();
        return BGL_ECUDA;
    }
}

static void serve_group(Server *S, bgl_ctx *ctx, std::vector<Extracted> &grp) {
    std::string msg;
    const bgl_status st = guarded([&] { layout_group(S, ctx, grp); }, msg);
    for (auto &x : grp) finish(S, x.r, st, msg);
}

// whether a request of n nodes (one component) avoids the FMM: KK, or
// ForceAtlas2 with exact repulsion (AUTO below its threshold; below 2,048
// nodes when the crossover is measured)
static bool avoids_fmm(const bgl_params &p, int64_t n) {
    if (n <= p.kk_max_nodes || p.repulsion == BGL_REP_EXACT) return true;
    if (p.repulsion == BGL_REP_AUTO) return p.fmm_min_nodes >= 0 ? n < p.fmm_min_nodes : n < 2048;
    return false;
}

// whether a request of n nodes may share a layout: it is small, lays out
// without the FMM (the exact sums of all components of a run share their
// launches, each FMM evaluation has its own, so batched FMM requests would
// only run one after another) and without assembly into one frame
static bool batchable(const Server *S, const ServeRequest *r, int64_t n) {
    return S->batch_max > 1 && r->p.assemble == 0 && n <= S->batch_nodes && avoids_fmm(r->p, n);
}

static void worker_loop(Server *S, bgl_ctx *ctx) {
    cudaSetDevice(ctx->device);
    KhopScratch ws;
    auto next = [&](const ServeRequest *like) -> ServeRequest * {
        // the request at the head of the queue (any, or with like's parameters)
        std::unique_lock<std::mutex> lk(S->mu);
        if (!like) S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
        if (S->queue.empty()) return nullptr;
        ServeRequest *r = S->reqs[S->queue.front()].get();
        if (like && !params_equal(r->p, like->p)) return nullptr;
        S->queue.pop_front();
        return r;
    };
    for (;;) {
        ServeRequest *r0 = next(nullptr);
        if (!r0) {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->stop && S->queue.empty()) return;
            continue;
        }
        std::vector<Extracted> grp(1);
        grp[0].r = r0;
        std::string msg;
        bgl_status st = guarded([&] { extract(S, ctx, ws, grp[0]); }, msg);
        if (st != BGL_OK) {
            finish(S, r0, st, msg);
            continue;
        }
        // small requests queued behind it with the same parameters join it
        std::vector<Extracted> rest;
        if (batchable(S, r0, grp[0].n)) {
            int64_t total = grp[0].n;
            while ((int)grp.size() < S->batch_max) {
                ServeRequest *r = next(r0);
                if (!r) break;
                Extracted x;
                x.r = r;
                st = guarded([&] { extract(S, ctx, ws, x); }, msg);
                if (st != BGL_OK) {
                    finish(S, r, st, msg);
                    continue;
                }
                if (!batchable(S, r, x.n) || total + x.n > S->batch_nodes) {
                    rest.push_back(std::move(x));       // laid out on its own, next
                    break;
                }
                total += x.n;
                grp.push_back(std::move(x));
            }
        }
        serve_group(S, ctx, grp);
        for (auto &x : rest) {
            std::vector<Extracted> one;
            one.push_back(std::move(x));
            serve_group(S, ctx, one);
        }
    }
}

}  // namespace bgl

using namespace bgl;

extern "C" {

struct bgl_server {
    Server s;
};

bgl_status bgl_server_create(bgl_graph *resident, int32_t slots, int64_t hbm_budget, bgl_server **out) {
    if (!resident || !out || slots < 1 || slots > 64 || hbm_budget <= 0) return BGL_EINVAL;
    *out = nullptr;
    bgl_server *srv = new (std::nothrow) bgl_server();
    if (!srv) return BGL_ENOMEM;
    srv->s.R = resident;
    srv->s.budget = hbm_budget;
    for (int i = 0; i < slots; ++i) {
        bgl_ctx *c = nullptr;
        const bgl_status st = bgl_ctx_create(resident->ctx->device, &c);
        if (st != BGL_OK) {
            bgl_server_destroy(srv);
            return st;
        }
        srv->s.ctxs.push_back(c);
    }
    // the resident graph must be complete before other streams read it
    if (cudaStreamSynchronize(resident->ctx->stream) != cudaSuccess) {
        bgl_server_destroy(srv);
        return BGL_ECUDA;
    }
    for (bgl_ctx *c : srv->s.ctxs) srv->s.workers.emplace_back(worker_loop, &srv->s, c);
    *out = srv;
    return BGL_OK;
}

bgl_status bgl_server_submit(bgl_server *srv, int64_t seed, int32_t hops, int64_t max_nodes, const bgl_params *p,
                             int64_t *id) {
    if (!srv || !p || !id) return BGL_EINVAL;
    if (seed < 0 || seed >= srv->s.R->n || hops < 0 || max_nodes < 1) return BGL_EINVAL;
    try {
        check_params(p);
    } catch (const Error &e) {
        return e.status;
    }
    std::unique_ptr<ServeRequest> r(new ServeRequest());
    r->seed = seed;
    r->hops = hops;
    r->cap = max_nodes;
    r->p = *p;
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(srv->s.mu);
    if (srv->s.stop) return BGL_ESTATE;
    *id = srv->s.next_id++;
    srv->s.reqs[*id] = std::move(r);
    srv->s.queue.push_back(*id);
    srv->s.cv_work.notify_one();
    return BGL_OK;
}

bgl_status bgl_server_wait(bgl_server *srv, int64_t id, int64_t *n_nodes, double *times, int64_t *bytes) {
    if (!srv) return BGL_EINVAL;
    std::unique_lock<std::mutex> lk(srv->s.mu);
    auto it = srv->s.reqs.find(id);
    if (it == srv->s.reqs.end()) return BGL_EINVAL;
    ServeRequest *r = it->second.get();
    srv->s.cv_done.wait(lk, [&] { return r->done; });
    if (n_nodes) *n_nodes = (int64_t)r->nodes.size();
    if (times) {
        times[0] = r->t_submit;
        times[1] = r->t_admit;
        times[2] = r->t_done;
    }
    if (bytes) {
        bytes[0] = r->footprint;
        bytes[1] = r->peak;
    }
    return r->status;
}

bgl_status bgl_server_fetch(bgl_server *srv, int64_t id, int32_t *node_ids, float *xy) {
    if (!srv) return BGL_EINVAL;
    std::lock_guard<std::mutex> lk(srv->s.mu);
    auto it = srv->s.reqs.find(id);
    if (it == srv->s.reqs.end() || !it->second->done) return BGL_EINVAL;
    ServeRequest *r = it->second.get();
    const bgl_status st = r->status;
    if (st == BGL_OK) {
        if (node_ids) std::copy(r->nodes.begin(), r->nodes.end(), node_ids);
        if (xy) std::copy(r->xy.begin(), r->xy.end(), xy);
    }
    srv->s.reqs.erase(it);
    return st;
}

bgl_status bgl_server_batching(bgl_server *srv, int32_t max_requests, int64_t max_nodes) {
    if (!srv || max_requests < 1 || max_nodes < 0) return BGL_EINVAL;
    srv->s.batch_nodes = max_nodes;
    srv->s.batch_max = max_requests;
    return BGL_OK;
}

bgl_status bgl_server_batch_stats(bgl_server *srv, int64_t *batches, int64_t *batched) {
    if (!srv) return BGL_EINVAL;
    std::lock_guard<std::mutex> lk(srv->s.mu);
    if (batches) *batches = srv->s.batches;
    if (batched) *batched = srv->s.batched;
    return BGL_OK;
}

bgl_status bgl_server_stats(bgl_server *srv, int64_t *inflight_max_bytes) {
    if (!srv) return BGL_EINVAL;
    std::lock_guard<std::mutex> lk(srv->s.mu);
    if (inflight_max_bytes) *inflight_max_bytes = srv->s.inflight_max;
    return BGL_OK;
}

bgl_status bgl_server_destroy(bgl_server *srv) {
    if (!srv) return BGL_OK;
    {
        std::lock_guard<std::mutex> lk(srv->s.mu);
        srv->s.stop = true;
        srv->s.cv_work.notify_all();
        srv->s.cv_mem.notify_all();
    }
    for (auto &t : srv->s.workers) t.join();
    for (bgl_ctx *c : srv->s.ctxs) bgl_ctx_destroy(c);
    delete srv;
    return BGL_OK;
}

bgl_status bgl_graph_khop(bgl_graph *g, int64_t seed, int32_t hops, int64_t max_nodes, int64_t *n_nodes,
                          int32_t *node_ids, int64_t *n_edges, int32_t *u, int32_t *v) {
    if (!g || !n_nodes) return BGL_EINVAL;
    bgl_ctx *c = g->ctx;
    try {
        cudaSetDevice(c->device);
        KhopScratch ws;
        DevBuf<int32_t> du, dv;
        int64_t m = 0;
        const int64_t n = khop_extract(c, g, ws, seed, hops, max_nodes, du, dv, m);
        *n_nodes = n;
        if (n_edges) *n_edges = n < 0 ? 0 : m;
        if (n >= 0) {
            if (node_ids)
                BGL_CUDA(cudaMemcpyAsync(node_ids, ws.vis.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream));
            if (u && m)
                BGL_CUDA(cudaMemcpyAsync(u, du.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, c->stream));
            if (v && m)
                BGL_CUDA(cudaMemcpyAsync(v, dv.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, c->stream));
        }
        BGL_CUDA(cudaStreamSynchronize(c->stream));
        c->last_error.clear();
        return BGL_OK;
    } catch (const Error &e) {
        c->last_error = e.what();
        return e.status;
    } catch (const std::exception &e) {
        c->last_error = e.what();
        return BGL_ECUDA;
    }
}

}  // extern "C"
