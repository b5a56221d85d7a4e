// C ABI of the layout library (include/bgl.h): contexts, the caching device
// allocator, argument validation and the host <-> device copies around the
// device pipeline.  No exception crosses the ABI: every entry point maps
// failures to a bgl_status and keeps the message for bgl_last_error().
#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "bgl_internal.cuh"
#include "fmm.cuh"

namespace bgl {

void fail(bgl_status s, const std::string &msg) { throw Error(s, msg); }

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void check_cuda(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")";
    if (e == cudaErrorMemoryAllocation) throw Error(BGL_ENOMEM, m);
    throw Error(BGL_ECUDA, m);
}

Allocator::~Allocator() {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto &kv : free_) cudaFree(kv.second);
    for (auto &kv : live_) cudaFree(kv.first);
}

void Allocator::release_cache() {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto &kv : free_) cudaFree(kv.second);
    free_.clear();
    cached_ = 0;
}

void *Allocator::alloc(size_t bytes) {
    if (forbid) throw Error(BGL_ESTATE, "internal: device allocation inside a captured CUDA graph");
    if (fail_after.load(std::memory_order_relaxed) >= 0 && fail_after.fetch_sub(1) == 0) {
        fail_after.store(-1);
        throw Error(BGL_ENOMEM, "device allocation refused by bgl_debug_fail_alloc");
    }
    bytes = (bytes + 255) & ~size_t(255);
    {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = free_.lower_bound(bytes);
        if (it != free_.end() && it->first <= bytes + bytes / 4 + 4096) {
            void *p = it->second;
            size_t sz = it->first;
            free_.erase(it);
            cached_ -= sz;
            live_[p] = sz;
            live_bytes_ += sz;
            peak_bytes_ = std::max(peak_bytes_, live_bytes_);
            return p;
        }
    }
    void *p = nullptr;
    // stream-ordered: a new block does not synchronise the device, so
    // contexts that allocate while others compute (the serving workers) do
    // not stall each other; every entry point ends with a stream
    // synchronisation, so a cached block is complete before any reuse
    cudaError_t e = stream_ ? cudaMallocAsync(&p, bytes, *stream_) : cudaMalloc(&p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        release_cache();
        e = stream_ ? cudaMallocAsync(&p, bytes, *stream_) : cudaMalloc(&p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? BGL_ENOMEM : BGL_ECUDA,
                    std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lk(mu_);
    live_[p] = bytes;
    live_bytes_ += bytes;
    peak_bytes_ = std::max(peak_bytes_, live_bytes_);
    return p;
}

void Allocator::free(void *p) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = live_.find(p);
    if (it == live_.end()) return;
    free_.emplace(it->second, p);
    cached_ += it->second;
    live_bytes_ -= it->second;
    live_.erase(it);
}

void check_params(const bgl_params *p) {
    BGL_REQUIRE(p != nullptr, "params is NULL");
    BGL_REQUIRE(p->kk_max_nodes >= 0 && p->kk_max_nodes <= 255, "kk_max_nodes must be in [0, 255]");
    BGL_REQUIRE(p->fa2_iters >= 0, "fa2_iters must be >= 0");
    BGL_REQUIRE(p->kr >= 0 && p->kg >= 0, "kr and kg must be >= 0");
    BGL_REQUIRE(p->ks > 0 && p->ksmax > 0 && p->tau > 0, "ks, ksmax and tau must be > 0");
    BGL_REQUIRE(p->repulsion >= BGL_REP_EXACT && p->repulsion <= BGL_REP_AUTO, "repulsion must be 0, 1 or 2");
    BGL_REQUIRE(p->fmm_p >= 1 && p->fmm_p <= 24, "fmm_p must be in [1, 24]");
    BGL_REQUIRE(p->leaf_size >= 1 && p->leaf_size <= 256, "leaf_size must be in [1, 256]");
    BGL_REQUIRE(p->fmm_min_nodes >= -1, "fmm_min_nodes must be >= -1");
    BGL_REQUIRE(p->swing_variant == 0 || p->swing_variant == 1, "swing_variant must be 0 or 1");
    BGL_REQUIRE(p->kk_sweeps >= 0, "kk_sweeps must be >= 0");
    BGL_REQUIRE(p->kk_l > 0, "kk_l must be > 0");
    BGL_REQUIRE(p->kk_tol >= 0, "kk_tol must be >= 0");
    BGL_REQUIRE(p->assemble == 0 || p->assemble == 1, "assemble must be 0 or 1");
    BGL_REQUIRE(p->m2l_bf16 == 0 || p->m2l_bf16 == 1, "m2l_bf16 must be 0 or 1");
}

}  // namespace bgl

using namespace bgl;

namespace {

// Runs one C-ABI call: device made current, exceptions turned into statuses,
// and the call's NVTX range named after the calling entry point.
template <class F>
bgl_status guarded(bgl_ctx *c, F &&fn, const char *name = __builtin_FUNCTION()) {
    BGL_RANGE(name);
    try {
        if (c) BGL_CUDA(cudaSetDevice(c->device));
        fn();
        if (c) c->last_error.clear();
        return BGL_OK;
    } catch (const Error &e) {
        if (c) c->last_error = e.what();
        return e.status;
    } catch (const std::bad_alloc &) {
        if (c) c->last_error = "host allocation failed";
        return BGL_ENOMEM;
    } catch (const std::exception &e) {
        if (c) c->last_error = e.what();
        return BGL_ECUDA;
    } catch (...) {
        if (c) c->last_error = "unknown failure";
        return BGL_ECUDA;
    }
}

void check_offsets(int64_t n_tx, const int64_t *off, const char *what) {
    BGL_REQUIRE(off != nullptr, std::string(what) + " is NULL");
    BGL_REQUIRE(off[0] == 0, std::string(what) + "[0] must be 0");
    for (int64_t t = 0; t < n_tx; ++t)
        BGL_REQUIRE(off[t + 1] >= off[t], std::string(what) + " must never decrease");
}

template <typename T>
void h2d(bgl_ctx *c, T *d, const T *h, size_t n) {
    if (n) BGL_CUDA(cudaMemcpyAsync(d, h, sizeof(T) * n, cudaMemcpyHostToDevice, c->stream));
}
template <typename T>
void d2h(bgl_ctx *c, T *h, const T *d, size_t n) {
    if (n) BGL_CUDA(cudaMemcpyAsync(h, d, sizeof(T) * n, cudaMemcpyDeviceToHost, c->stream));
}
void sync(bgl_ctx *c) { BGL_CUDA(cudaStreamSynchronize(c->stream)); }

__global__ void scatter_xy_kernel(const float2 *__restrict__ xy, const int32_t *__restrict__ nodes, int64_t n,
                                  float2 *__restrict__ out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[nodes[q]] = xy[q];
}

void require_comp(const bgl_graph *g) {
    if (!g->has_comp) fail(BGL_ESTATE, "run bgl_components first");
}
void require_c(const bgl_graph *g, int64_t c) {
    require_comp(g);
    BGL_REQUIRE(c >= 0 && c < g->n_comp, "component index out of range");
}


__global__ void gather_xy_kernel(const float2 *__restrict__ xy_nodes, const int32_t *__restrict__ nodes, int64_t n,
                                 float2 *__restrict__ out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = xy_nodes[nodes[q]];
}

}  // namespace

namespace bgl {

// Full layout into a device array in node-id order.  The Kamada-Kawai
// components and the ForceAtlas2 components are independent (Section 4), so
// the KK size classes run beside the ForceAtlas2 iterations: each class on
// a stream of its own, captured into the same CUDA graph as the iteration
// loop (one graph launch lays out every component).
void layout_device(bgl_graph *g, const bgl_params *p, float *d_xy_out) {
    check_params(p);
    require_comp(g);
    split_device(g, p->kk_max_nodes);
    bgl_ctx *c = g->ctx;
    DevBuf<float2> xy(c->alloc, g->n);
    const int64_t q_fa2 = g->h_comp_off[g->n_fa2];
    std::unique_ptr<KkRun, void (*)(KkRun *)> kk(kk_prepare(g, g->n_fa2, g->n_comp), kk_destroy);
    const int nk = kk_classes(kk.get());
    std::vector<cudaStream_t> ks;
    std::vector<cudaEvent_t> kev;
    auto release = [&] {
        for (auto e : kev) cudaEventDestroy(e);
        for (auto st : ks) cudaStreamDestroy(st);
        kev.clear();
        ks.clear();
    };
    try {
        for (int i = 0; i < nk; ++i) {
            cudaStream_t st;
            BGL_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            ks.push_back(st);
        }
        for (int i = 0; i < nk + 1; ++i) {
            cudaEvent_t e;
            BGL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            kev.push_back(e);
        }
        // small components: Kamada-Kawai, one stream per size class, forked
        // from and joined back to stream s
        SideWork kk_work = [&](cudaStream_t s) {
            BGL_CUDA(cudaEventRecord(kev[nk], s));
            for (int i = 0; i < nk; ++i) {
                BGL_CUDA(cudaStreamWaitEvent(ks[i], kev[nk], 0));
                kk_enqueue(kk.get(), i, p, xy.p, 0, true, p->kk_sweeps, nullptr, ks[i]);
                BGL_CUDA(cudaEventRecord(kev[i], ks[i]));
            }
            for (int i = 0; i < nk; ++i) BGL_CUDA(cudaStreamWaitEvent(s, kev[i], 0));
        };
        if (g->n_fa2 > 0) {
            // large components: ForceAtlas2, with the KK classes beside the iterations
            init_positions(g, p, xy.p, 0, q_fa2);
            fa2_layout(g, p, xy.p, 0, 0, g->n_fa2, p->fa2_iters, nullptr, nk ? kk_work : SideWork());
        } else if (nk) {
            kk_work(c->stream);
        }
        BGL_CUDA(cudaStreamSynchronize(c->stream));
    } catch (...) {
        // nothing may still write to the scratch when it goes back to the allocator
        cudaDeviceSynchronize();
        release();
        throw;
    }
    release();
    if (g->n > 0 && p->assemble) {
        assemble_device(g, p, xy.p, reinterpret_cast<float2 *>(d_xy_out), nullptr);
    } else if (g->n > 0) {
        scatter_xy_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, c->stream>>>(xy.p, g->nodes.p, g->n,
                                                                                 reinterpret_cast<float2 *>(d_xy_out));
        BGL_LAUNCH_CHECK();
    }
}

}  // namespace bgl

extern "C" {

void bgl_params_default(bgl_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->seed = 0;
    p->kk_max_nodes = 50;
    p->fa2_iters = 50;
    p->kr = 1.0;
    p->kg = 1.0;
    p->ks = 0.1;
    p->ksmax = 10.0;
    p->tau = 1.0;
    p->repulsion = BGL_REP_AUTO;
    p->fmm_p = 8;
    p->leaf_size = 64;
    p->fmm_min_nodes = 8192;
    p->swing_variant = 0;
    p->kk_sweeps = 200;
    p->kk_l = 1.0;
    p->kk_tol = 0.0;
}

bgl_status bgl_ctx_create(int device, bgl_ctx **out) {
    if (!out) return BGL_EINVAL;
    *out = nullptr;
    bgl_ctx *c = nullptr;
    try {
        c = new bgl_ctx();
    } catch (...) {
        return BGL_ENOMEM;
    }
    c->device = device;
    bgl_status s = guarded(nullptr, [&] {
        int count = 0;
        BGL_CUDA(cudaGetDeviceCount(&count));
        BGL_REQUIRE(device >= 0 && device < count, "no such CUDA device");
        BGL_CUDA(cudaSetDevice(device));
        BGL_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
        BGL_CUDA(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
        c->stream = c->own_stream;
        c->alloc = new Allocator(device, &c->stream);
        BGL_CUDA(cudaMalloc(&c->d_flag, 4 * sizeof(int)));
        BGL_CUDA(cudaMemset(c->d_flag, 0, 4 * sizeof(int)));
        BGL_CUDA(cudaMallocHost(&c->h_flag, 4 * sizeof(int)));
        c->noalloc_scratch = static_cast<unsigned char *>(noalloc_scratch_address());
    });
    if (s != BGL_OK) {
        bgl_ctx_destroy(c);
        return s;
    }
    *out = c;
    return BGL_OK;
}

void bgl_ctx_destroy(bgl_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    delete c->alloc;
    if (c->d_flag) cudaFree(c->d_flag);
    if (c->h_flag) cudaFreeHost(c->h_flag);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

bgl_status bgl_ctx_set_stream(bgl_ctx *c, void *stream) {
    if (!c) return BGL_EINVAL;
    return guarded(c, [&] { c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream; });
}

bgl_status bgl_ctx_sync(bgl_ctx *c) {
    if (!c) return BGL_EINVAL;
    return guarded(c, [&] {
        // the allocation-free iteration records non-finite positions in
        // d_flag[2]; report that record once and clear it
        BGL_CUDA(cudaMemcpyAsync(c->h_flag + 2, c->d_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        if (c->h_flag[2]) {
            c->h_flag[2] = 0;
            BGL_CUDA(cudaMemsetAsync(c->d_flag + 2, 0, sizeof(int), c->stream));
            sync(c);
            fail(BGL_ENUMERIC, "fa2_iteration_noalloc: a position became non-finite");
        }
    });
}

const char *bgl_last_error(const bgl_ctx *c) { return c ? c->last_error.c_str() : "context is NULL"; }

bgl_status bgl_graph_build(bgl_ctx *c, int64_t n_tx, const int64_t *in_off, const uint64_t *in_addr,
                           const int64_t *out_off, const uint64_t *out_addr, bgl_graph **out) {
    if (!c || !out) return BGL_EINVAL;
    return guarded(c, [&] {
        BGL_REQUIRE(n_tx >= 0, "n_tx must be >= 0");
        check_offsets(n_tx, in_off, "in_off");
        check_offsets(n_tx, out_off, "out_off");
        const int64_t n_in = in_off[n_tx], n_out = out_off[n_tx];
        BGL_REQUIRE(n_in == 0 || in_addr, "in_addr is NULL");
        BGL_REQUIRE(n_out == 0 || out_addr, "out_addr is NULL");
        DevBuf<int64_t> dio(c->alloc, n_tx + 1), doo(c->alloc, n_tx + 1);
        DevBuf<uint64_t> dia(c->alloc, n_in), doa(c->alloc, n_out);
        h2d(c, dio.p, in_off, n_tx + 1);
        h2d(c, doo.p, out_off, n_tx + 1);
        h2d(c, dia.p, in_addr, n_in);
        h2d(c, doa.p, out_addr, n_out);
        bgl_graph *g = new bgl_graph();
        g->ctx = c;
        try {
            graph_build_device(g, n_tx, n_in, n_out, dio.p, dia.p, doo.p, doa.p);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    });
}

bgl_status bgl_graph_build_dev(bgl_ctx *c, int64_t n_tx, int64_t n_in, int64_t n_out, const int64_t *d_in_off,
                               const uint64_t *d_in_addr, const int64_t *d_out_off, const uint64_t *d_out_addr,
                               bgl_graph **out) {
    if (!c || !out) return BGL_EINVAL;
    return guarded(c, [&] {
        BGL_REQUIRE(n_tx >= 0 && n_in >= 0 && n_out >= 0, "sizes must be >= 0");
        BGL_REQUIRE(d_in_off && d_out_off, "offset arrays are NULL");
        BGL_REQUIRE((n_in == 0 || d_in_addr) && (n_out == 0 || d_out_addr), "address arrays are NULL");
        bgl_graph *g = new bgl_graph();
        g->ctx = c;
        try {
            graph_build_device(g, n_tx, n_in, n_out, d_in_off, d_in_addr, d_out_off, d_out_addr);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    });
}

bgl_status bgl_graph_from_edges(bgl_ctx *c, int64_t n, int64_t m, const int32_t *u, const int32_t *v,
                                bgl_graph **out) {
    if (!c || !out) return BGL_EINVAL;
    return guarded(c, [&] {
        BGL_REQUIRE(n >= 0 && n < (int64_t(1) << 31) - 1, "n out of range");
        BGL_REQUIRE(m >= 0, "m must be >= 0");
        BGL_REQUIRE(m == 0 || (u && v), "edge arrays are NULL");
        for (int64_t k = 0; k < m; ++k)
            BGL_REQUIRE(u[k] >= 0 && u[k] < n && v[k] >= 0 && v[k] < n, "edge endpoint out of range");
        DevBuf<int32_t> du(c->alloc, m), dv(c->alloc, m);
        h2d(c, du.p, u, m);
        h2d(c, dv.p, v, m);
        bgl_graph *g = new bgl_graph();
        g->ctx = c;
        try {
            graph_from_edges_device(g, n, m, du.p, dv.p);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    });
}

bgl_status bgl_graph_sizes(const bgl_graph *g, int64_t *n_nodes, int64_t *n_addr, int64_t *n_dir_edges,
                           int64_t *n_undir_edges) {
    if (!g) return BGL_EINVAL;
    if (n_nodes) *n_nodes = g->n;
    if (n_addr) *n_addr = g->n_addr;
    if (n_dir_edges) *n_dir_edges = g->n_dir;
    if (n_undir_edges) *n_undir_edges = g->n_undir;
    return BGL_OK;
}

bgl_status bgl_graph_addresses(const bgl_graph *g, uint64_t *key_out) {
    if (!g || !key_out) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        d2h(g->ctx, key_out, g->addr.p, g->n_addr);
        sync(g->ctx);
    });
}

bgl_status bgl_graph_edges(const bgl_graph *g, int32_t *src, int32_t *dst) {
    if (!g) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        if (src) d2h(g->ctx, src, g->src.p, g->n_dir);
        if (dst) d2h(g->ctx, dst, g->dst.p, g->n_dir);
        sync(g->ctx);
    });
}

bgl_status bgl_graph_csr(const bgl_graph *g, int64_t *off, int32_t *adj) {
    if (!g) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        if (off) d2h(g->ctx, off, g->off.p, g->n + 1);
        if (adj) d2h(g->ctx, adj, g->adj.p, 2 * g->n_undir);
        sync(g->ctx);
    });
}

bgl_status bgl_degrees(const bgl_graph *g, int32_t *deg_out) {
    if (!g || !deg_out) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        std::vector<int64_t> off(g->n + 1);
        d2h(g->ctx, off.data(), g->off.p, g->n + 1);
        sync(g->ctx);
        for (int64_t v = 0; v < g->n; ++v) deg_out[v] = (int32_t)(off[v + 1] - off[v]);
    });
}

bgl_status bgl_graph_destroy(bgl_graph *g) {
    if (!g) return BGL_OK;
    bgl_ctx *c = g->ctx;
    return guarded(c, [&] {
        sync(c);
        fa2_session_destroy(g->session);
        g->session = nullptr;
        delete g;
    });
}

bgl_status bgl_components(bgl_graph *g, int32_t *label_out, int64_t *n_comp) {
    if (!g) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        // a session refers to the component arrays being rebuilt
        fa2_session_destroy(g->session);
        g->session = nullptr;
        components_device(g);
        if (label_out) {
            d2h(g->ctx, label_out, g->label.p, g->n);
            sync(g->ctx);
        }
        if (n_comp) *n_comp = g->n_comp;
    });
}

bgl_status bgl_component_nodes(const bgl_graph *g, int64_t *comp_off, int32_t *comp_label, int32_t *nodes) {
    if (!g) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        require_comp(g);
        if (comp_off) std::copy(g->h_comp_off.begin(), g->h_comp_off.end(), comp_off);
        if (comp_label) d2h(g->ctx, comp_label, g->comp_label.p, g->n_comp);
        if (nodes) d2h(g->ctx, nodes, g->nodes.p, g->n);
        sync(g->ctx);
    });
}

bgl_status bgl_split(bgl_graph *g, int32_t kk_max_nodes, int64_t *n_kk, int64_t *n_fa2) {
    if (!g) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        split_device(g, kk_max_nodes);
        if (n_kk) *n_kk = g->n_kk;
        if (n_fa2) *n_fa2 = g->n_fa2;
    });
}

bgl_status bgl_layout(bgl_graph *g, const bgl_params *p, float *xy_out) {
    if (!g || !xy_out) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        DevBuf<float> out(g->ctx->alloc, 2 * g->n);
        layout_device(g, p, out.p);
        d2h(g->ctx, xy_out, out.p, 2 * g->n);
        sync(g->ctx);
    });
}

bgl_status bgl_layout_dev(bgl_graph *g, const bgl_params *p, float *d_xy_out) {
    if (!g || !d_xy_out) return BGL_EINVAL;
    return guarded(g->ctx, [&] { layout_device(g, p, d_xy_out); });
}

bgl_status bgl_kk_distances(bgl_graph *g, int64_t c, int32_t *d_out) {
    if (!g || !d_out) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        require_c(g, c);
        int64_t n = g->h_comp_off[c + 1] - g->h_comp_off[c];
        BGL_REQUIRE(n <= 255, "kk_distances: component has more than 255 nodes");
        DevBuf<int32_t> d(g->ctx->alloc, n * n);
        kk_distances(g, c, d.p);
        d2h(g->ctx, d_out, d.p, n * n);
        sync(g->ctx);
    });
}

bgl_status bgl_kk_run(bgl_graph *g, int64_t c, const bgl_params *p, float *xy_inout) {
    if (!g || !xy_inout) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        check_params(p);
        require_c(g, c);
        int64_t q0 = g->h_comp_off[c], n = g->h_comp_off[c + 1] - q0;
        BGL_REQUIRE(n <= 255, "kk_run: component has more than 255 nodes");
        DevBuf<float2> xy(g->ctx->alloc, n);
        h2d(g->ctx, xy.p, reinterpret_cast<const float2 *>(xy_inout), n);
        kk_layout(g, p, xy.p, q0, c, c + 1, false);
        d2h(g->ctx, reinterpret_cast<float2 *>(xy_inout), xy.p, n);
        sync(g->ctx);
    });
}

static bgl_status forces_common(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in, float *f_out,
                                int what) {
    if (!g || !xy_in || !f_out) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        check_params(p);
        require_c(g, c);
        int64_t q0 = g->h_comp_off[c], n = g->h_comp_off[c + 1] - q0;
        DevBuf<float2> xy(g->ctx->alloc, n), f(g->ctx->alloc, n);
        h2d(g->ctx, xy.p, reinterpret_cast<const float2 *>(xy_in), n);
        fa2_forces(g, p, xy.p, f.p, c, what);
        d2h(g->ctx, reinterpret_cast<float2 *>(f_out), f.p, n);
        sync(g->ctx);
    });
}

bgl_status bgl_fa2_forces(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in, float *f_out) {
    return forces_common(g, c, p, xy_in, f_out, 0);
}

bgl_status bgl_fa2_repulsion(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in, float *f_out) {
    return forces_common(g, c, p, xy_in, f_out, 1);
}

bgl_status bgl_fa2_step(bgl_graph *g, int64_t c, const bgl_params *p, int32_t iters, float *xy_inout,
                        double *stats_out) {
    if (!g || !xy_inout) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        check_params(p);
        require_c(g, c);
        BGL_REQUIRE(iters >= 0, "iters must be >= 0");
        int64_t q0 = g->h_comp_off[c], n = g->h_comp_off[c + 1] - q0;
        DevBuf<float2> xy(g->ctx->alloc, n);
        DevBuf<double> st(g->ctx->alloc, 3 * (size_t)std::max(iters, 1));
        h2d(g->ctx, xy.p, reinterpret_cast<const float2 *>(xy_inout), n);
        fa2_layout(g, p, xy.p, q0, c, c + 1, iters, stats_out ? st.p : nullptr);
        d2h(g->ctx, reinterpret_cast<float2 *>(xy_inout), xy.p, n);
        if (stats_out) d2h(g->ctx, stats_out, st.p, 3 * (size_t)iters);
        sync(g->ctx);
    });
}

bgl_status bgl_assemble(bgl_graph *g, const bgl_params *p, const float *xy_in, float *xy_out, int64_t *rank_out,
                        int64_t *parent_out, float *scale_out, float *radius_out, float *centre_out) {
    if (!g || !xy_in || !xy_out) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        check_params(p);
        require_comp(g);
        bgl_ctx *c = g->ctx;
        DevBuf<float2> in(c->alloc, std::max<int64_t>(g->n, 1)), comp(c->alloc, std::max<int64_t>(g->n, 1)),
            out(c->alloc, std::max<int64_t>(g->n, 1));
        h2d(c, in.p, reinterpret_cast<const float2 *>(xy_in), g->n);
        if (g->n > 0) {
            gather_xy_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, c->stream>>>(in.p, g->nodes.p, g->n, comp.p);
            BGL_LAUNCH_CHECK();
        }
        AssemblyOut info;
        assemble_device(g, p, comp.p, out.p, &info);
        d2h(c, reinterpret_cast<float2 *>(xy_out), out.p, g->n);
        sync(c);
        const int64_t C = g->n_comp;
        if (C > 0 && !info.rank.empty()) {
            if (rank_out) std::copy(info.rank.begin(), info.rank.end(), rank_out);
            if (parent_out) std::copy(info.parent0.begin(), info.parent0.end(), parent_out);
            if (scale_out) std::copy(info.scale.begin(), info.scale.end(), scale_out);
            if (radius_out) std::copy(info.radius.begin(), info.radius.end(), radius_out);
            if (centre_out)
                for (int64_t i = 0; i < C; ++i) {
                    centre_out[2 * i] = info.centre0[i].x;
                    centre_out[2 * i + 1] = info.centre0[i].y;
                }
        }
    });
}

bgl_status bgl_fa2_session_begin(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in) {
    if (!g || !xy_in) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        check_params(p);
        require_c(g, c);
        Fa2Session *s = fa2_session_create(g, p, c, reinterpret_cast<const float2 *>(xy_in));
        fa2_session_destroy(g->session);
        g->session = s;
    });
}

bgl_status bgl_fa2_session_advance(bgl_graph *g, int32_t iters, double *stats_out) {
    if (!g) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        if (!g->session) fail(BGL_ESTATE, "no ForceAtlas2 session: call bgl_fa2_session_begin or bgl_state_load");
        BGL_REQUIRE(iters >= 0, "iters must be >= 0");
        fa2_session_advance(g->session, iters, stats_out);
    });
}

bgl_status bgl_fa2_session_positions(bgl_graph *g, float *xy_out, int64_t *iters_done) {
    if (!g || !xy_out) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        if (!g->session) fail(BGL_ESTATE, "no ForceAtlas2 session: call bgl_fa2_session_begin or bgl_state_load");
        const int64_t k = fa2_session_positions(g->session, reinterpret_cast<float2 *>(xy_out));
        if (iters_done) *iters_done = k;
    });
}

bgl_status bgl_state_save(bgl_graph *g, void *buf, size_t *len) {
    if (!g || !len) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        if (!g->session) fail(BGL_ESTATE, "no ForceAtlas2 session to save");
        const size_t need = fa2_session_state_bytes(g->session);
        if (!buf) {
            *len = need;
            return;
        }
        BGL_REQUIRE(*len >= need, "state: buffer too small (query the size with buf = NULL)");
        fa2_session_save(g->session, buf);
        *len = need;
    });
}

bgl_status bgl_state_load(bgl_graph *g, const void *buf, size_t len) {
    if (!g || !buf) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        Fa2Session *s = fa2_session_load(g, buf, len);
        fa2_session_destroy(g->session);
        g->session = s;
    });
}

bgl_status bgl_fmm_stats(bgl_graph *g, int64_t c, const bgl_params *p, const float *xy_in, int32_t reps,
                         double *out) {
    if (!g || !xy_in || !out) return BGL_EINVAL;
    return guarded(g->ctx, [&] {
        check_params(p);
        require_c(g, c);
        BGL_REQUIRE(reps >= 1, "reps must be >= 1");
        int64_t q0 = g->h_comp_off[c], n = g->h_comp_off[c + 1] - q0;
        DevBuf<float2> xy(g->ctx->alloc, n);
        h2d(g->ctx, xy.p, reinterpret_cast<const float2 *>(xy_in), n);
        FmmPlan *pl = fmm_create(g, p, c);
        try {
            fmm_profile(pl, xy.p, q0, reps, out);
            int e = fmm_error(pl);
            if (e) fail(e & 1 ? BGL_ETIMEOUT : BGL_ENOMEM, "fmm_stats: device error bits " + std::to_string(e));
        } catch (...) {
            fmm_destroy(pl);
            throw;
        }
        fmm_destroy(pl);
    });
}

bgl_status bgl_fa2_iteration_noalloc(bgl_ctx *ctx, int64_t n, const int64_t *d_off, const int32_t *d_adj,
                                     const float *d_mass, float *d_xy, float *d_fprev, float *d_f, double *d_sg,
                                     const bgl_params *p) {
    if (!ctx) return BGL_EINVAL;
    return guarded(ctx, [&] {
        check_params(p);
        fa2_iteration_noalloc(ctx, n, d_off, d_adj, d_mass, reinterpret_cast<float2 *>(d_xy),
                              reinterpret_cast<float2 *>(d_fprev), reinterpret_cast<float2 *>(d_f), d_sg, p);
    });
}

int64_t bgl_launch_count(void) { return bgl::launch_count(); }

bgl_status bgl_peak_probe(bgl_ctx *c, double *out) {
    if (!c || !out) return BGL_EINVAL;
    return guarded(c, [&] { peak_probe(c, out); });
}

bgl_status bgl_debug_fail_alloc(bgl_ctx *c, int64_t after) {
    if (!c || after < -1) return BGL_EINVAL;
    c->alloc->fail_after.store(after);
    return BGL_OK;
}

}  // extern "C"
