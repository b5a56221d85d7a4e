// Internal declarations of the GB300 layout library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/bgl.h"

namespace bgl {

// ------------------------------------------------------------------ errors

struct Error : std::runtime_error {
    bgl_status status;
    Error(bgl_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] void fail(bgl_status s, const std::string &msg);
void check_params(const bgl_params *p);     // BGL_EINVAL on any parameter out of range
void check_cuda(cudaError_t e, const char *what, const char *file, int line);
#define BGL_CUDA(call) ::bgl::check_cuda((call), #call, __FILE__, __LINE__)
void count_launches(int64_t k);   // kernels launched through the library
int64_t launch_count();
#define BGL_LAUNCH_CHECK()                                                        \
    do {                                                                          \
        ::bgl::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__); \
        ::bgl::count_launches(1);                                                 \
    } while (0)
#define BGL_REQUIRE(cond, msg) \
    do {                       \
        if (!(cond)) ::bgl::fail(BGL_EINVAL, msg); \
    } while (0)

// ------------------------------------------------------------- tracing

// NVTX range over a host-side phase: every C-ABI call, and inside a layout
// the graph build, components, size split, Kamada-Kawai and ForceAtlas2
// phases and the FMM evaluation's phases.  A trace tool that is attached
// (NVTX injection) shows them on its timeline and maps them onto the
// kernels launched inside; without one a range costs a few nanoseconds.
// Ranges are host markers: work captured into a CUDA graph is marked where
// it was captured (once per layout), not where the graph replays it.
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
#else
struct Range {
    explicit Range(const char *) {}
};
#endif
#define BGL_RANGE_CAT2(a, b) a##b
#define BGL_RANGE_CAT(a, b) BGL_RANGE_CAT2(a, b)
#define BGL_RANGE(name) ::bgl::Range BGL_RANGE_CAT(bgl_range_, __LINE__)(name)

// ------------------------------------------------------------- allocator

// Caching device allocator: freed blocks are kept per context and reused
// for later requests of the same or a slightly smaller size, so repeated
// layouts of similar graphs do not call cudaMalloc/cudaFree.
class Allocator {
  public:
    // stream (may be null): new blocks come from the device's stream-ordered
    // pool on *stream; null: cudaMalloc
    explicit Allocator(int device, cudaStream_t *stream = nullptr) : device_(device), stream_(stream) {}
    ~Allocator();
    void *alloc(size_t bytes);
    void free(void *p);
    size_t cached_bytes() const { return cached_; }
    size_t live_bytes() const { return live_bytes_; }
    // largest live total since the last reset_peak
    size_t peak_bytes() const { return peak_bytes_; }
    void reset_peak() {
        std::lock_guard<std::mutex> lk(mu_);
        peak_bytes_ = live_bytes_;
    }
    void release_cache();
    // set while a stream capture is open: allocating then would bake a
    // block that is freed after the capture into the replayed graph
    bool forbid = false;
    // test aid (bgl_debug_fail_alloc): >= 0 makes the allocation after this
    // many more successful ones fail with BGL_ENOMEM; -1 never
    std::atomic<int64_t> fail_after{-1};

  private:
    int device_;
    cudaStream_t *stream_ = nullptr;
    std::mutex mu_;
    std::multimap<size_t, void *> free_;      // size -> block
    std::map<void *, size_t> live_;           // block -> size
    size_t cached_ = 0;
    size_t live_bytes_ = 0, peak_bytes_ = 0;
};

// Device array owned through the context allocator.
template <typename T>
struct DevBuf {
    Allocator *a = nullptr;
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(Allocator *al, size_t count) { reset(al, count); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : a(o.a), p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); a = o.a; p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void reset(Allocator *al, size_t count) {
        release();
        a = al;
        n = count;
        p = static_cast<T *>(al->alloc(sizeof(T) * (count > 0 ? count : 1)));
    }
    // grow-only: keeps the block when it is already big enough
    void ensure(Allocator *al, size_t count) {
        if (p && count <= n) return;
        reset(al, count);
    }
    void release() {
        if (p && a) a->free(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return sizeof(T) * n; }
};

}  // namespace bgl

// ------------------------------------------------------------- handles

struct bgl_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    bgl::Allocator *alloc = nullptr;
    std::string last_error;
    int *d_flag = nullptr;        // device error/flag words (4 ints): [0] per-call checks, [1] ForceAtlas2
                                  // runs, [2] allocation-free iterations (read by bgl_ctx_sync)
    int *h_flag = nullptr;        // pinned mirror
    unsigned char *noalloc_scratch = nullptr;   // device address of the allocation-free scratch array
    // autotuner choices: exact-repulsion targets per thread by log2 of the pairs
    std::mutex tune_mu;
    std::map<int, int> tune_exact;
    // measured exact/FMM choice by component size octave (fmm_min_nodes = -1)
    std::map<int, bool> tune_fmm;
};

namespace bgl {
// device address of the allocation-free iteration's scratch array on the
// current device (cudaGetSymbolAddress; allocates nothing)
void *noalloc_scratch_address();
// ALU throughput probes (probe.cu): out[5] = FP32 lanes, MUFU reciprocals and
// pairs per SM clock, the SM count, and packed FP32x2 pairs per SM clock
void peak_probe(bgl_ctx *c, double *out);
struct Fa2Session;
void fa2_session_destroy(Fa2Session *s);
}  // namespace bgl

struct bgl_graph {
    bgl_ctx *ctx = nullptr;
    bgl::Fa2Session *session = nullptr;   // resumable ForceAtlas2 run (bgl_fa2_session_*)
    int64_t n_tx = 0, n_addr = 0, n = 0;
    int64_t n_dir = 0, n_undir = 0;
    bgl::DevBuf<uint64_t> addr;         // [n_addr] address keys in id order
    bgl::DevBuf<int32_t> src, dst;      // [n_dir] directed edges sorted by (src, dst)
    bgl::DevBuf<int64_t> off;           // [n+1] undirected CSR
    bgl::DevBuf<int32_t> adj;           // [2 n_undir]
    // components (Section 4)
    bool has_comp = false;
    int64_t n_comp = 0;
    bgl::DevBuf<int32_t> label;         // [n]
    bgl::DevBuf<int64_t> comp_off;      // [n_comp+1] in component order
    bgl::DevBuf<int32_t> comp_label;    // [n_comp]
    bgl::DevBuf<int32_t> nodes;         // [n] node ids in component order
    bgl::DevBuf<int32_t> pos;           // [n] component-order position of each node id
    bgl::DevBuf<int32_t> node_comp;     // [n] component index of each component-order position
    bgl::DevBuf<int64_t> coff;          // [n+1] CSR in component order (local = position)
    bgl::DevBuf<int32_t> cadj;          // [2 n_undir]
    bgl::DevBuf<float> mass;            // [n] degree + 1, component order
    bgl::DevBuf<int32_t> seed_id;       // [n] id seeding each node's initial position (empty: the node id)
    std::vector<int64_t> h_comp_off;    // host copy of comp_off
    // split
    int32_t kk_max = -1;
    int64_t n_kk = 0, n_fa2 = 0;
};

namespace bgl {

// ------------------------------------------------------------- primitives (sort.cu)

// Exclusive prefix sum of n values (in may equal out).  Returns nothing;
// total (if not null) receives the sum on the device.
void scan_exclusive_i64(bgl_ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *d_total);
void scan_exclusive_i32(bgl_ctx *c, const int32_t *in, int32_t *out, int64_t n, int32_t *d_total);

// Stable LSD radix sort of (key, value) pairs on bits [0, bits) of the key.
// keys/vals are sorted in place (with internal double buffers).  vals may be null.
void radix_sort_u64(bgl_ctx *c, uint64_t *keys, uint32_t *vals, int64_t n, int bits);
void radix_sort_u32(bgl_ctx *c, uint32_t *keys, uint32_t *vals, int64_t n, int bits);

// Preallocated temporaries for sorting up to `cap` 32-bit keys with values,
// so that a sort can run inside a captured CUDA graph.
struct SortWorkspace {
    DevBuf<uint32_t> keys, vals, keys2, vals2;   // two scratch buffers for the passes
    DevBuf<int32_t> hist, tiles;
    int64_t cap = 0;
    void reserve(Allocator *a, int64_t n, cudaStream_t s);
};
// With gpts, the last pass writes gpts[i] = {gxy[v].x, gxy[v].y, gmass[v], v}
// (v = the value of sorted key i, as int bits) instead of the sorted values.
void radix_sort_u32_ws(bgl_ctx *c, SortWorkspace &ws, uint32_t *keys, uint32_t *vals, int64_t n, int bits,
                       const float2 *gxy = nullptr, const float *gmass = nullptr, float4 *gpts = nullptr);
// nonzero if a bounded wait of a workspace sort gave up (synchronises)
int sort_workspace_error(bgl_ctx *c, SortWorkspace &ws);
// The same sort in two halves, so that a caller's kernel can count the digit
// histograms while it makes the keys: radix_sort_u32_ws_begin clears the
// counts and returns them; every block of the caller's kernel (256 threads)
// then calls os_block_hist (sort_hist.cuh) on its keys; and
// radix_sort_u32_ws_scatter runs the four passes.
struct OsHist {
    uint32_t *hist;      // 4 x 256 digit counts
    uint32_t *base;      // 4 x 256 exclusive digit bases (written by the last block)
    unsigned *counter;   // arrival count of the blocks (reset by the last block)
    unsigned *tickets;   // 4 pass tickets
    uint32_t *status;    // 4 x ntiles x 256 look-back status words
    int64_t ntiles;      // tiles of 256 x 16 keys
};
// With clear = false the caller zeroes hist and tickets in a kernel that
// runs before its histogram kernel, and each block of the histogram kernel
// (one per tile) zeroes its tile's status words (os_clear_status).
OsHist radix_sort_u32_ws_begin(bgl_ctx *c, SortWorkspace &ws, int64_t n, bool clear = true);
// The bounded waits of the scatter passes: err (null: the workspace's own
// word) receives bit 1 when a wait gives up, and a pass started after that
// does nothing; spin is the poll limit (0: the default, about half a second
// of polling); stall_first = 1 makes the first tile of every pass withhold
// its counts, so that the waits on it run out -- a test aid for the
// failure path (BGL_ETIMEOUT), memory-safe because a tile that gives up
// still writes inside [0, n).
struct OsWait {
    int *err = nullptr;
    long long spin = 0;
    int stall_first = 0;
};
// d_skip (device int, may be null = 0): the passes below *d_skip (0 or 2)
// return at once, so the keys end up ordered by their top 32 - 8 * skip
// bits only (stable: equal top bits keep the input order).  Read by each
// pass when it starts.
void radix_sort_u32_ws_scatter(bgl_ctx *c, SortWorkspace &ws, uint32_t *keys, uint32_t *vals, int64_t n,
                               const float2 *gxy = nullptr, const float *gmass = nullptr, float4 *gpts = nullptr,
                               const int *d_skip = nullptr, OsWait wait = OsWait());

int bits_for(uint64_t max_value);   // number of bits needed to hold max_value

// ------------------------------------------------------------- graph.cu

void graph_build_device(bgl_graph *g, int64_t n_tx, int64_t n_in, int64_t n_out, const int64_t *d_in_off,
                        const uint64_t *d_in_addr, const int64_t *d_out_off, const uint64_t *d_out_addr);
void graph_from_edges_device(bgl_graph *g, int64_t n, int64_t m, const int32_t *d_u, const int32_t *d_v);
void components_device(bgl_graph *g);
void split_device(bgl_graph *g, int32_t kk_max);

// ------------------------------------------------------------- layout kernels

// initial positions (SplitMix64 per node id) for component-order range
// [q0, q1), written to xy[q - q0]
void init_positions(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t q0, int64_t q1);

// KK on components [c0, c1) (each at most 255 nodes); xy[q - qbase] holds the
// position of component-order position q.  If init is true the kernel first
// sets SplitMix64 initial positions scaled by l * diam / 2; otherwise it
// starts from xy.
void kk_layout(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t qbase, int64_t c0, int64_t c1, bool init);
// KK launches split in preparation (all scratch allocated) and launches that
// allocate nothing, one per size class, on any stream
struct KkRun;
KkRun *kk_prepare(bgl_graph *g, int64_t c0, int64_t c1);
void kk_destroy(KkRun *run);
int kk_classes(const KkRun *run);
void kk_enqueue(const KkRun *run, int i, const bgl_params *p, float2 *xy, int64_t qbase, bool init, int sweeps,
                int32_t *d_out, cudaStream_t s);
void kk_distances(bgl_graph *g, int64_t c, int32_t *d_out_dev);

// ForceAtlas2 on components [c0, c1) (exact or FMM per component);
// xy[q - qbase] holds the position of component-order position q;
// `iters` iterations from F_{-1} = 0, s_G = 1.  d_stats (device, may be
// null): swing, traction, s_G per iteration of component c0.
// Work that runs beside the ForceAtlas2 iterations: enqueued on the given
// stream (it may fork to streams of its own and must join back); with the
// device-side loop it is captured and launched in the same graph.
using SideWork = std::function<void(cudaStream_t)>;
void fa2_layout(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t qbase, int64_t c0, int64_t c1, int iters,
                double *d_stats, const SideWork &side = SideWork());
// Assembly of the component layouts into one frame (assemble.cu, Section 4):
// xy_comp[q] the per-component layout at component-order position q,
// xy_out the assembled frame in node-id order; info (may be null) receives
// per-component results for parity checks.
struct AssemblyOut {
    int levels = 0;
    std::vector<int64_t> rank, parent0;
    std::vector<float> scale, radius;
    std::vector<float2> centre0;
};
void assemble_device(bgl_graph *g, const bgl_params *p, const float2 *xy_comp, float2 *xy_out_nodes,
                     AssemblyOut *info);

// Resumable ForceAtlas2 run on one component (fa2.cu): positions,
// F_{t-1}, s_G and the iteration count stay on the device between calls.
Fa2Session *fa2_session_create(bgl_graph *g, const bgl_params *p, int64_t c, const float2 *h_xy);
void fa2_session_advance(Fa2Session *s, int iters, double *h_stats);
int64_t fa2_session_positions(Fa2Session *s, float2 *h_xy);     // returns the iterations done
size_t fa2_session_state_bytes(const Fa2Session *s);
void fa2_session_save(Fa2Session *s, void *buf);
Fa2Session *fa2_session_load(bgl_graph *g, const void *buf, size_t len);

// the whole layout (split, KK, ForceAtlas2, assembly if asked) into a device
// array in node-id order (api.cu)
void layout_device(bgl_graph *g, const bgl_params *p, float *d_xy_out);

// one force evaluation on component c, xy and f indexed by q - comp_off[c];
// what: 0 total force, 1 repulsion only
void fa2_forces(bgl_graph *g, const bgl_params *p, const float2 *xy, float2 *f, int64_t c, int what);
// true if component c of n nodes uses the FMM under p
bool use_fmm(const bgl_params *p, int64_t n);

// one exact-repulsion ForceAtlas2 iteration on caller device arrays, with
// static scratch (noalloc.cu)
void fa2_iteration_noalloc(bgl_ctx *c, int64_t n, const int64_t *d_off, const int32_t *d_adj, const float *d_mass,
                           float2 *d_xy, float2 *d_fprev, float2 *d_f, double *d_sg, const bgl_params *p);

}  // namespace bgl
