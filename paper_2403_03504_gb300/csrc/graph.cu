// Graph construction (Section 2), connected components and the size split
// (Section 4), all on the device with sort/scan primitives.
//
// Address ids by first appearance: the endpoints are laid out in scan order
// (tx 0 inputs, tx 0 outputs, tx 1 inputs, ...); a stable radix sort of
// (address key, scan position) groups equal keys with the first appearance
// at the head of each run; flagging heads at their scan position and taking
// an exclusive scan of the flags numbers the addresses in first-appearance
// order.  Directed and undirected edge sets are deduplicated by sorting
// packed (src, dst) keys.  Components: atomicMin hooking of roots plus
// pointer jumping until no edge joins two roots, which leaves every node
// labelled with the smallest id of its component.
#include "bgl_internal.cuh"

namespace bgl {

namespace {

constexpr int TPB = 256;

inline unsigned blocks_for(int64_t n, int t = TPB) {
    int64_t b = (n + t - 1) / t;
    return (unsigned)(b > 0 ? b : 1);
}

__global__ void validate_offsets_kernel(const int64_t *in_off, const int64_t *out_off, int64_t T, int64_t n_in,
                                        int64_t n_out, int *flag) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > T) return;
    bool bad = false;
    if (t == 0) bad = in_off[0] != 0 || out_off[0] != 0;
    else bad = in_off[t] < in_off[t - 1] || out_off[t] < out_off[t - 1];
    if (t == T) bad = bad || in_off[T] != n_in || out_off[T] != n_out;
    if (bad) atomicOr(flag, 1);
}

// endpoint arrays indexed by scan position
__global__ void expand_endpoints_kernel(const int64_t *__restrict__ in_off, const uint64_t *__restrict__ in_addr,
                                        const int64_t *__restrict__ out_off, const uint64_t *__restrict__ out_addr,
                                        int64_t T, uint64_t *__restrict__ ep_key, int32_t *__restrict__ ep_tx,
                                        uint8_t *__restrict__ ep_out, uint32_t *__restrict__ ep_pos) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int64_t i0 = in_off[t], i1 = in_off[t + 1], o0 = out_off[t], o1 = out_off[t + 1];
    int64_t base = i0 + o0;
    for (int64_t j = 0; j < i1 - i0; ++j) {
        int64_t p = base + j;
        ep_key[p] = in_addr[i0 + j];
        ep_tx[p] = (int32_t)t;
        ep_out[p] = 0;
        ep_pos[p] = (uint32_t)p;
    }
    base += i1 - i0;
    for (int64_t j = 0; j < o1 - o0; ++j) {
        int64_t p = base + j;
        ep_key[p] = out_addr[o0 + j];
        ep_tx[p] = (int32_t)t;
        ep_out[p] = 1;
        ep_pos[p] = (uint32_t)p;
    }
}

template <typename K>
__global__ void head_flags_kernel(const K *__restrict__ k, int64_t n, int32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}

__global__ void mark_first_kernel(const int32_t *__restrict__ head, const uint32_t *__restrict__ spos, int64_t n,
                                  int32_t *__restrict__ isfirst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (head[i]) isfirst[spos[i]] = 1;
}

// run u of sorted index i = (exclusive scan of heads)[i] + head[i] - 1
__global__ void run_rank_kernel(const int32_t *__restrict__ head, const int32_t *__restrict__ hscan,
                                const uint32_t *__restrict__ spos, const int32_t *__restrict__ rank_at_pos,
                                const uint64_t *__restrict__ skey, int64_t n, int32_t *__restrict__ runrank,
                                uint64_t *__restrict__ addr_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !head[i]) return;
    int32_t r = rank_at_pos[spos[i]];
    runrank[hscan[i]] = r;
    addr_out[r] = skey[i];
}

__global__ void endpoint_edges_kernel(const int32_t *__restrict__ head, const int32_t *__restrict__ hscan,
                                      const uint32_t *__restrict__ spos, const int32_t *__restrict__ runrank,
                                      const int32_t *__restrict__ ep_tx, const uint8_t *__restrict__ ep_out,
                                      int64_t n, int64_t T, int b, uint64_t *__restrict__ ekey) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t u = hscan[i] + head[i] - 1;
    uint32_t p = spos[i];
    uint64_t a = (uint64_t)(T + runrank[u]);
    uint64_t t = (uint64_t)ep_tx[p];
    // Section 2: address -> tx for an input, tx -> address for an output
    ekey[p] = ep_out[p] ? ((t << b) | a) : ((a << b) | t);
}

template <typename K>
__global__ void compact_kernel(const K *__restrict__ in, const int32_t *__restrict__ flag,
                               const int32_t *__restrict__ fscan, int64_t n, K *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    out[fscan[i]] = in[i];
}

__global__ void unpack_edges_kernel(const uint64_t *__restrict__ k, int64_t m, int b, int32_t *__restrict__ src,
                                    int32_t *__restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t mask = (uint64_t(1) << b) - 1;
    src[i] = (int32_t)(k[i] >> b);
    dst[i] = (int32_t)(k[i] & mask);
}

__global__ void pack_edges_kernel(const int32_t *__restrict__ u, const int32_t *__restrict__ v, int64_t m, int b,
                                  uint64_t *__restrict__ k) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    k[i] = ((uint64_t)(uint32_t)u[i] << b) | (uint64_t)(uint32_t)v[i];
}

// both directions of each directed edge; self-loops flagged out
__global__ void undirected_keys_kernel(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t m,
                                       int b, uint64_t *__restrict__ k, int32_t *__restrict__ keep) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t s = (uint32_t)src[i], d = (uint32_t)dst[i];
    k[2 * i] = (s << b) | d;
    k[2 * i + 1] = (d << b) | s;
    int ok = s != d;
    keep[2 * i] = ok;
    keep[2 * i + 1] = ok;
}

__global__ void csr_rows_kernel(const uint64_t *__restrict__ k, int64_t m, int b, int32_t *__restrict__ adj,
                                int64_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t mask = (uint64_t(1) << b) - 1;
    adj[i] = (int32_t)(k[i] & mask);
    atomicAdd((unsigned long long *)&cnt[k[i] >> b], 1ull);
}

__global__ void iota_kernel(int32_t *a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}

// ---------------------------------------------------------------- components

__device__ __forceinline__ int32_t find_root(const int32_t *parent, int32_t v) {
    int32_t p = parent[v];
    while (p != v) {
        v = p;
        p = parent[v];
    }
    return v;
}

__global__ void hook_kernel(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t m,
                            int32_t *parent, int *changed) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int32_t a = find_root(parent, src[i]);
    int32_t b = find_root(parent, dst[i]);
    if (a == b) return;
    int32_t lo = a < b ? a : b, hi = a < b ? b : a;
    atomicMin(&parent[hi], lo);
    *changed = 1;
}

__global__ void jump_kernel(int32_t *parent, int64_t n) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    parent[v] = find_root(parent, (int32_t)v);
}

__global__ void comp_size_kernel(const int32_t *__restrict__ label, int64_t n, int32_t *__restrict__ size) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) atomicAdd(&size[label[v]], 1);
}

__global__ void root_flag_kernel(const int32_t *__restrict__ label, int64_t n, int32_t *__restrict__ flag) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flag[v] = label[v] == (int32_t)v;
}

// key orders components by size descending, then label ascending
__global__ void comp_key_kernel(const int32_t *__restrict__ flag, const int32_t *__restrict__ fscan,
                                const int32_t *__restrict__ size, int64_t n, int b, uint64_t *__restrict__ key) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || !flag[v]) return;
    key[fscan[v]] = ((uint64_t)(n - size[v]) << b) | (uint64_t)v;
}

__global__ void comp_unpack_kernel(const uint64_t *__restrict__ key, int64_t nc, int64_t n, int b,
                                   int32_t *__restrict__ comp_label, int64_t *__restrict__ comp_size,
                                   int32_t *__restrict__ cidx) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    uint64_t mask = (uint64_t(1) << b) - 1;
    int32_t l = (int32_t)(key[c] & mask);
    comp_label[c] = l;
    comp_size[c] = n - (int64_t)(key[c] >> b);
    cidx[l] = (int32_t)c;
}

__global__ void node_key_kernel(const int32_t *__restrict__ label, const int32_t *__restrict__ cidx, int64_t n,
                                uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    key[v] = (uint32_t)cidx[label[v]];
    val[v] = (uint32_t)v;
}

__global__ void node_order_kernel(const uint32_t *__restrict__ ckey, const uint32_t *__restrict__ node, int64_t n,
                                  const int64_t *__restrict__ off, int32_t *__restrict__ nodes,
                                  int32_t *__restrict__ pos, int32_t *__restrict__ node_comp,
                                  int64_t *__restrict__ cdeg, float *__restrict__ mass) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    int32_t v = (int32_t)node[q];
    nodes[q] = v;
    pos[v] = (int32_t)q;
    node_comp[q] = (int32_t)ckey[q];
    int64_t d = off[v + 1] - off[v];
    cdeg[q] = d;
    mass[q] = (float)(d + 1);   // ForceAtlas2 mass: degree + 1
}

// the last q in [lo, hi] with coff[q] <= k (coff non-decreasing, coff[lo] <= k)
__device__ __forceinline__ int64_t owner_of(const int64_t *__restrict__ coff, int64_t lo, int64_t hi, int64_t k) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (coff[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Component-order adjacency, one thread per entry k of the m2 entries (so a
// hub's list is spread over many threads): its node q is the one whose range
// [coff[q], coff[q + 1]) holds k, found by a binary search inside the nodes
// of the block's entries; cadj[k] = pos[adj[off[v] + k - coff[q]]], v =
// nodes[q].
__global__ void comp_csr_kernel(const int32_t *__restrict__ nodes, const int32_t *__restrict__ pos,
                                const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                const int64_t *__restrict__ coff, int64_t n, int64_t m2, int32_t *__restrict__ cadj) {
    __shared__ int64_t qrange[2];
    const int64_t k0 = (int64_t)blockIdx.x * blockDim.x;
    if (k0 >= m2) return;
    if (threadIdx.x < 2) {
        const int64_t kk = threadIdx.x == 0 ? k0 : min(m2, k0 + (int64_t)blockDim.x) - 1;
        qrange[threadIdx.x] = owner_of(coff, 0, n - 1, kk);
    }
    __syncthreads();
    const int64_t k = k0 + threadIdx.x;
    if (k >= m2) return;
    const int64_t q = owner_of(coff, qrange[0], qrange[1], k);
    const int32_t v = nodes[q];
    cadj[k] = pos[adj[off[v] + (k - coff[q])]];
}

}  // namespace

// Deduplicated directed edges from packed keys (src << b | dst), then the
// undirected CSR.  Consumes ekey (sorted in place).
static void finish_edges(bgl_graph *g, uint64_t *ekey, int64_t m, int b) {
    bgl_ctx *c = g->ctx;
    Allocator *A = c->alloc;
    cudaStream_t s = c->stream;
    radix_sort_u64(c, ekey, nullptr, m, 2 * b);
    DevBuf<int32_t> hd(A, m), hs(A, m);
    DevBuf<int32_t> tot(A, 1);
    head_flags_kernel<uint64_t><<<blocks_for(m), TPB, 0, s>>>(ekey, m, hd.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i32(c, hd.p, hs.p, m, tot.p);
    int32_t md = 0;
    BGL_CUDA(cudaMemcpyAsync(&md, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    DevBuf<uint64_t> uk(A, md);
    compact_kernel<uint64_t><<<blocks_for(m), TPB, 0, s>>>(ekey, hd.p, hs.p, m, uk.p);
    BGL_LAUNCH_CHECK();
    g->n_dir = md;
    g->src.reset(A, md);
    g->dst.reset(A, md);
    unpack_edges_kernel<<<blocks_for(md), TPB, 0, s>>>(uk.p, md, b, g->src.p, g->dst.p);
    BGL_LAUNCH_CHECK();

    // undirected: both directions, drop self-loops, sort, dedupe, CSR
    int64_t m2 = 2 * md;
    DevBuf<uint64_t> k2(A, m2);
    DevBuf<int32_t> keep(A, m2), ks(A, m2);
    undirected_keys_kernel<<<blocks_for(md), TPB, 0, s>>>(g->src.p, g->dst.p, md, b, k2.p, keep.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i32(c, keep.p, ks.p, m2, tot.p);
    int32_t mk = 0;
    BGL_CUDA(cudaMemcpyAsync(&mk, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    DevBuf<uint64_t> k3(A, mk);
    compact_kernel<uint64_t><<<blocks_for(m2), TPB, 0, s>>>(k2.p, keep.p, ks.p, m2, k3.p);
    BGL_LAUNCH_CHECK();
    radix_sort_u64(c, k3.p, nullptr, mk, 2 * b);
    DevBuf<int32_t> h3(A, mk), s3(A, mk);
    head_flags_kernel<uint64_t><<<blocks_for(mk), TPB, 0, s>>>(k3.p, mk, h3.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i32(c, h3.p, s3.p, mk, tot.p);
    int32_t mu = 0;
    BGL_CUDA(cudaMemcpyAsync(&mu, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    DevBuf<uint64_t> k4(A, mu);
    compact_kernel<uint64_t><<<blocks_for(mk), TPB, 0, s>>>(k3.p, h3.p, s3.p, mk, k4.p);
    BGL_LAUNCH_CHECK();
    g->n_undir = mu / 2;
    g->adj.reset(A, mu);
    g->off.reset(A, g->n + 1);
    DevBuf<int64_t> cnt(A, g->n + 1);
    BGL_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * (g->n + 1), s));
    csr_rows_kernel<<<blocks_for(mu), TPB, 0, s>>>(k4.p, mu, b, g->adj.p, cnt.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i64(c, cnt.p, g->off.p, g->n + 1, nullptr);
    g->has_comp = false;
}

void graph_build_device(bgl_graph *g, int64_t T, int64_t n_in, int64_t n_out, const int64_t *d_in_off,
                        const uint64_t *d_in_addr, const int64_t *d_out_off, const uint64_t *d_out_addr) {
    BGL_RANGE("graph build (Section 2)");
    bgl_ctx *c = g->ctx;
    Allocator *A = c->alloc;
    cudaStream_t s = c->stream;
    const int64_t M = n_in + n_out;
    BGL_REQUIRE(T >= 0 && n_in >= 0 && n_out >= 0, "graph_build: negative size");
    BGL_REQUIRE(T + M < (int64_t(1) << 31) - 1, "graph_build: more than 2^31 nodes or endpoints");

    BGL_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
    validate_offsets_kernel<<<blocks_for(T + 1), TPB, 0, s>>>(d_in_off, d_out_off, T, n_in, n_out, c->d_flag);
    BGL_LAUNCH_CHECK();
    BGL_CUDA(cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    if (c->h_flag[0]) fail(BGL_EINVAL, "graph_build: offsets must start at 0, never decrease and end at n_in/n_out");

    g->n_tx = T;
    DevBuf<uint64_t> key(A, M);
    DevBuf<int32_t> ep_tx(A, M);
    DevBuf<uint8_t> ep_out(A, M);
    DevBuf<uint32_t> spos(A, M);
    if (T > 0) {
        expand_endpoints_kernel<<<blocks_for(T), TPB, 0, s>>>(d_in_off, d_in_addr, d_out_off, d_out_addr, T, key.p,
                                                              ep_tx.p, ep_out.p, spos.p);
        BGL_LAUNCH_CHECK();
    }
    // stable sort by key: heads of runs are first appearances
    radix_sort_u64(c, key.p, spos.p, M, 64);
    DevBuf<int32_t> head(A, M), hscan(A, M), isfirst(A, M), rank(A, M), tot(A, 1);
    head_flags_kernel<uint64_t><<<blocks_for(M), TPB, 0, s>>>(key.p, M, head.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i32(c, head.p, hscan.p, M, tot.p);
    int32_t U = 0;
    BGL_CUDA(cudaMemcpyAsync(&U, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaMemsetAsync(isfirst.p, 0, sizeof(int32_t) * (M > 0 ? M : 1), s));
    mark_first_kernel<<<blocks_for(M), TPB, 0, s>>>(head.p, spos.p, M, isfirst.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i32(c, isfirst.p, rank.p, M, nullptr);
    BGL_CUDA(cudaStreamSynchronize(s));
    g->n_addr = U;
    g->n = T + U;
    g->addr.reset(A, U);
    DevBuf<int32_t> runrank(A, U);
    run_rank_kernel<<<blocks_for(M), TPB, 0, s>>>(head.p, hscan.p, spos.p, rank.p, key.p, M, runrank.p, g->addr.p);
    BGL_LAUNCH_CHECK();
    const int b = bits_for((uint64_t)(g->n > 0 ? g->n - 1 : 0)) > 0 ? bits_for((uint64_t)(g->n - 1)) : 1;
    DevBuf<uint64_t> ekey(A, M);
    endpoint_edges_kernel<<<blocks_for(M), TPB, 0, s>>>(head.p, hscan.p, spos.p, runrank.p, ep_tx.p, ep_out.p, M, T,
                                                        b, ekey.p);
    BGL_LAUNCH_CHECK();
    // release endpoint buffers before the edge sorts
    key.release(); ep_tx.release(); ep_out.release(); spos.release();
    head.release(); hscan.release(); isfirst.release(); rank.release(); runrank.release();
    finish_edges(g, ekey.p, M, b);
}

void graph_from_edges_device(bgl_graph *g, int64_t n, int64_t m, const int32_t *d_u, const int32_t *d_v) {
    BGL_RANGE("graph from edges");
    bgl_ctx *c = g->ctx;
    g->n_tx = 0;
    g->n_addr = 0;
    g->n = n;
    const int b = n > 1 ? bits_for((uint64_t)(n - 1)) : 1;
    DevBuf<uint64_t> ekey(c->alloc, m);
    if (m > 0) {
        pack_edges_kernel<<<blocks_for(m), TPB, 0, c->stream>>>(d_u, d_v, m, b, ekey.p);
        BGL_LAUNCH_CHECK();
    }
    finish_edges(g, ekey.p, m, b);
}

void components_device(bgl_graph *g) {
    BGL_RANGE("components (Section 4)");
    bgl_ctx *c = g->ctx;
    Allocator *A = c->alloc;
    cudaStream_t s = c->stream;
    const int64_t n = g->n;
    g->label.reset(A, n);
    iota_kernel<<<blocks_for(n), TPB, 0, s>>>(g->label.p, n);
    BGL_LAUNCH_CHECK();
    int rounds = 0;
    for (;;) {
        BGL_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
        if (g->n_dir > 0) {
            hook_kernel<<<blocks_for(g->n_dir), TPB, 0, s>>>(g->src.p, g->dst.p, g->n_dir, g->label.p, c->d_flag);
            BGL_LAUNCH_CHECK();
        }
        jump_kernel<<<blocks_for(n), TPB, 0, s>>>(g->label.p, n);
        BGL_LAUNCH_CHECK();
        BGL_CUDA(cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaStreamSynchronize(s));
        if (!c->h_flag[0]) break;
        if (++rounds > 64 + 2 * bits_for((uint64_t)n)) fail(BGL_ETIMEOUT, "components: hooking did not converge");
    }
    // sizes, component order (size desc, label asc)
    DevBuf<int32_t> size(A, n), flag(A, n), fscan(A, n), tot(A, 1);
    BGL_CUDA(cudaMemsetAsync(size.p, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));
    comp_size_kernel<<<blocks_for(n), TPB, 0, s>>>(g->label.p, n, size.p);
    root_flag_kernel<<<blocks_for(n), TPB, 0, s>>>(g->label.p, n, flag.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i32(c, flag.p, fscan.p, n, tot.p);
    int32_t nc = 0;
    BGL_CUDA(cudaMemcpyAsync(&nc, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    g->n_comp = nc;
    const int b = n > 0 ? (bits_for((uint64_t)n) > 0 ? bits_for((uint64_t)n) : 1) : 1;
    DevBuf<uint64_t> ckey(A, nc);
    comp_key_kernel<<<blocks_for(n), TPB, 0, s>>>(flag.p, fscan.p, size.p, n, b, ckey.p);
    BGL_LAUNCH_CHECK();
    radix_sort_u64(c, ckey.p, nullptr, nc, 2 * b);
    g->comp_label.reset(A, nc);
    g->comp_off.reset(A, nc + 1);
    DevBuf<int64_t> csize(A, nc + 1);
    DevBuf<int32_t> cidx(A, n);
    comp_unpack_kernel<<<blocks_for(nc), TPB, 0, s>>>(ckey.p, nc, n, b, g->comp_label.p, csize.p, cidx.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i64(c, csize.p, g->comp_off.p, nc, g->comp_off.p + nc);
    // nodes grouped by component, ascending id inside (stable sort by index)
    DevBuf<uint32_t> nkey(A, n), nval(A, n);
    node_key_kernel<<<blocks_for(n), TPB, 0, s>>>(g->label.p, cidx.p, n, nkey.p, nval.p);
    BGL_LAUNCH_CHECK();
    radix_sort_u32(c, nkey.p, nval.p, n, nc > 1 ? bits_for((uint64_t)(nc - 1)) : 0);
    g->nodes.reset(A, n);
    g->pos.reset(A, n);
    g->node_comp.reset(A, n);
    g->mass.reset(A, n);
    g->coff.reset(A, n + 1);
    DevBuf<int64_t> cdeg(A, n + 1);
    node_order_kernel<<<blocks_for(n), TPB, 0, s>>>(nkey.p, nval.p, n, g->off.p, g->nodes.p, g->pos.p,
                                                    g->node_comp.p, cdeg.p, g->mass.p);
    BGL_LAUNCH_CHECK();
    scan_exclusive_i64(c, cdeg.p, g->coff.p, n, g->coff.p + n);
    g->cadj.reset(A, 2 * g->n_undir);
    if (g->n_undir > 0) {
        comp_csr_kernel<<<blocks_for(2 * g->n_undir), TPB, 0, s>>>(g->nodes.p, g->pos.p, g->off.p, g->adj.p,
                                                                   g->coff.p, n, 2 * g->n_undir, g->cadj.p);
        BGL_LAUNCH_CHECK();
    }
    g->h_comp_off.resize(nc + 1);
    BGL_CUDA(cudaMemcpyAsync(g->h_comp_off.data(), g->comp_off.p, sizeof(int64_t) * (nc + 1),
                             cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    g->has_comp = true;
    g->kk_max = -1;
}

void split_device(bgl_graph *g, int32_t kk_max) {
    BGL_RANGE("size split (Section 4)");
    if (!g->has_comp) fail(BGL_ESTATE, "split: run bgl_components first");
    BGL_REQUIRE(kk_max >= 0, "split: kk_max_nodes must be >= 0");
    // components are sorted by size descending: FA2 ones come first
    int64_t lo = 0, hi = g->n_comp;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        int64_t sz = g->h_comp_off[mid + 1] - g->h_comp_off[mid];
        if (sz > kk_max) lo = mid + 1;
        else hi = mid;
    }
    g->n_fa2 = lo;
    g->n_kk = g->n_comp - lo;
    g->kk_max = kk_max;
}

}  // namespace bgl
