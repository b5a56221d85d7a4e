// Kamada-Kawai layout of small components (Section 3.1) and the initial
// positions shared by every component.
//
// A group of G lanes lays out one component of at most 255 nodes; lane gl
// owns the nodes gl, gl + G, ... (CPL of them at most):
//  1. all-pairs hop distances by a BFS from every node into a uint8 matrix:
//     for components of up to 64 nodes in shared memory (lane s runs the
//     BFS of sources s, s + G, ...), for larger ones in global memory (the
//     group expands one source at a time in a shared row), so that a few
//     large components do not take all of an SM's shared memory; with unit
//     edge weights this equals the Floyd-Warshall result the paper names, at
//     O(n (n + E)) instead of O(n^3) work.  For the sweeps each row holds a
//     lane's distances contiguously (rewritten after the BFS in shared
//     memory), so a lane reads its part of a row with one vector load;
//  2. optional initial positions (SplitMix64 per node id, or per the seed
//     id a graph carries) scaled by l * diameter / 2, in shared memory;
//  3. Gauss-Seidel sweeps: for m = 0..n-1 the lanes sum the gradient and
//     Hessian of the KK energy over all i != m (each lane over its own
//     nodes; xor-butterfly sums so every lane holds identical totals), take
//     a safeguarded 2x2 Newton-Raphson step (kk_step, FP32; the FP64 rate of
//     GB300 is a small fraction of its FP32 rate) and the owner lane moves
//     p_m.
// Small components share a warp: lane groups of 4, 8 or 16 lanes by
// component size class, each group laying out its own component.
#include <algorithm>
#include <memory>
#include <vector>

#include "bgl_internal.cuh"
#include "kk_common.cuh"

namespace bgl {

namespace {

// the id that seeds node v's initial position: v, or sid[v] for a graph that
// carries its own (a union of subgraphs, each keeping its own ids)
__device__ __forceinline__ int32_t seed_id_of(const int32_t *__restrict__ sid, int32_t v) { return sid ? sid[v] : v; }

__global__ void init_positions_kernel(const int32_t *__restrict__ nodes, const int32_t *__restrict__ sid, int64_t q0,
                                      int64_t q1, int64_t qbase, uint64_t seed, float2 *__restrict__ xy) {
    int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q1) return;
    xy[q - qbase] = initial_position(seed, seed_id_of(sid, nodes[q]));
}

template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// two group sums at once, the adds packed (FP32x2; each component the same
// add, in the same order, as group_sum)
template <int G>
__device__ __forceinline__ float2 group_sum2(float2 v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
        v = __fadd2_rn(v, make_float2(__shfl_xor_sync(mask, v.x, o), __shfl_xor_sync(mask, v.y, o)));
    return v;
}

struct KKArgs {
    const int64_t *comp_off;
    const int64_t *coff;
    const int32_t *cadj;
    const int32_t *nodes;
    const int32_t *sid;    // seed ids of the nodes (null: the node ids)
    float2 *xy;            // indexed by q - qbase
    int64_t qbase;
    int64_t c0, nc;        // components [c0, c0 + nc)
    int maxn;              // largest component in the launch
    int gpb;               // lane groups per block
    uint64_t seed;
    float l;
    int sweeps;
    float tol;
    int init;
    int32_t *d_out;        // optional int32 distance matrix of component c0
    uint8_t *gdist;        // distances in global memory (null: in shared memory)
    const int64_t *gdist_off;  // [nc] start of component c0 + k's matrix in gdist
};

// Distance rows are padded to a multiple of 8 bytes (padding 255).
__host__ __device__ __forceinline__ int kk_row_stride(int n) { return (n + 7) & ~7; }
constexpr size_t KK_TABLE_BYTES = 256 * sizeof(float2);

// Row stride of a shared-memory distance matrix: G CPL when the rows are
// rewritten lane-major for the sweeps (CPL a multiple of 4), else node order
// padded to 8 bytes.
__host__ __device__ __forceinline__ int kk_smem_stride(int G, int CPL, int n) {
    return CPL % 4 == 0 ? G * CPL : kk_row_stride(n);
}

// Shared memory of one lane group: its distance matrix (maxn rows of rs
// bytes) or, with the matrices in global memory, one BFS row; then the
// positions (float2) of its component's nodes and of the lanes' padding
// slots up to `slots` (G CPL), and each node's sum of k_mi (float), each
// part 16-byte aligned.
struct KkGroupLayout {
    size_t pos, ksum, bytes;
};
__host__ __device__ __forceinline__ KkGroupLayout kk_group_layout(int maxn, bool glob, int rs, int slots) {
    const size_t a = 16;
    const size_t d = glob ? (size_t)kk_row_stride(maxn) : (size_t)maxn * rs;
    KkGroupLayout L;
    L.pos = (d + a - 1) / a * a;
    L.ksum = L.pos + (8 * (size_t)(slots > maxn ? slots : maxn) + a - 1) / a * a;
    L.bytes = L.ksum + (4 * (size_t)maxn + a - 1) / a * a;
    return L;
}

// Lane gl's distances to its nodes gl, gl + G, ... in one row of the
// distance matrix.  In shared memory (node order, row stride ds) byte by
// byte; in global memory (GLOB: each lane's CPL bytes contiguous at gl CPL,
// row stride G CPL, 255 past the component) as CPL / 4 words from one vector
// load, a byte taken out only where it is used.
template <int G, int CPL, bool GLOB>
struct KkRow {
    uint8_t b[CPL];
    __device__ __forceinline__ void load(const uint8_t *row, int gl, int ds) {
#pragma unroll
        for (int j = 0; j < CPL; ++j) b[j] = gl + j * G < ds ? row[gl + j * G] : 255;
    }
    __device__ __forceinline__ int get(int j) const { return b[j]; }
};

template <int G, int CPL>
struct KkRow<G, CPL, true> {
    static_assert(CPL % 4 == 0, "a lane's part of a global-memory row is whole words");
    uint32_t w[CPL / 4];
    __device__ __forceinline__ void load(const uint8_t *row, int gl, int) {
        const uint8_t *src = row + gl * CPL;           // 4 CPL-byte aligned (row stride G CPL)
        if constexpr (CPL == 4) {
            w[0] = *reinterpret_cast<const uint32_t *>(src);
        } else if constexpr (CPL == 8) {
            const uint2 t = *reinterpret_cast<const uint2 *>(src);
            w[0] = t.x;
            w[1] = t.y;
        } else {
#pragma unroll
            for (int q = 0; q < CPL / 16; ++q) {
                const uint4 t = reinterpret_cast<const uint4 *>(src)[q];
                w[4 * q] = t.x;
                w[4 * q + 1] = t.y;
                w[4 * q + 2] = t.z;
                w[4 * q + 3] = t.w;
            }
        }
    }
    __device__ __forceinline__ int get(int j) const { return (int)((w[j / 4] >> (8 * (j % 4))) & 255u); }
};

// One group of G lanes per component (G = 4, 8, 16 or 32); lane gl owns the
// nodes gl + j G (j < CPL): their distances to the current node m are read
// one step ahead (the next row's loads are in flight during the current
// step).  The positions live in the group's shared memory, so node m's is
// one broadcast load and its move one store.  GLOB: the distance matrix is
// in global memory (components of more than 64 nodes).
template <int G, int CPL, bool GLOB>
__global__ void kk_kernel(KKArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int grp = threadIdx.x / G;                 // group in the block
    const int gl = threadIdx.x % G;                  // lane in the group
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((lane / G) * G));
    const int64_t c = a.c0 + (int64_t)blockIdx.x * a.gpb + grp;
    const bool live = c < a.c0 + a.nc;
    const int64_t q0 = live ? a.comp_off[c] : 0;
    const int n = live ? (int)(a.comp_off[c + 1] - q0) : 0;
    constexpr bool glob = GLOB;
    // rows lane-major during the sweeps (one vector load per lane and row):
    // in global memory always, in shared memory when CPL is a multiple of 4
    constexpr bool PACKED = GLOB || CPL % 4 == 0;
    constexpr int GDS = G * CPL;                     // row stride of a lane-major matrix
    const int nds = kk_row_stride(n);                // node-order row (a BFS row in shared memory)
    const int ds = PACKED ? GDS : nds;               // row stride of the distance matrix
    const KkGroupLayout gl_ = kk_group_layout(a.maxn, glob, kk_smem_stride(G, CPL, a.maxn), GDS);
    // per-block table: s_kl[d] = (k, k l) with k = d^-2 and l = l_unit d,
    // zero for d = 0 and d = 255
    float2 *s_kl = reinterpret_cast<float2 *>(smem);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const bool ok = i != 0 && i != 255;
        const float k = 1.0f / (float)(i * i);
        s_kl[i] = ok ? make_float2(k, k * (a.l * (float)i)) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (c >= a.c0 + a.nc) return;
    unsigned char *base = smem + KK_TABLE_BYTES + (size_t)grp * gl_.bytes;
    uint8_t *dist = glob ? a.gdist + a.gdist_off[c - a.c0] : base;
    float2 *pos = reinterpret_cast<float2 *>(base + gl_.pos);
    float *ksum = reinterpret_cast<float *>(base + gl_.ksum);

    // 1. BFS from every node (Section 3.1: all-pairs shortest paths, unit weights)
    if (glob) {
        // large component: one source at a time, the group expanding each
        // level together in a shared row, which then goes to global memory
        uint8_t *row = base;
        for (int s = 0; s < n; ++s) {
            for (int v = gl; v < nds; v += G) row[v] = v == s ? 0 : 255;
            __syncwarp(gmask);
            for (int k = 0; k < 254; ++k) {
                bool grew = false;
                for (int v = gl; v < n; v += G) {
                    if (row[v] != k) continue;
                    for (int64_t e = a.coff[q0 + v]; e < a.coff[q0 + v + 1]; ++e) {
                        const int w = (int)(a.cadj[e] - q0);
                        if (row[w] == 255) {
                            row[w] = (uint8_t)(k + 1);   // lanes reaching w write the same value
                            grew = true;
                        }
                    }
                }
                __syncwarp(gmask);
                if (!__any_sync(gmask, grew)) break;
            }
            // lane gl's nodes gl, gl + G, ... at gl CPL .. gl CPL + CPL - 1
            for (int j = 0; j < CPL; ++j) {
                const int v = gl + j * G;
                dist[(size_t)s * GDS + gl * CPL + j] = v < n ? row[v] : (uint8_t)255;
            }
            __syncwarp(gmask);
        }
        __threadfence_block();
    }
    for (int s = gl; !glob && s < n; s += G) {
        uint8_t *row = dist + (size_t)s * ds;
        for (int v = 0; v < ds; ++v) row[v] = 255;
        row[s] = 0;
        for (int k = 0; k < 254; ++k) {
            bool grew = false;
            for (int v = 0; v < n; ++v) {
                if (row[v] != k) continue;
                for (int64_t e = a.coff[q0 + v]; e < a.coff[q0 + v + 1]; ++e) {
                    int w = (int)(a.cadj[e] - q0);
                    if (row[w] == 255) {
                        row[w] = (uint8_t)(k + 1);
                        grew = true;
                    }
                }
            }
            if (!grew) break;
        }
    }
    __syncwarp(gmask);
    // slot of node v in a row
    auto slot = [&](int v) { return glob ? (v % G) * CPL + v / G : v; };
    int diam = 0;
    for (int i = gl; i < n * n; i += G) {
        int d = dist[(size_t)(i / n) * ds + slot(i % n)];
        if (d != 255 && d > diam) diam = d;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) diam = max(diam, __shfl_xor_sync(gmask, diam, o));

    if (a.d_out && c == a.c0) {
        for (int i = gl; i < n * n; i += G) {
            const int d = dist[(size_t)(i / n) * ds + slot(i % n)];
            a.d_out[i] = d == 255 ? -1 : d;
        }
    }

    // 2. positions of the component's nodes, and sum_i k_mi of every node m
    // (constant over the sweeps: the Hessian's diagonal is that sum minus the
    // position-dependent terms)
    const float scale = a.l * (float)diam * 0.5f;
    // the lanes' slots past the component: a finite position (0, 0), whose
    // pair terms are exactly zero (k = k l = 0 for the 255 distance)
    for (int v = n + gl; v < GDS; v += G) pos[v] = make_float2(0.f, 0.f);
    for (int v = gl; v < n; v += G) {
        float2 p;
        if (a.init) {
            p = initial_position(a.seed, seed_id_of(a.sid, a.nodes[q0 + v]));
            p.x *= scale;
            p.y *= scale;
        } else {
            p = a.xy[q0 + v - a.qbase];
        }
        pos[v] = p;
        const uint8_t *row = dist + (size_t)(glob ? 0 : v) * ds;
        float sk = 0.f;
        if (!glob) {
            for (int i = 0; i < n; ++i) sk += s_kl[row[i]].x;
        }
        ksum[v] = sk;
    }
    if constexpr (!GLOB && PACKED) {
        // the rows to the lane-major layout of the sweeps (lane gl's nodes gl,
        // gl + G, ... at gl CPL ..), each lane rewriting its own rows once
        // every lane has read the node-order ones (diameter, export)
        __syncwarp(gmask);
        for (int s = gl; s < n; s += G) {
            uint8_t *row = dist + (size_t)s * GDS;
            uint32_t w[GDS / 4];
#pragma unroll
            for (int q = 0; q < GDS / 4; ++q) w[q] = reinterpret_cast<const uint32_t *>(row)[q];
#pragma unroll
            for (int v = 0; v < GDS; ++v)
                row[(v % G) * CPL + v / G] = (uint8_t)((w[v / 4] >> (8 * (v % 4))) & 255u);
        }
    }
    if (glob) {
        // one row at a time from global memory, the group's lanes over its entries
        for (int v = 0; v < n; ++v) {
            const uint8_t *row = dist + (size_t)v * ds;
            float sk = 0.f;
            for (int j = 0; j < CPL && gl + j * G < n; ++j) sk += s_kl[row[gl * CPL + j]].x;
            sk = group_sum<G>(sk, gmask);
            if (gl == 0) ksum[v] = sk;
        }
    }
    __syncwarp(gmask);

    // 3. Gauss-Seidel Newton-Raphson sweeps.  k_mi = d^-2 and k_mi l_mi come
    // from the block's table (0 for d = 0: the node itself; and for the 255
    // padding of a row), and r^2 carries a 1e-30 shift, so the pair terms
    // need no branch (the node itself adds exactly 0).  Per pair:
    //   g += k (1 - l / r) (p_m - p_i),
    //   H_xx -= k l dy^2 / r^3,  H_yy -= k l dx^2 / r^3,  H_xy += k l dx dy / r^3
    // (the diagonal's sum_i k_mi is added once per node step).
    KkRow<G, CPL, PACKED> dn;
    dn.load(dist, gl, ds);
    for (int sw = 0; sw < a.sweeps; ++sw) {
        float gmax2 = 0.f;                           // largest squared gradient norm of the sweep
        for (int m = 0; m < n; ++m) {
            const KkRow<G, CPL, PACKED> d = dn;
            // next row (m + 1, or row 0 for the next sweep) in flight
            dn.load(dist + (size_t)(m + 1 < n ? m + 1 : 0) * ds, gl, ds);
            const float2 pm = pos[m];
            // (g_x, g_y) and (H_yy, H_xx) accumulate in FP32x2 pairs, each
            // component the same operations as the scalar terms
            float2 g2 = make_float2(0.f, 0.f), h2 = make_float2(0.f, 0.f);
            float hxy = 0.f;
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                if (j * G >= n) break;                   // the group's component has no node there
                const float2 kl = s_kl[d.get(j)];
                const float2 pi = pos[gl + j * G];
                const float2 d = __ffma2_rn(pi, make_float2(-1.f, -1.f), pm);   // p_m - p_i, exact sign flip
                const float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, 1e-30f));
                const float rinv = rsqrtf(r2);
                // w = k l / r^3 (k l first: zero for the node itself, whose
                // 1/r^3 would overflow), c = k - w r^2 = k (1 - l / r)
                const float w = (kl.y * rinv) * (rinv * rinv);
                const float c = fmaf(-w, r2, kl.x);
                g2 = __ffma2_rn(make_float2(c, c), d, g2);
                const float2 nwd = __fmul2_rn(make_float2(-w, -w), d);         // (-w dx, -w dy)
                h2 = __ffma2_rn(nwd, make_float2(d.x, d.y), h2);                 // H_yy -= w dx^2, H_xx -= w dy^2
                hxy = fmaf(-nwd.x, d.y, hxy);
            }
            // h2 holds (H_yy, H_xx)
            const float2 gs = group_sum2<G>(g2, gmask);
            const float2 hs = group_sum2<G>(make_float2(h2.y, h2.x), gmask);
            const float gx = gs.x, gy = gs.y, hxx = hs.x, hyy = hs.y;
            hxy = group_sum<G>(hxy, gmask);
            const float km = ksum[m];
            gmax2 = fmaxf(gmax2, fmaf(gx, gx, gy * gy));
            float dxm, dym;
            // every lane holds the same sums and takes the same step; the
            // node's owner stores the new position
            if (kk_step(gx, gy, km + hxx, hxy, km + hyy, a.l, &dxm, &dym) && gl == m % G)
                pos[m] = make_float2(pm.x + dxm, pm.y + dym);
            __syncwarp(gmask);
        }
        if (a.tol > 0.f && gmax2 < a.tol * a.tol) break;
    }
    for (int v = gl; v < n; v += G) a.xy[q0 + v - a.qbase] = pos[v];
}

size_t kk_group_bytes(int maxn, bool glob, int rs, int slots) {
    return kk_group_layout(maxn, glob, rs, slots).bytes;
}


// lanes per component of the three largest size classes: 32 (0), 16 (1) or
// 8 (2), with correspondingly more nodes per lane
#ifndef BGL_KK_WIDE
#define BGL_KK_WIDE 1
#endif
// lanes per component of the classes of 9-32 nodes: 16 and 8 (0), or 8 and
// 4 with twice the nodes per lane (1)
#ifndef BGL_KK_NARROW
#define BGL_KK_NARROW 1
#endif

// components above this size keep their distance matrix in global memory
constexpr int KK_SMEM_MAX_N = 64;

}  // namespace

void init_positions(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t q0, int64_t q1) {
    if (q1 <= q0) return;
    int64_t n = q1 - q0;
    init_positions_kernel<<<(unsigned)((n + 255) / 256), 256, 0, g->ctx->stream>>>(g->nodes.p, g->seed_id.p, q0, q1,
                                                                                   q0, p->seed, xy);
    BGL_LAUNCH_CHECK();
}

// One size class of a KK launch: components [c0, c1) in groups of G lanes
// with up to CPL nodes per lane; distances in global memory above 64 nodes.
struct KkClass {
    int G = 0, CPL = 0;
    int64_t c0 = 0, c1 = 0;
    int maxn = 1, gpb = 1;
    size_t smem = 0;
    DevBuf<uint8_t> gdist;
    DevBuf<int64_t> gdist_off;
};

struct KkRun {
    bgl_graph *g = nullptr;
    std::vector<std::unique_ptr<KkClass>> cls;
};

template <int G, int CPL>
static void kk_prepare_class(KkRun &run, int64_t c0, int64_t c1) {
    if (c1 <= c0) return;
    bgl_graph *g = run.g;
    auto k = std::make_unique<KkClass>();
    k->G = G;
    k->CPL = CPL;
    k->c0 = c0;
    k->c1 = c1;
    int maxn = (int)(g->h_comp_off[c0 + 1] - g->h_comp_off[c0]);   // components sorted by size, descending
    BGL_REQUIRE(maxn <= G * CPL && maxn <= 255, "kk: component larger than its size class");
    if (maxn < 1) maxn = 1;
    k->maxn = maxn;
    const bool glob = maxn > KK_SMEM_MAX_N;
    const size_t gb = kk_group_bytes(maxn, glob, kk_smem_stride(G, CPL, maxn), G * CPL);
    const int max_groups = 256 / G;
    k->gpb = (int)std::min<size_t>(max_groups, std::max<size_t>(1, (size_t)(200 * 1024) / gb));
    k->smem = KK_TABLE_BYTES + gb * k->gpb;
    if (glob) {
        // global distance matrices: n_c rows of G CPL bytes per component
        // (a lane's part of a row contiguous and aligned for one vector load)
        BGL_REQUIRE(CPL % 4 == 0, "kk: distances in global memory need a multiple of 4 nodes per lane");
        std::vector<int64_t> off(c1 - c0);
        int64_t tot = 0;
        for (int64_t c = c0; c < c1; ++c) {
            const int64_t nc = g->h_comp_off[c + 1] - g->h_comp_off[c];
            off[c - c0] = tot;
            tot += nc * (int64_t)(G * CPL);
        }
        k->gdist.reset(g->ctx->alloc, std::max<int64_t>(tot, 8));
        k->gdist_off.reset(g->ctx->alloc, off.size());
        BGL_CUDA(cudaMemcpyAsync(k->gdist_off.p, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice,
                                 g->ctx->stream));
        BGL_CUDA(cudaStreamSynchronize(g->ctx->stream));
    }
    if constexpr (CPL % 4 == 0) {
        if (glob) {
            BGL_CUDA(cudaFuncSetAttribute(kk_kernel<G, CPL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          220 * 1024));
        }
    }
    if (!glob)
        BGL_CUDA(cudaFuncSetAttribute(kk_kernel<G, CPL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      220 * 1024));
    run.cls.push_back(std::move(k));
}

template <int G, int CPL>
static void kk_enqueue_class(const KkRun &run, const KkClass &k, const bgl_params *p, float2 *xy, int64_t qbase,
                             bool init, int sweeps, int32_t *d_out, cudaStream_t s) {
    bgl_graph *g = run.g;
    KKArgs a;
    a.comp_off = g->comp_off.p;
    a.coff = g->coff.p;
    a.cadj = g->cadj.p;
    a.nodes = g->nodes.p;
    a.sid = g->seed_id.p;
    a.xy = xy;
    a.qbase = qbase;
    a.c0 = k.c0;
    a.nc = k.c1 - k.c0;
    a.maxn = k.maxn;
    a.gpb = k.gpb;
    a.seed = p->seed;
    a.l = (float)p->kk_l;
    a.sweeps = sweeps;
    a.tol = (float)p->kk_tol;
    a.init = init ? 1 : 0;
    a.d_out = d_out;
    a.gdist = k.gdist.p;
    a.gdist_off = k.gdist_off.p;
    const int64_t blocks = (a.nc + k.gpb - 1) / k.gpb;
    bool launched = false;
    if constexpr (CPL % 4 == 0) {
        if (k.gdist.p) {
            kk_kernel<G, CPL, true><<<(unsigned)blocks, G * k.gpb, k.smem, s>>>(a);
            launched = true;
        }
    }
    if (!launched) {
        BGL_REQUIRE(!k.gdist.p, "kk: distances in global memory need a multiple of 4 nodes per lane");
        kk_kernel<G, CPL, false><<<(unsigned)blocks, G * k.gpb, k.smem, s>>>(a);
    }
    BGL_LAUNCH_CHECK();
}

// first component index in [c0, c1) with at most `size` nodes (sizes descend)
static int64_t first_at_most(const bgl_graph *g, int64_t c0, int64_t c1, int64_t size) {
    int64_t lo = c0, hi = c1;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (g->h_comp_off[mid + 1] - g->h_comp_off[mid] > size) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Components in size classes (lanes x nodes per lane, BGL_KK_WIDE = 1 and
// BGL_KK_NARROW = 1): (128, 255] nodes 16 x 16, (64, 128] 16 x 8, (32, 64]
// 16 x 4, (16, 32] 8 x 4, (8, 16] 4 x 4, (4, 8] 4 x 2, <= 4 4 x 1; distances
// in global memory above 64 nodes.
// Preparing allocates every class's scratch (held until the run is
// destroyed) so that the launches need no allocation and no synchronisation.
KkRun *kk_prepare(bgl_graph *g, int64_t c0, int64_t c1) {
    BGL_RANGE("Kamada-Kawai: size classes, scratch, BFS distances (Section 3.1)");
    auto run = std::make_unique<KkRun>();
    run->g = g;
    if (c1 > c0) {
        const int64_t a128 = first_at_most(g, c0, c1, 128), a64 = first_at_most(g, c0, c1, 64),
                      a32 = first_at_most(g, c0, c1, 32), a16 = first_at_most(g, c0, c1, 16),
                      a8 = first_at_most(g, c0, c1, 8), a4 = first_at_most(g, c0, c1, 4);
#if BGL_KK_WIDE == 2
        kk_prepare_class<8, 32>(*run, c0, a128);
        kk_prepare_class<8, 16>(*run, a128, a64);
        kk_prepare_class<8, 8>(*run, a64, a32);
#elif BGL_KK_WIDE == 1
        kk_prepare_class<16, 16>(*run, c0, a128);
        kk_prepare_class<16, 8>(*run, a128, a64);
        kk_prepare_class<16, 4>(*run, a64, a32);
#else
        kk_prepare_class<32, 8>(*run, c0, a128);
        kk_prepare_class<32, 4>(*run, a128, a64);
        kk_prepare_class<32, 2>(*run, a64, a32);
#endif
#if BGL_KK_NARROW
        kk_prepare_class<8, 4>(*run, a32, a16);
        kk_prepare_class<4, 4>(*run, a16, a8);
#else
        kk_prepare_class<16, 2>(*run, a32, a16);
        kk_prepare_class<8, 2>(*run, a16, a8);
#endif
        kk_prepare_class<4, 2>(*run, a8, a4);
        kk_prepare_class<4, 1>(*run, a4, c1);
    }
    return run.release();
}

void kk_destroy(KkRun *run) { delete run; }

int kk_classes(const KkRun *run) { return (int)run->cls.size(); }

// launches size class i on stream s
void kk_enqueue(const KkRun *run, int i, const bgl_params *p, float2 *xy, int64_t qbase, bool init, int sweeps,
                int32_t *d_out, cudaStream_t s) {
    BGL_RANGE("Kamada-Kawai: Newton sweeps of one size class (Section 3.1)");
    const KkClass &k = *run->cls[i];
    switch (k.G * 64 + k.CPL) {
#if BGL_KK_WIDE == 2
        case 8 * 64 + 32: kk_enqueue_class<8, 32>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        case 8 * 64 + 16: kk_enqueue_class<8, 16>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        case 8 * 64 + 8: kk_enqueue_class<8, 8>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
#elif BGL_KK_WIDE == 1
        case 16 * 64 + 16: kk_enqueue_class<16, 16>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        case 16 * 64 + 8: kk_enqueue_class<16, 8>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        case 16 * 64 + 4: kk_enqueue_class<16, 4>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
#else
        case 32 * 64 + 8: kk_enqueue_class<32, 8>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        case 32 * 64 + 4: kk_enqueue_class<32, 4>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        case 32 * 64 + 2: kk_enqueue_class<32, 2>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
#endif
#if BGL_KK_NARROW
        case 8 * 64 + 4: kk_enqueue_class<8, 4>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        case 4 * 64 + 4: kk_enqueue_class<4, 4>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
#else
        case 16 * 64 + 2: kk_enqueue_class<16, 2>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        case 8 * 64 + 2: kk_enqueue_class<8, 2>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
#endif
        case 4 * 64 + 2: kk_enqueue_class<4, 2>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
        default: kk_enqueue_class<4, 1>(*run, k, p, xy, qbase, init, sweeps, d_out, s); break;
    }
}

static void kk_launch(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t qbase, int64_t c0, int64_t c1, bool init,
                      int sweeps, int32_t *d_out) {
    if (c1 <= c0) return;
    std::unique_ptr<KkRun> run(kk_prepare(g, c0, c1));
    for (int i = 0; i < kk_classes(run.get()); ++i)
        kk_enqueue(run.get(), i, p, xy, qbase, init, sweeps, d_out, g->ctx->stream);
    // the scratch goes back to the caching allocator only once the kernels are done
    BGL_CUDA(cudaStreamSynchronize(g->ctx->stream));
}

void kk_layout(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t qbase, int64_t c0, int64_t c1, bool init) {
    kk_launch(g, p, xy, qbase, c0, c1, init, p->kk_sweeps, nullptr);
}

void kk_distances(bgl_graph *g, int64_t c, int32_t *d_out_dev) {
    bgl_params p;
    bgl_params_default(&p);
    DevBuf<float2> tmp(g->ctx->alloc, g->h_comp_off[c + 1] - g->h_comp_off[c]);
    kk_launch(g, &p, tmp.p, g->h_comp_off[c], c, c + 1, false, 0, d_out_dev);
}

}  // namespace bgl
