// Assembly of the component layouts into one frame (Section 4).
//
// After every component has its own layout, the method rescales them to a
// similar density, links the components into a tree -- a random order, each
// component joined to the largest one before it, with edge lengths of half
// the two diameters plus a constant -- and lays that tree out with
// Kamada-Kawai, splitting it into pieces when it is too large and
// reassembling the pieces the same way.  On the device:
//   comp_stats    one block per component: centroid, scale (mean edge
//                 length 1), radius (largest distance from the centroid after
//                 scaling); FP64 sums in a fixed order
//   meta order    SplitMix64 key per component, stable radix sort
//   per level     items (components, then pieces) in order, cut into chunks
//                 of at most K; one warp per chunk: the largest-previous tree,
//                 its weighted path lengths, Kamada-Kawai on them (FP32,
//                 Gauss-Seidel, the safeguarded Newton step of Section 3.1
//                 with l d_ij replaced by the path length and steps capped at
//                 the chunk's mean edge length); the chunk is centred on its
//                 items' mean and becomes one item of the next level
//   compose       every node: scaled local position plus the offsets of the
//                 items holding it at every level
// Readings: density = mean edge length 1 (components without edges keep
// scale 1); diameter = twice the largest distance from the centroid; the
// constant is 1; "small enough" = kk_max_nodes; pieces = consecutive runs of
// at most kk_max_nodes items in the random order; initial positions of a
// chunk from SplitMix64 by item index with seed + level + 1, scaled by half
// the largest path length.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bgl_internal.cuh"
#include "kk_common.cuh"

namespace bgl {

namespace {

constexpr float KAPPA = 1.0f;                              // added to every meta-edge
constexpr uint64_t META_SALT = 0x5851F42D4C957F2Dull;      // order stream, apart from position streams
constexpr int ASM_MAX_K = 255;

// per component (component order) from c0 on, one block each: centroid,
// scale, radius.  Edge lengths in FP32, sums in FP64 (a fixed order).
__global__ void __launch_bounds__(1024) comp_stats_kernel(const float2 *__restrict__ xy, const int64_t *__restrict__ comp_off,
                                                          int64_t c0, const int64_t *__restrict__ coff,
                                                          const int32_t *__restrict__ cadj, double2 *centroid,
                                                          float *scale, float *radius, int64_t *size) {
    const int64_t c = c0 + blockIdx.x;
    const int64_t q0 = comp_off[c], q1 = comp_off[c + 1];
    __shared__ double red[3][32];
    __shared__ float redf[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sx = 0.0, sy = 0.0, sl = 0.0;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const float2 p = xy[q];
        sx += p.x;
        sy += p.y;
        for (int64_t e = coff[q]; e < coff[q + 1]; ++e) {
            const float2 o = xy[cadj[e]];
            const float dx = p.x - o.x, dy = p.y - o.y;
            sl += (double)sqrtf(fmaf(dx, dx, dy * dy));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sl += __shfl_xor_sync(0xffffffffu, sl, o);
    }
    if (lane == 0) {
        red[0][warp] = sx;
        red[1][warp] = sy;
        red[2][warp] = sl;
    }
    __syncthreads();
    double tx = 0.0, ty = 0.0, tl = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        tx += red[0][w];
        ty += red[1][w];
        tl += red[2][w];
    }
    const double n = (double)(q1 - q0);
    const double cx = tx / n, cy = ty / n;
    const int64_t e2 = coff[q1] - coff[q0];          // every edge twice
    const double s = (e2 > 0 && tl > 0.0) ? (double)e2 / tl : 1.0;
    float rmax = 0.f;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const float2 p = xy[q];
        const float dx = (float)(((double)p.x - cx) * s), dy = (float)(((double)p.y - cy) * s);
        rmax = fmaxf(rmax, sqrtf(dx * dx + dy * dy));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if (lane == 0) redf[warp] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, redf[w]);
        centroid[c] = make_double2(cx, cy);
        scale[c] = (float)s;
        radius[c] = r;
        size[c] = q1 - q0;
    }
}

__global__ void meta_keys_kernel(int64_t C, uint64_t seed, uint64_t *keys, uint32_t *vals) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    uint64_t st = (seed ^ META_SALT) ^ ((uint64_t)c * 0x9E3779B97F4A7C15ull);
    keys[c] = splitmix64(st);
    vals[c] = (uint32_t)c;
}

// rank of every component and the level-0 items in rank order
__global__ void meta_items_kernel(int64_t C, const uint32_t *__restrict__ order, const float *__restrict__ radius,
                                  const int64_t *__restrict__ size, int64_t *rank, float *item_r, int64_t *item_n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const uint32_t c = order[i];
    rank[c] = i;
    item_r[i] = radius[c];
    item_n[i] = size[c];
}

struct ChunkArgs {
    int64_t m;                 // items at this level
    int K;                     // chunk size
    const float *item_r;       // [m]
    const int64_t *item_n;     // [m]
    float *dist;               // [chunks * K * K] scratch
    float2 *offset;            // [m] out: item centre minus its chunk's centre
    int64_t *parent;           // [m] out: parent item (global index), -1 for a chunk's first item
    float *next_r;             // [chunks] out
    int64_t *next_n;           // [chunks] out
    float2 *centre;            // [m] out (may be null): item centres before centring
    uint64_t seed;             // seed + level + 1
    int sweeps;
};

// One warp per chunk; with K <= ASM_SMEM_K the chunk's distance matrix is
// kept in dynamic shared memory (K * K floats per warp), else in a.dist.
constexpr int ASM_SMEM_K = 64;

__global__ void __launch_bounds__(128) chunk_kernel(ChunkArgs a) {
    extern __shared__ float s_dist[];
    __shared__ int s_par[4][ASM_MAX_K + 1];
    __shared__ float s_len[4][ASM_MAX_K + 1];
    __shared__ float s_root[4][ASM_MAX_K + 1];       // path length from the chunk's first item
    __shared__ float2 s_p[4][ASM_MAX_K + 1];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t chunk = (int64_t)blockIdx.x * 4 + wib;
    const int64_t a0 = chunk * a.K;
    if (a0 >= a.m) return;
    const int m = (int)(a.m - a0 < (int64_t)a.K ? a.m - a0 : (int64_t)a.K);
    int *par = s_par[wib];
    float *len = s_len[wib], *root = s_root[wib];
    float2 *p = s_p[wib];
    // the largest-previous tree (first of equals), edge length r_a + r_b + kappa
    if (lane == 0) {
        int best = 0;
        par[0] = -1;
        len[0] = 0.f;
        root[0] = 0.f;
        for (int k = 1; k < m; ++k) {
            par[k] = best;
            len[k] = a.item_r[a0 + k] + a.item_r[a0 + best] + KAPPA;
            root[k] = root[best] + len[k];
            if (a.item_n[a0 + k] > a.item_n[a0 + best]) best = k;
        }
    }
    __syncwarp();
    for (int k = lane; k < m; k += 32) a.parent[a0 + k] = par[k] >= 0 ? a0 + par[k] : -1;
    // path lengths d(s, k): along the parent links, d(s, k) = d(s, par k) + len k
    // unless k is an ancestor of s (then root[s] - root[k])
    float *d = a.K <= ASM_SMEM_K ? s_dist + (size_t)wib * a.K * a.K : a.dist + chunk * (int64_t)a.K * a.K;
    float dmax = 0.f;
    for (int s = lane; s < m; s += 32) {
        float *row = d + (int64_t)s * m;
        for (int k = 0; k < m; ++k) row[k] = -1.f;
        for (int x = s; x >= 0; x = par[x]) row[x] = root[s] - root[x];
        for (int k = 1; k < m; ++k)
            if (row[k] < 0.f) row[k] = row[par[k]] + len[k];
        for (int k = 0; k < m; ++k) dmax = fmaxf(dmax, row[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    __syncwarp();
    // Kamada-Kawai on the weighted tree
    float lsum = 0.f;
    for (int k = 1 + lane; k < m; k += 32) lsum += len[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    const float cap = m > 1 ? lsum / (float)(m - 1) : 1.f;
    const float half = 0.5f * dmax;
    for (int k = lane; k < m; k += 32) {
        const float2 q = initial_position(a.seed, (int32_t)(a0 + k));
        p[k] = make_float2(q.x * half, q.y * half);
    }
    __syncwarp();
    for (int sw = 0; sw < a.sweeps && m > 1; ++sw) {
        for (int mm = 0; mm < m; ++mm) {
            const float2 pm = p[mm];
            const float *row = d + (int64_t)mm * m;
            float gx = 0.f, gy = 0.f, hxx = 0.f, hxy = 0.f, hyy = 0.f;
            for (int i = lane; i < m; i += 32) {
                const float dmi = row[i];
                if (i == mm || !(dmi > 0.f)) continue;
                const float dx = pm.x - p[i].x, dy = pm.y - p[i].y;
                const float r2 = dx * dx + dy * dy;
                if (r2 == 0.f) continue;
                const float k = 1.0f / (dmi * dmi);
                const float rinv = rsqrtf(r2);
                const float t = dmi * rinv;           // d_mi / r
                const float u = t * rinv * rinv;      // d_mi / r^3
                gx += k * dx * (1.f - t);
                gy += k * dy * (1.f - t);
                hxx += k * (1.f - u * dy * dy);
                hyy += k * (1.f - u * dx * dx);
                hxy += k * u * dx * dy;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                gx += __shfl_xor_sync(0xffffffffu, gx, o);
                gy += __shfl_xor_sync(0xffffffffu, gy, o);
                hxx += __shfl_xor_sync(0xffffffffu, hxx, o);
                hxy += __shfl_xor_sync(0xffffffffu, hxy, o);
                hyy += __shfl_xor_sync(0xffffffffu, hyy, o);
            }
            float dxm, dym;
            if (kk_step(gx, gy, hxx, hxy, hyy, cap, &dxm, &dym) && lane == 0) p[mm] = make_float2(pm.x + dxm, pm.y + dym);
            __syncwarp();
        }
    }
    // centre the chunk; next-level item
    float cx = 0.f, cy = 0.f;
    for (int k = lane; k < m; k += 32) {
        cx += p[k].x;
        cy += p[k].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cx += __shfl_xor_sync(0xffffffffu, cx, o);
        cy += __shfl_xor_sync(0xffffffffu, cy, o);
    }
    cx /= (float)m;
    cy /= (float)m;
    float rr = 0.f;
    long long nn = 0;
    for (int k = lane; k < m; k += 32) {
        const float2 o = make_float2(p[k].x - cx, p[k].y - cy);
        a.offset[a0 + k] = o;
        if (a.centre) a.centre[a0 + k] = p[k];
        rr = fmaxf(rr, sqrtf(o.x * o.x + o.y * o.y) + a.item_r[a0 + k]);
        nn += a.item_n[a0 + k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, o));
        nn += __shfl_xor_sync(0xffffffffu, nn, o);
    }
    if (lane == 0) {
        a.next_r[chunk] = rr;
        a.next_n[chunk] = nn;
    }
}

// final positions (node-id order): scaled local position plus every level's offset
__global__ void compose_kernel(int64_t n, const float2 *__restrict__ xy, const int32_t *__restrict__ nodes,
                               const int32_t *__restrict__ node_comp, const int64_t *__restrict__ rank,
                               const double2 *__restrict__ centroid, const float *__restrict__ scale,
                               const float2 *__restrict__ offs, const int64_t *__restrict__ level_base, int levels,
                               int K, float2 *__restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int c = node_comp[q];
    const float2 p = xy[q];
    const double2 cc = centroid[c];
    const float s = scale[c];
    float x = (float)(((double)p.x - cc.x) * s), y = (float)(((double)p.y - cc.y) * s);
    int64_t idx = rank[c];
    for (int L = 0; L < levels; ++L) {
        const float2 o = offs[level_base[L] + idx];
        x += o.x;
        y += o.y;
        idx /= K;
    }
    out[nodes[q]] = make_float2(x, y);
}

}  // namespace

void assemble_device(bgl_graph *g, const bgl_params *p, const float2 *xy_comp, float2 *xy_out_nodes,
                     AssemblyOut *info) {
    BGL_RANGE("assembly into one frame (Section 4)");
    bgl_ctx *ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    Allocator *A = ctx->alloc;
    const int64_t C = g->n_comp;
    const int K = std::max(2, std::min(ASM_MAX_K, (int)p->kk_max_nodes));
    if (C <= 0 || g->n <= 0) return;
    BGL_REQUIRE(C < (int64_t(1) << 32), "assemble: too many components");
    DevBuf<double2> centroid(A, C);
    DevBuf<float> scale(A, C), radius(A, C);
    DevBuf<int64_t> size(A, C), rank(A, C);
    // components in descending size: the large ones get 1024 threads
    int64_t nbig = 0;
    while (nbig < C && g->h_comp_off[nbig + 1] - g->h_comp_off[nbig] > 4096) ++nbig;
    if (nbig > 0) {
        comp_stats_kernel<<<(unsigned)nbig, 1024, 0, s>>>(xy_comp, g->comp_off.p, 0, g->coff.p, g->cadj.p, centroid.p,
                                                         scale.p, radius.p, size.p);
        BGL_LAUNCH_CHECK();
    }
    if (C > nbig) {
        comp_stats_kernel<<<(unsigned)(C - nbig), 128, 0, s>>>(xy_comp, g->comp_off.p, nbig, g->coff.p, g->cadj.p,
                                                              centroid.p, scale.p, radius.p, size.p);
        BGL_LAUNCH_CHECK();
    }
    DevBuf<uint64_t> keys(A, C);
    DevBuf<uint32_t> order(A, C);
    meta_keys_kernel<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(C, p->seed, keys.p, order.p);
    BGL_LAUNCH_CHECK();
    radix_sort_u64(ctx, keys.p, order.p, C, 64);
    // levels: items in order, chunks of K
    std::vector<int64_t> counts(1, C);
    while (counts.back() > 1) counts.push_back((counts.back() + K - 1) / K);
    const int levels = (int)counts.size() - 1 > 0 ? (int)counts.size() - 1 : 1;
    std::vector<int64_t> base(levels + 1, 0);
    for (int L = 0; L < levels; ++L) base[L + 1] = base[L] + counts[L];
    DevBuf<float2> offs(A, base[levels]);
    DevBuf<int64_t> parent(A, base[levels]), level_base(A, levels + 1);
    DevBuf<float2> centre0(A, C);
    DevBuf<float> ir(A, C), nr(A, C);
    DevBuf<int64_t> in(A, C), nnext(A, C);
    meta_items_kernel<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(C, order.p, radius.p, size.p, rank.p, ir.p, in.p);
    BGL_LAUNCH_CHECK();
    const int64_t max_chunks = (C + K - 1) / K;
    const bool sdist = K <= ASM_SMEM_K;
    DevBuf<float> dist(A, sdist ? 1 : max_chunks * (int64_t)K * K);
    const size_t chunk_smem = sdist ? sizeof(float) * 4 * (size_t)K * K : 0;
    // the static arrays plus this can pass the 48 KB default
    BGL_CUDA(cudaFuncSetAttribute(chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chunk_smem));
    for (int L = 0; L < levels; ++L) {
        const int64_t m = counts[L], chunks = (m + K - 1) / K;
        ChunkArgs a;
        a.m = m;
        a.K = K;
        a.item_r = ir.p;
        a.item_n = in.p;
        a.dist = dist.p;
        a.offset = offs.p + base[L];
        a.parent = parent.p + base[L];
        a.next_r = nr.p;
        a.next_n = nnext.p;
        a.centre = L == 0 ? centre0.p : nullptr;
        a.seed = p->seed + (uint64_t)L + 1;
        a.sweeps = p->kk_sweeps;
        chunk_kernel<<<(unsigned)((chunks + 3) / 4), 128, chunk_smem, s>>>(a);
        BGL_LAUNCH_CHECK();
        std::swap(ir, nr);
        std::swap(in, nnext);
    }
    BGL_CUDA(cudaMemcpyAsync(level_base.p, base.data(), sizeof(int64_t) * (levels + 1), cudaMemcpyHostToDevice, s));
    compose_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(g->n, xy_comp, g->nodes.p, g->node_comp.p, rank.p,
                                                                  centroid.p, scale.p, offs.p, level_base.p, levels,
                                                                  K, xy_out_nodes);
    BGL_LAUNCH_CHECK();
    if (info) {
        info->levels = levels;
        info->rank.resize(C);
        info->parent0.resize(C);
        info->scale.resize(C);
        info->radius.resize(C);
        info->centre0.resize(C);
        BGL_CUDA(cudaMemcpyAsync(info->rank.data(), rank.p, sizeof(int64_t) * C, cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaMemcpyAsync(info->parent0.data(), parent.p, sizeof(int64_t) * C, cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaMemcpyAsync(info->scale.data(), scale.p, sizeof(float) * C, cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaMemcpyAsync(info->radius.data(), radius.p, sizeof(float) * C, cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaMemcpyAsync(info->centre0.data(), centre0.p, sizeof(float2) * C, cudaMemcpyDeviceToHost, s));
    }
    // the scratch returns to the caching allocator when this function ends
    BGL_CUDA(cudaStreamSynchronize(s));
}

}  // namespace bgl
