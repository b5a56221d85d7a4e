// Kamada-Kawai layout of small components (Section 3.1) and the initial
// positions shared by every component.
//
// A group of lanes lays out one component of at most 255 nodes:
//  1. all-pairs hop distances by a BFS from every node (lane s runs the BFS
//     of sources s, s+32, ...) into a uint8 matrix in shared memory; with
//     unit edge weights this equals the Floyd-Warshall result the paper
//     names, at O(n (n + E)) instead of O(n^3) work;
//  2. optional initial positions (SplitMix64 per node id) scaled by
//     l * diameter / 2;
//  3. Gauss-Seidel sweeps: for m = 0..n-1 the lanes sum the gradient and
//     Hessian of the KK energy over all i != m (lane-strided FP32 terms,
//     xor-butterfly reduction so every lane holds identical sums), take a
//     safeguarded 2x2 Newton-Raphson step (kk_step, FP32; the FP64 rate of
//     GB300 is a small fraction of its FP32 rate) and move p_m in shared
//     memory.
// Small components share a warp: lane groups of 4, 8, 16 or 32 lanes by
// component size class, each group laying out its own component.
#include <algorithm>

#include "bgl_internal.cuh"

namespace bgl {

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// x, y uniform on [-1, 1), exactly representable in FP32
__device__ __forceinline__ float2 initial_position(uint64_t seed, int32_t id) {
    uint64_t s = seed ^ ((uint64_t)(int64_t)id * 0x9E3779B97F4A7C15ull);
    uint64_t hx = splitmix64(s), hy = splitmix64(s);
    float x = (float)(hx >> 40) * 0x1.0p-24f * 2.0f - 1.0f;
    float y = (float)(hy >> 40) * 0x1.0p-24f * 2.0f - 1.0f;
    return make_float2(x, y);
}

__global__ void init_positions_kernel(const int32_t *__restrict__ nodes, int64_t q0, int64_t q1, int64_t qbase,
                                      uint64_t seed, float2 *__restrict__ xy) {
    int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q1) return;
    xy[q - qbase] = initial_position(seed, nodes[q]);
}

template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Safeguarded Newton-Raphson step (Section 3.1) in FP32: with
// H = l1 P1 + l2 P2 (l1 >= l2, P1 + P2 = I), delta = -(P1 g / e1 + P2 g / e2)
// where e_i = l_i for positive curvature and max(|l_i|, 0.1 max|l|) otherwise;
// steps longer than l are shortened to l.  Returns false for H = 0.
__device__ __forceinline__ bool kk_step(float gx, float gy, float a, float b, float c, float l, float *dx,
                                        float *dy) {
    const float h = 0.5f * (a - c);
    const float dd = sqrtf(h * h + b * b);
    const float tr = 0.5f * (a + c);
    const float l1 = tr + dd, l2 = tr - dd;
    const float big = fmaxf(fabsf(l1), fabsf(l2));
    if (big == 0.0f) return false;
    const float fl = 0.1f * big;
    const float e1 = l1 > 1e-12f * big ? l1 : fmaxf(fabsf(l1), fl);
    const float e2 = l2 > 1e-12f * big ? l2 : fmaxf(fabsf(l2), fl);
    float sx, sy;
    if (dd == 0.0f) {
        sx = -gx / e1;
        sy = -gy / e1;
    } else {
        const float p1x = ((h + dd) * gx + b * gy) / (2.0f * dd);
        const float p1y = (b * gx + (dd - h) * gy) / (2.0f * dd);
        sx = -(p1x / e1 + (gx - p1x) / e2);
        sy = -(p1y / e1 + (gy - p1y) / e2);
    }
    const float len = sqrtf(sx * sx + sy * sy);
    if (len > l) {
        sx *= l / len;
        sy *= l / len;
    }
    *dx = sx;
    *dy = sy;
    return true;
}

struct KKArgs {
    const int64_t *comp_off;
    const int64_t *coff;
    const int32_t *cadj;
    const int32_t *nodes;
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
};

// One group of G lanes per component (G = 4, 8, 16 or 32).
template <int G>
__global__ void kk_kernel(KKArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int grp = threadIdx.x / G;                 // group in the block
    const int gl = threadIdx.x % G;                  // lane in the group
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((lane / G) * G));
    const int64_t c = a.c0 + (int64_t)blockIdx.x * a.gpb + grp;
    if (c >= a.c0 + a.nc) return;
    const int64_t q0 = a.comp_off[c];
    const int n = (int)(a.comp_off[c + 1] - q0);
    const size_t dbytes = ((size_t)a.maxn * a.maxn + 15) & ~size_t(15);
    unsigned char *base = smem + (size_t)grp * (dbytes + 8 * (size_t)a.maxn);
    uint8_t *dist = base;
    float *px = reinterpret_cast<float *>(base + dbytes);
    float *py = px + a.maxn;

    // 1. BFS from every node (Section 3.1: all-pairs shortest paths, unit weights)
    for (int s = gl; s < n; s += G) {
        uint8_t *row = dist + (size_t)s * n;
        for (int v = 0; v < n; ++v) row[v] = 255;
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
    int diam = 0;
    for (int i = gl; i < n * n; i += G) {
        int d = dist[i];
        if (d != 255 && d > diam) diam = d;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) diam = max(diam, __shfl_xor_sync(gmask, diam, o));

    if (a.d_out && c == a.c0) {
        for (int i = gl; i < n * n; i += G) a.d_out[i] = dist[i] == 255 ? -1 : (int32_t)dist[i];
    }

    // 2. positions
    const float scale = a.l * (float)diam * 0.5f;
    for (int v = gl; v < n; v += G) {
        float2 p;
        if (a.init) {
            p = initial_position(a.seed, a.nodes[q0 + v]);
            p.x *= scale;
            p.y *= scale;
        } else {
            p = a.xy[q0 + v - a.qbase];
        }
        px[v] = p.x;
        py[v] = p.y;
    }
    __syncwarp(gmask);

    // 3. Gauss-Seidel Newton-Raphson sweeps
    for (int sw = 0; sw < a.sweeps; ++sw) {
        float gmax = 0.f;
        for (int m = 0; m < n; ++m) {
            const float xm = px[m], ym = py[m];
            const uint8_t *drow = dist + (size_t)m * n;
            float gx = 0.f, gy = 0.f, hxx = 0.f, hxy = 0.f, hyy = 0.f;
            for (int i = gl; i < n; i += G) {
                int d = drow[i];
                if (i == m || d == 0 || d == 255) continue;
                float dx = xm - px[i], dy = ym - py[i];
                float r2 = dx * dx + dy * dy;
                if (r2 == 0.f) continue;
                float fd = (float)d;
                float k = 1.0f / (fd * fd);
                float lm = a.l * fd;
                float rinv = rsqrtf(r2);
                float t = lm * rinv;              // l_mi / r
                float u = t * rinv * rinv;        // l_mi / r^3
                gx += k * dx * (1.f - t);
                gy += k * dy * (1.f - t);
                hxx += k * (1.f - u * dy * dy);
                hyy += k * (1.f - u * dx * dx);
                hxy += k * u * dx * dy;
            }
            gx = group_sum<G>(gx, gmask);
            gy = group_sum<G>(gy, gmask);
            hxx = group_sum<G>(hxx, gmask);
            hxy = group_sum<G>(hxy, gmask);
            hyy = group_sum<G>(hyy, gmask);
            gmax = fmaxf(gmax, sqrtf(gx * gx + gy * gy));
            float dxm, dym;
            if (kk_step(gx, gy, hxx, hxy, hyy, a.l, &dxm, &dym) && gl == 0) {
                px[m] = xm + dxm;
                py[m] = ym + dym;
            }
            __syncwarp(gmask);
        }
        if (a.tol > 0.f && gmax < a.tol) break;
    }
    for (int v = gl; v < n; v += G) a.xy[q0 + v - a.qbase] = make_float2(px[v], py[v]);
}

size_t kk_warp_bytes(int maxn) {
    return (((size_t)maxn * maxn + 15) & ~size_t(15)) + 8 * (size_t)maxn;
}

}  // namespace

void init_positions(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t q0, int64_t q1) {
    if (q1 <= q0) return;
    int64_t n = q1 - q0;
    init_positions_kernel<<<(unsigned)((n + 255) / 256), 256, 0, g->ctx->stream>>>(g->nodes.p, q0, q1, q0, p->seed,
                                                                                   xy);
    BGL_LAUNCH_CHECK();
}

template <int G>
static void kk_launch_group(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t qbase, int64_t c0, int64_t c1,
                            bool init, int sweeps, int32_t *d_out) {
    if (c1 <= c0) return;
    int maxn = (int)(g->h_comp_off[c0 + 1] - g->h_comp_off[c0]);   // components sorted by size, descending
    BGL_REQUIRE(maxn <= 255, "kk: components must have at most 255 nodes");
    if (maxn < 1) maxn = 1;
    const size_t gb = kk_warp_bytes(maxn);
    const int max_groups = 256 / G;
    const int gpb = (int)std::min<size_t>(max_groups, std::max<size_t>(1, (size_t)(200 * 1024) / gb));
    const size_t smem = gb * gpb;
    BGL_CUDA(cudaFuncSetAttribute(kk_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    KKArgs a;
    a.comp_off = g->comp_off.p;
    a.coff = g->coff.p;
    a.cadj = g->cadj.p;
    a.nodes = g->nodes.p;
    a.xy = xy;
    a.qbase = qbase;
    a.c0 = c0;
    a.nc = c1 - c0;
    a.maxn = maxn;
    a.gpb = gpb;
    a.seed = p->seed;
    a.l = (float)p->kk_l;
    a.sweeps = sweeps;
    a.tol = (float)p->kk_tol;
    a.init = init ? 1 : 0;
    a.d_out = d_out;
    const int64_t blocks = (a.nc + gpb - 1) / gpb;
    kk_kernel<G><<<(unsigned)blocks, G * gpb, smem, g->ctx->stream>>>(a);
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

// Components in size classes, each with lane groups of its size:
// > 16 nodes: 32 lanes, 9..16: 16, 5..8: 8, <= 4: 4.
static void kk_launch(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t qbase, int64_t c0, int64_t c1, bool init,
                      int sweeps, int32_t *d_out) {
    if (c1 <= c0) return;
    if (d_out) {   // one component, distances exported
        kk_launch_group<32>(g, p, xy, qbase, c0, c1, init, sweeps, d_out);
        return;
    }
    const int64_t a16 = first_at_most(g, c0, c1, 16), a8 = first_at_most(g, c0, c1, 8),
                  a4 = first_at_most(g, c0, c1, 4);
    kk_launch_group<32>(g, p, xy, qbase, c0, a16, init, sweeps, nullptr);
    kk_launch_group<16>(g, p, xy, qbase, a16, a8, init, sweeps, nullptr);
    kk_launch_group<8>(g, p, xy, qbase, a8, a4, init, sweeps, nullptr);
    kk_launch_group<4>(g, p, xy, qbase, a4, c1, init, sweeps, nullptr);
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
