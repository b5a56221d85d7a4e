// ForceAtlas2 iteration (Section 3.2) on the device.
//
// One iteration over the ForceAtlas2 components [c0, c1):
//   K1 repulsion      exact: tiles of 512 targets per block, sources of the
//                     same component staged 1024 at a time in shared memory;
//                     FMM components run the pipeline in fmm.cu instead.
//                     f <- F_rep = kr m_i sum_j m_j (p_i - p_j) / |p_i - p_j|^2
//   K2 attraction     fa <- -sum_{j adjacent} (p_i - p_j) - kg m_i p_i; one
//      + gravity      thread per node; nodes of degree > 128 in chunks of 2048
//                     entries, one block each, combined in chunk order.  It
//                     runs on a second stream beside the repulsion, whose
//                     final writes add fa: f <- F_rep + fa
//   K3 swing/traction per-node |F_t - F_{t-1}|, |F_t + F_{t-1}| summed in FP64
//                     per tile (warp shuffles); the last block to finish sums
//                     each component's tiles (a warp per component, fixed
//                     order) and updates s_G = min(tau trc / swg, 1.5 s_G)
//   K4 update         s_n = ks s_G / (1 + s_G sqrt|F_t - F_{t-1}|), capped at
//                     ksmax / |F_t|; p_n += s_n F_t; F_{t-1} <- F_t
// The sequence has fixed launch shapes, so it is captured once as the body of
// a device-side WHILE loop in a CUDA graph: one launch runs all iterations.  Every sum has a fixed order, so
// runs are bitwise reproducible.
#include <cstdlib>
#include <cstring>

#include "bgl_internal.cuh"
#include "fa2_update.cuh"
#include "fmm.cuh"
#include "p2p.cuh"

namespace bgl {

namespace {

// pairs of a thread's targets summed with packed FP32x2 arithmetic in the
// exact kernel (the rest scalar)
#ifndef BGL_EXACT_PACKED
#define BGL_EXACT_PACKED 2
#endif
constexpr int EX_THREADS = 256;                // a tile is EX_THREADS x R targets, R = 1, 2 or 4 (autotuned)
constexpr int EX_STILE = 1024;                 // sources per shared-memory stage
constexpr int HEAVY_DEG = 128;
constexpr int HEAVY_CHUNK = 2048;              // adjacency entries per block for high-degree nodes
constexpr int RED_TILE = 256;                  // nodes per swing/traction tile (one per thread)

struct Tile {
    int32_t comp;      // component index relative to c0
    int32_t pad;
    int64_t t0, t1;    // target positions [t0, t1)
};


// K1 (exact): repulsion of every target in the tile from every node of its component
template <int EX_R>
__global__ void __launch_bounds__(EX_THREADS) exact_repulsion_kernel(
    const Tile *__restrict__ tiles, const int64_t *__restrict__ comp_off, int64_t c0, const float2 *__restrict__ xy,
    const float *__restrict__ mass, int64_t qbase, float kr, const float2 *__restrict__ fa, float2 *__restrict__ f) {
    __shared__ float4 src[EX_STILE];
    const Tile t = tiles[blockIdx.x];
    const int64_t s_begin = comp_off[c0 + t.comp], s_end = comp_off[c0 + t.comp + 1];
    float zx[EX_R], zy[EX_R], sx[EX_R], sy[EX_R], cx[EX_R], cy[EX_R];
#pragma unroll
    for (int r = 0; r < EX_R; ++r) {
        int64_t q = t.t0 + threadIdx.x + r * EX_THREADS;
        float2 p = q < t.t1 ? xy[q - qbase] : make_float2(0.f, 0.f);
        zx[r] = p.x;
        zy[r] = p.y;
        sx[r] = sy[r] = cx[r] = cy[r] = 0.f;
    }
    for (int64_t s0 = s_begin; s0 < s_end; s0 += EX_STILE) {
        const int cnt = (int)(s_end - s0 < EX_STILE ? s_end - s0 : EX_STILE);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += EX_THREADS) {
            float2 p = xy[s0 + k - qbase];
            src[k] = make_float4(p.x, p.y, mass[s0 + k], 0.f);
        }
        __syncthreads();
        float ax[EX_R], ay[EX_R];
#pragma unroll
        for (int r = 0; r < EX_R; ++r) ax[r] = ay[r] = 0.f;
        {
            // targets 2k, 2k + 1 (k < R2) in packed FP32x2 (negated targets
            // and sums, bitwise the scalar pair's result), the rest scalar
            constexpr int R2 = EX_R / 2 < BGL_EXACT_PACKED ? EX_R / 2 : BGL_EXACT_PACKED;
            float2 nzx[R2 > 0 ? R2 : 1], nzy[R2 > 0 ? R2 : 1], gx[R2 > 0 ? R2 : 1], gy[R2 > 0 ? R2 : 1];
#pragma unroll
            for (int k = 0; k < R2; ++k) {
                nzx[k] = make_float2(-zx[2 * k], -zx[2 * k + 1]);
                nzy[k] = make_float2(-zy[2 * k], -zy[2 * k + 1]);
                gx[k] = gy[k] = make_float2(0.f, 0.f);
            }
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                const float4 q = src[j];
#pragma unroll
                for (int k = 0; k < R2; ++k) p2p_pair2(nzx[k], nzy[k], q, gx[k], gy[k]);
#pragma unroll
                for (int r = 2 * R2; r < EX_R; ++r) p2p_pair(zx[r], zy[r], q, ax[r], ay[r]);
            }
#pragma unroll
            for (int k = 0; k < R2; ++k) {
                ax[2 * k] = -gx[k].x;
                ax[2 * k + 1] = -gx[k].y;
                ay[2 * k] = -gy[k].x;
                ay[2 * k + 1] = -gy[k].y;
            }
        }
        // blocked accumulation: each stage's partial sum enters a
        // compensated (Kahan) running total
#pragma unroll
        for (int r = 0; r < EX_R; ++r) {
            float y = ax[r] - cx[r];
            float s = sx[r] + y;
            cx[r] = (s - sx[r]) - y;
            sx[r] = s;
            y = ay[r] - cy[r];
            s = sy[r] + y;
            cy[r] = (s - sy[r]) - y;
            sy[r] = s;
        }
    }
#pragma unroll
    for (int r = 0; r < EX_R; ++r) {
        int64_t q = t.t0 + threadIdx.x + r * EX_THREADS;
        if (q >= t.t1) continue;
        float km = kr * mass[q];
        const float2 a = fa ? fa[q - qbase] : make_float2(0.f, 0.f);
        f[q - qbase] = make_float2(fmaf(km, sx[r], a.x), fmaf(km, sy[r], a.y));
    }
}

// K2: attraction and gravity written to fa (Section 3.2).  Blocks below
// n_light_blocks: one thread per node of degree <= HEAVY_DEG.  The others:
// one block per chunk of HEAVY_CHUNK adjacency entries of a node of higher
// degree; the chunk sums go to `part` and the last chunk of the node to
// finish adds them in chunk order (arrival count per node).
struct HeavyChunk {
    int32_t q;        // component-order position of the node
    int32_t h;        // index of the node among the heavy nodes
    int32_t first;    // index of the node's first chunk
    int32_t nchunk;   // chunks of the node
    int64_t e0, e1;   // adjacency entries of this chunk
};

__global__ void attraction_gravity_kernel(const float2 *__restrict__ xy, const float *__restrict__ mass,
                                          const int64_t *__restrict__ coff, const int32_t *__restrict__ cadj,
                                          int64_t q0, int64_t q1, int64_t qbase, float kg,
                                          const HeavyChunk *__restrict__ chunks, int64_t n_light_blocks,
                                          float2 *part, int *arrive, float2 *__restrict__ fa) {
    if (blockIdx.x < n_light_blocks) {
        int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (q >= q1) return;
        int64_t e0 = coff[q], e1 = coff[q + 1];
        if (e1 - e0 > HEAVY_DEG) return;
        float2 p = xy[q - qbase];
        float ax = 0.f, ay = 0.f;
        for (int64_t e = e0; e < e1; ++e) {
            float2 o = xy[cadj[e] - qbase];
            ax -= p.x - o.x;
            ay -= p.y - o.y;
        }
        float km = kg * mass[q];
        fa[q - qbase] = make_float2(ax - km * p.x, ay - km * p.y);
        return;
    }
    __shared__ float rx[32], ry[32];
    __shared__ bool last;
    const int64_t k = (int64_t)blockIdx.x - n_light_blocks;
    const HeavyChunk ch = chunks[k];
    const float2 p = xy[ch.q - qbase];
    float ax = 0.f, ay = 0.f;
    for (int64_t e = ch.e0 + threadIdx.x; e < ch.e1; e += blockDim.x) {
        float2 o = xy[cadj[e] - qbase];
        ax -= p.x - o.x;
        ay -= p.y - o.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { rx[warp] = ax; ry[warp] = ay; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    float sx = 0.f, sy = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sx += rx[w]; sy += ry[w]; }
    part[k] = make_float2(sx, sy);
    __threadfence();
    last = atomicAdd(&arrive[ch.h], 1) == ch.nchunk - 1;
    if (!last) return;
    __threadfence();
    sx = 0.f;
    sy = 0.f;
    for (int j = 0; j < ch.nchunk; ++j) {
        const float2 v = __ldcg(&part[ch.first + j]);
        sx += v.x;
        sy += v.y;
    }
    arrive[ch.h] = 0;
    const float km = kg * mass[ch.q];
    fa[ch.q - qbase] = make_float2(sx - km * p.x, sy - km * p.y);
}

__global__ void heavy_flag_kernel(const int64_t *__restrict__ coff, int64_t q0, int64_t n, int32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (coff[q0 + i + 1] - coff[q0 + i]) > HEAVY_DEG;
}

__global__ void heavy_list_kernel(const int32_t *__restrict__ flag, const int32_t *__restrict__ fscan, int64_t q0,
                                  int64_t n, int32_t *__restrict__ heavy) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) heavy[fscan[i]] = (int32_t)(q0 + i);
}

__global__ void heavy_rows_kernel(const int32_t *__restrict__ heavy, const int64_t *__restrict__ coff, int64_t nh,
                                  int64_t *__restrict__ rows) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nh) return;
    rows[2 * i] = coff[heavy[i]];
    rows[2 * i + 1] = coff[heavy[i] + 1];
}

struct RedArgs {
    const Tile *tiles;        // node tiles, each inside one component
    const int64_t *tile_off;  // per component: first tile, [ncomp+1]
    int ncomp;
    const float2 *f, *fprev;
    const float *mass;
    int64_t qbase;
    int variant;
    double tau;
    double2 *partial;         // [ntiles]
    double *sg;               // [ncomp]
    unsigned *counter;        // [ncomp] tiles of each component done, zero between launches
    double *stats;            // optional, component 0
    int *iter;                // iteration counter for stats
};

// K3: swing / traction sums (Section 3.2) and the global speed of each component
__global__ void swing_traction_kernel(RedArgs a) {
    __shared__ double ws[32], wt[32];
    __shared__ bool last;
    const Tile t = a.tiles[blockIdx.x];
    // FP32 within a warp (32 terms), FP64 across warps, tiles and components
    // (FP64 issue is scarce on this part, so it is kept off the per-node
    // path).  The order is the fused FMM iteration's (combine_kernel): tiles
    // of 256 consecutive nodes of a component, one node per thread, so a
    // component gets the same s_G whether it is iterated alone or with others.
    float sw = 0.f, tr = 0.f;
    const int i = threadIdx.x;
    if (i < (int)(t.t1 - t.t0)) {
        const int64_t q = t.t0 + i;
        fa2_swing_terms(a.f[q - a.qbase], a.fprev[q - a.qbase], a.mass[q], a.variant, sw, tr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { ws[warp] = (double)sw; wt[warp] = (double)tr; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, u = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s += ws[w]; u += wt[w]; }
        a.partial[blockIdx.x] = make_double2(s, u);
        __threadfence();
        const unsigned ntc = (unsigned)(a.tile_off[t.comp + 1] - a.tile_off[t.comp]);
        last = atomicAdd(&a.counter[t.comp], 1u) == ntc - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the component's last tile to finish adds its tile sums in the fused
    // iteration's order (combine_kernel's last block, also 256 threads):
    // thread t sums the tiles t, t + 256, ... in order, a butterfly in each
    // warp, then the warps' results in warp order
    const int c = t.comp;
    const int64_t k0 = a.tile_off[c], nk = a.tile_off[c + 1] - k0;
    double swg = 0.0, trc = 0.0;
    for (int64_t k = threadIdx.x; k < nk; k += blockDim.x) {
        const double2 v = __ldcg(&a.partial[k0 + k]);   // written by other blocks: bypass L1
        swg += v.x;
        trc += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        swg += __shfl_xor_sync(0xffffffffu, swg, o);
        trc += __shfl_xor_sync(0xffffffffu, trc, o);
    }
    __syncthreads();
    if (lane == 0) {
        ws[warp] = swg;
        wt[warp] = trc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        swg = 0.0;
        trc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            swg += ws[w];
            trc += wt[w];
        }
        const double s_new = fa2_global_speed(swg, trc, a.sg[c], a.tau);
        a.sg[c] = s_new;
        if (c == 0) {
            if (a.stats) {
                const int it = *a.iter;
                a.stats[3 * it] = swg;
                a.stats[3 * it + 1] = trc;
                a.stats[3 * it + 2] = s_new;
            }
            *a.iter += 1;
        }
        a.counter[c] = 0u;
    }
}

// K4: node speeds and the position update
__global__ void update_kernel(const float2 *__restrict__ f, float2 *__restrict__ fprev, float2 *__restrict__ xy,
                              const int32_t *__restrict__ node_comp, const double *__restrict__ sg, int64_t q0,
                              int64_t q1, int64_t qbase, int64_t c0, float ks, float ksmax, int *bad) {
    int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q1) return;
    const float2 F = f[q - qbase], P = fprev[q - qbase];
    const float2 p = fa2_move(xy[q - qbase], F, P, (float)sg[node_comp[q] - c0], ks, ksmax);
    if (!isfinite(p.x) || !isfinite(p.y)) *bad = 1;
    xy[q - qbase] = p;
    fprev[q - qbase] = F;
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

static void launch_exact(int r, int ntiles, const Tile *tiles, const int64_t *comp_off, int64_t c0, const float2 *xy,
                         const float *mass, int64_t qbase, float kr, const float2 *fa, float2 *f, cudaStream_t s) {
    if (r == 1)
        exact_repulsion_kernel<1><<<ntiles, EX_THREADS, 0, s>>>(tiles, comp_off, c0, xy, mass, qbase, kr, fa, f);
    else if (r == 4)
        exact_repulsion_kernel<4><<<ntiles, EX_THREADS, 0, s>>>(tiles, comp_off, c0, xy, mass, qbase, kr, fa, f);
    else
        exact_repulsion_kernel<2><<<ntiles, EX_THREADS, 0, s>>>(tiles, comp_off, c0, xy, mass, qbase, kr, fa, f);
    BGL_LAUNCH_CHECK();
}

// tiles of EX_THREADS * r targets over the given components (indices >= c0)
static std::vector<Tile> exact_tiles(const bgl_graph *g, int64_t c0, const std::vector<int64_t> &comps, int r) {
    std::vector<Tile> ex;
    const int64_t tile = (int64_t)EX_THREADS * r;
    for (int64_t c : comps) {
        const int64_t a = g->h_comp_off[c], b = g->h_comp_off[c + 1];
        for (int64_t t = a; t < b; t += tile) ex.push_back(Tile{(int32_t)(c - c0), 0, t, std::min(b, t + tile)});
    }
    return ex;
}

// Autotuner of the exact tiles: the first time a context meets a set of
// exact components of a given scale (log2 of the pairs of one evaluation),
// each R in {1, 2, 4} is timed on one evaluation (after one warm-up launch),
// and the fastest is kept for that scale.  Small sets (under 2^24 pairs)
// take R = 2 untimed.
static int exact_tile_choice(bgl_graph *g, const bgl_params *p, const std::vector<int64_t> &comps) {
    if (comps.empty()) return 2;
    double pairs = 0.0;
    for (int64_t c : comps) {
        const double n = (double)(g->h_comp_off[c + 1] - g->h_comp_off[c]);
        pairs += n * n;
    }
    if (pairs < (double)(1 << 24)) return 2;
    const int scale = (int)std::log2(pairs);
    bgl_ctx *ctx = g->ctx;
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        auto it = ctx->tune_exact.find(scale);
        if (it != ctx->tune_exact.end()) return it->second;
    }
    cudaStream_t s = ctx->stream;
    const int64_t c0 = comps.front();
    const int64_t q0 = g->h_comp_off[c0], q1 = g->h_comp_off[comps.back() + 1];
    DevBuf<float2> xy(ctx->alloc, q1 - q0), f(ctx->alloc, q1 - q0);
    init_positions(g, p, xy.p, q0, q1);
    cudaEvent_t e0, e1;
    BGL_CUDA(cudaEventCreate(&e0));
    BGL_CUDA(cudaEventCreate(&e1));
    int best = 2;
    float best_ms = 1e30f;
    try {
        for (int r : {1, 2, 4}) {
            const std::vector<Tile> ex = exact_tiles(g, c0, comps, r);
            DevBuf<Tile> tiles(ctx->alloc, ex.size());
            BGL_CUDA(cudaMemcpyAsync(tiles.p, ex.data(), sizeof(Tile) * ex.size(), cudaMemcpyHostToDevice, s));
            launch_exact(r, (int)ex.size(), tiles.p, g->comp_off.p, c0, xy.p, g->mass.p, q0, (float)p->kr, nullptr,
                         f.p, s);
            BGL_CUDA(cudaEventRecord(e0, s));
            launch_exact(r, (int)ex.size(), tiles.p, g->comp_off.p, c0, xy.p, g->mass.p, q0, (float)p->kr, nullptr,
                         f.p, s);
            BGL_CUDA(cudaEventRecord(e1, s));
            BGL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            BGL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = r;
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tune_exact[scale] = best;
    return best;
}

bool use_fmm(const bgl_params *p, int64_t n) {
    if (p->repulsion == BGL_REP_FMM) return true;
    if (p->repulsion == BGL_REP_EXACT) return false;
    return n >= p->fmm_min_nodes;
}

// Measured exact/FMM crossover (repulsion AUTO with fmm_min_nodes = -1).
// Components below TUNE_LO nodes take the exact sum, those of TUNE_HI or
// more the FMM.  In between, the first component of each size octave that a
// context meets is measured at its initial positions: one FMM evaluation
// (its cost as it runs, one component after another on the stream), and
// the exact sum's pair rate with the component's tiles repeated until they
// fill every SM (the rate the exact tiles of a batch of components reach
// together); the FMM is kept for that octave (and that p and leaf size) if
// its evaluation takes less than n^2 pairs at that rate.
constexpr int64_t TUNE_LO = 2048, TUNE_HI = 1 << 17;

static bool use_fmm_for(bgl_graph *g, const bgl_params *p, int64_t c) {
    const int64_t n = g->h_comp_off[c + 1] - g->h_comp_off[c];
    if (p->repulsion != BGL_REP_AUTO || p->fmm_min_nodes >= 0) return use_fmm(p, n);
    if (n < TUNE_LO) return false;
    if (n >= TUNE_HI) return true;
    bgl_ctx *ctx = g->ctx;
    const int key = (int)std::log2((double)n) * 10000 + p->fmm_p * 300 + p->leaf_size;
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        auto it = ctx->tune_fmm.find(key);
        if (it != ctx->tune_fmm.end()) return it->second;
    }
    cudaStream_t s = ctx->stream;
    const int64_t q0 = g->h_comp_off[c], q1 = g->h_comp_off[c + 1];
    DevBuf<float2> xy(ctx->alloc, n), f(ctx->alloc, n);
    init_positions(g, p, xy.p, q0, q1);
    const std::vector<Tile> one = exact_tiles(g, c, std::vector<int64_t>{c}, 2);
    // repeated until there are four tiles per SM (each copy writes the same forces)
    const int reps = std::max<int>(1, (4 * ctx->num_sms + (int)one.size() - 1) / (int)one.size());
    std::vector<Tile> ex;
    for (int r = 0; r < reps; ++r) ex.insert(ex.end(), one.begin(), one.end());
    DevBuf<Tile> tiles(ctx->alloc, ex.size());
    BGL_CUDA(cudaMemcpyAsync(tiles.p, ex.data(), sizeof(Tile) * ex.size(), cudaMemcpyHostToDevice, s));
    FmmPlan *pl = fmm_create(g, p, c);
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    float ms_fmm = 0.f, ms_exact = 0.f;
    try {
        for (auto &ev : e) BGL_CUDA(cudaEventCreate(&ev));
        fmm_repulsion(pl, xy.p, q0, f.p, q0);
        BGL_CUDA(cudaEventRecord(e[0], s));
        fmm_repulsion(pl, xy.p, q0, f.p, q0);
        BGL_CUDA(cudaEventRecord(e[1], s));
        launch_exact(2, (int)ex.size(), tiles.p, g->comp_off.p, c, xy.p, g->mass.p, q0, (float)p->kr, nullptr, f.p, s);
        BGL_CUDA(cudaEventRecord(e[2], s));
        launch_exact(2, (int)ex.size(), tiles.p, g->comp_off.p, c, xy.p, g->mass.p, q0, (float)p->kr, nullptr, f.p, s);
        BGL_CUDA(cudaEventRecord(e[3], s));
        BGL_CUDA(cudaEventSynchronize(e[3]));
        BGL_CUDA(cudaEventElapsedTime(&ms_fmm, e[0], e[1]));
        BGL_CUDA(cudaEventElapsedTime(&ms_exact, e[2], e[3]));
        const int err = fmm_error(pl);
        if (err & 1) fail(BGL_ETIMEOUT, "fmm: a bounded device-side wait gave up");
        if (err & 8) fail(BGL_ENUMERIC, "fmm: non-finite positions");
        if (err) fail(BGL_ENOMEM, "fmm: tree or list capacity exceeded (error bits " + std::to_string(err) + ")");
    } catch (...) {
        for (auto ev : e)
            if (ev) cudaEventDestroy(ev);
        fmm_destroy(pl);
        throw;
    }
    for (auto ev : e) cudaEventDestroy(ev);
    fmm_destroy(pl);
    // the exact sum of this component alone, at the batched pair rate
    const double exact_ms = (double)ms_exact / reps;
    const bool fmm = ms_fmm < exact_ms;
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tune_fmm[key] = fmm;
    return fmm;
}

// Everything one set of ForceAtlas2 components needs across iterations.
struct Fa2Run {
    bgl_graph *g;
    const bgl_params *p;
    float2 *xy;
    int64_t qbase, c0, c1, q0, q1;
    DevBuf<Tile> ex_tiles, red_tiles;
    int ex_r = 2;                 // targets per thread of the exact tiles
    DevBuf<int64_t> red_tile_off;
    int n_ex_tiles = 0, n_red_tiles = 0;
    DevBuf<float2> f, fprev, fa;
    DevBuf<double2> partial;
    DevBuf<double> sg;
    DevBuf<unsigned> counter;
    DevBuf<int> iter;
    DevBuf<int> loop;              // iterations done by the device-side loop of one graph launch
    DevBuf<HeavyChunk> chunks;
    DevBuf<float2> chunk_part;
    DevBuf<int> chunk_arrive;
    int64_t n_chunks = 0;
    std::vector<FmmPlan *> fmm;   // one per FMM component
    std::vector<int64_t> fmm_comp;
    cudaStream_t side = nullptr;  // attraction + gravity, beside the repulsion
    cudaEvent_t ev_fork = nullptr, ev_fa = nullptr;
    // A run whose only component is on the FMM path iterates fused: the FMM's
    // combine pass sums swing and traction and sets s_G, and one kernel moves
    // the points and makes the next evaluation's root square (no swing/traction
    // kernel, no bounding-box kernel).  BGL_FUSED_ITERATION=0 turns it off.
    bool fused = false;

    void enable_fuse(double *d_stats) {
        if (!fused) {
            const char *v = std::getenv("BGL_FUSED_ITERATION");
            if (v && v[0] == '0') return;
            if (fmm.size() != 1 || n_ex_tiles != 0 || c1 - c0 != 1) return;
        }
        FmmFuse fz;
        fz.fprev = fprev.p;
        fz.variant = p->swing_variant;
        fz.tau = p->tau;
        fz.sg = sg.p;
        fz.stats = d_stats;
        fz.iter = iter.p;
        fz.ks = (float)p->ks;
        fz.ksmax = (float)p->ksmax;
        fz.bad = g->ctx->d_flag + 1;
        fmm_fuse(fmm[0], fz);
        fused = true;
    }

    Fa2Run(bgl_graph *g_, const bgl_params *p_, float2 *xy_, int64_t qbase_, int64_t c0_, int64_t c1_)
        : g(g_), p(p_), xy(xy_), qbase(qbase_), c0(c0_), c1(c1_) {
        Allocator *A = g->ctx->alloc;
        cudaStream_t s = g->ctx->stream;
        q0 = g->h_comp_off[c0];
        q1 = g->h_comp_off[c1];
        const int64_t n = q1 - q0;
        std::vector<Tile> ex, red;
        std::vector<int64_t> ex_comps;
        std::vector<int64_t> roff(1, 0);
        for (int64_t c = c0; c < c1; ++c) {
            int64_t a = g->h_comp_off[c], b = g->h_comp_off[c + 1];
            if (use_fmm_for(g, p, c)) {
                fmm.push_back(fmm_create(g, p, c));
                fmm_comp.push_back(c);
            } else {
                ex_comps.push_back(c);
            }
            for (int64_t t = a; t < b; t += RED_TILE) red.push_back(Tile{(int32_t)(c - c0), 0, t, std::min(b, t + RED_TILE)});
            roff.push_back((int64_t)red.size());
        }
        ex_r = exact_tile_choice(g, p, ex_comps);
        ex = exact_tiles(g, c0, ex_comps, ex_r);
        n_ex_tiles = (int)ex.size();
        n_red_tiles = (int)red.size();
        ex_tiles.reset(A, ex.size());
        red_tiles.reset(A, red.size());
        red_tile_off.reset(A, roff.size());
        if (!ex.empty())
            BGL_CUDA(cudaMemcpyAsync(ex_tiles.p, ex.data(), sizeof(Tile) * ex.size(), cudaMemcpyHostToDevice, s));
        BGL_CUDA(cudaMemcpyAsync(red_tiles.p, red.data(), sizeof(Tile) * red.size(), cudaMemcpyHostToDevice, s));
        BGL_CUDA(cudaMemcpyAsync(red_tile_off.p, roff.data(), sizeof(int64_t) * roff.size(), cudaMemcpyHostToDevice, s));
        f.reset(A, n);
        fa.reset(A, n);
        fprev.reset(A, n);
        BGL_CUDA(cudaMemsetAsync(fprev.p, 0, sizeof(float2) * n, s));
        partial.reset(A, red.size());
        std::vector<double> ones(c1 - c0, 1.0);
        sg.reset(A, c1 - c0);
        BGL_CUDA(cudaMemcpyAsync(sg.p, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, s));
        counter.reset(A, std::max<int64_t>(c1 - c0, 1));
        BGL_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned) * std::max<int64_t>(c1 - c0, 1), s));
        iter.reset(A, 1);
        BGL_CUDA(cudaMemsetAsync(iter.p, 0, sizeof(int), s));
        loop.reset(A, 1);
        // nodes of high degree: chunks of HEAVY_CHUNK adjacency entries
        DevBuf<int32_t> flag(A, n), fscan(A, n), tot(A, 1);
        heavy_flag_kernel<<<nblocks(n, 256), 256, 0, s>>>(g->coff.p, q0, n, flag.p);
        BGL_LAUNCH_CHECK();
        scan_exclusive_i32(g->ctx, flag.p, fscan.p, n, tot.p);
        int32_t nh = 0;
        BGL_CUDA(cudaMemcpyAsync(&nh, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        BGL_CUDA(cudaStreamSynchronize(s));
        std::vector<HeavyChunk> hc;
        if (nh > 0) {
            DevBuf<int32_t> heavy(A, nh);
            heavy_list_kernel<<<nblocks(n, 256), 256, 0, s>>>(flag.p, fscan.p, q0, n, heavy.p);
            BGL_LAUNCH_CHECK();
            DevBuf<int64_t> hrow(A, 2 * (size_t)nh);
            heavy_rows_kernel<<<nblocks(nh, 256), 256, 0, s>>>(heavy.p, g->coff.p, nh, hrow.p);
            BGL_LAUNCH_CHECK();
            std::vector<int32_t> hq(nh);
            std::vector<int64_t> ho(2 * (size_t)nh);
            BGL_CUDA(cudaMemcpyAsync(hq.data(), heavy.p, sizeof(int32_t) * nh, cudaMemcpyDeviceToHost, s));
            BGL_CUDA(cudaMemcpyAsync(ho.data(), hrow.p, sizeof(int64_t) * 2 * nh, cudaMemcpyDeviceToHost, s));
            BGL_CUDA(cudaStreamSynchronize(s));
            for (int32_t h = 0; h < nh; ++h) {
                const int64_t r0 = ho[2 * h], r1 = ho[2 * h + 1];
                const int32_t first = (int32_t)hc.size();
                const int32_t nchunk = (int32_t)((r1 - r0 + HEAVY_CHUNK - 1) / HEAVY_CHUNK);
                for (int32_t j = 0; j < nchunk; ++j)
                    hc.push_back(HeavyChunk{hq[h], h, first, nchunk, r0 + (int64_t)j * HEAVY_CHUNK,
                                            std::min<int64_t>(r1, r0 + (int64_t)(j + 1) * HEAVY_CHUNK)});
            }
        }
        n_chunks = (int64_t)hc.size();
        chunks.reset(A, hc.size());
        chunk_part.reset(A, hc.size());
        chunk_arrive.reset(A, std::max<int32_t>(nh, 1));
        BGL_CUDA(cudaMemsetAsync(chunk_arrive.p, 0, sizeof(int) * std::max<int32_t>(nh, 1), s));
        if (!hc.empty())
            BGL_CUDA(cudaMemcpyAsync(chunks.p, hc.data(), sizeof(HeavyChunk) * hc.size(), cudaMemcpyHostToDevice, s));
        BGL_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        BGL_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        BGL_CUDA(cudaEventCreateWithFlags(&ev_fa, cudaEventDisableTiming));
        BGL_CUDA(cudaStreamSynchronize(s));
    }
    ~Fa2Run() {
        for (auto *pl : fmm) fmm_destroy(pl);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_fa) cudaEventDestroy(ev_fa);
        if (side) cudaStreamDestroy(side);
    }

    // device-side failures of the FMM (bounded waits, capacities)
    void check_fmm() {
        for (auto *pl : fmm) {
            int e = fmm_error(pl);
            if (e & 1) fail(BGL_ETIMEOUT, "fmm: a bounded device-side wait gave up");
            if (e & 8) fail(BGL_ENUMERIC, "fmm: non-finite positions");
            if (e) fail(BGL_ENOMEM, "fmm: tree or list capacity exceeded (error bits " + std::to_string(e) + ")");
        }
    }

    // K1 + K2: f <- F (what 0) or F_rep (what 1).  K2 runs on the side
    // stream from the start; the repulsion kernels that write f last wait
    // for it (event ev_fa) and add fa.
    void forces(int what) {
        cudaStream_t s = g->ctx->stream;
        const bool att = what == 0;
        if (att) {
            BGL_RANGE("ForceAtlas2: attraction and gravity (Section 3.2)");
            BGL_CUDA(cudaEventRecord(ev_fork, s));
            BGL_CUDA(cudaStreamWaitEvent(side, ev_fork, 0));
            int64_t n = q1 - q0;
            int64_t nl = nblocks(n, 256);
            attraction_gravity_kernel<<<(unsigned)(nl + n_chunks), 256, 0, side>>>(
                xy, g->mass.p, g->coff.p, g->cadj.p, q0, q1, qbase, (float)p->kg, chunks.p, nl, chunk_part.p,
                chunk_arrive.p, fa.p - (q0 - qbase));
            BGL_LAUNCH_CHECK();
            BGL_CUDA(cudaEventRecord(ev_fa, side));
        }
        for (size_t k = 0; k < fmm.size(); ++k) {
            BGL_RANGE("ForceAtlas2: repulsion by the FMM (Section 3.2.1)");
            fmm_repulsion(fmm[k], xy, qbase, f.p, q0, att ? fa.p : nullptr, att ? ev_fa : nullptr);
        }
        if (att) BGL_CUDA(cudaStreamWaitEvent(s, ev_fa, 0));
        if (n_ex_tiles > 0) {
            BGL_RANGE("ForceAtlas2: exact repulsion (Section 3.2)");
            launch_exact(ex_r, n_ex_tiles, ex_tiles.p, g->comp_off.p, c0, xy, g->mass.p, qbase, (float)p->kr,
                         att ? fa.p - (q0 - qbase) : nullptr, f.p - (q0 - qbase), s);
        }
    }

    // one full iteration (K1..K4)
    void iteration(double *d_stats) {
        BGL_RANGE("ForceAtlas2 iteration: forces, swing/traction, update (Section 3.2)");
        cudaStream_t s = g->ctx->stream;
        if (fused) {
            // K3 in the FMM's combine pass, K4 with the next root square
            forces(0);
            BGL_RANGE("ForceAtlas2: node update (Section 3.2)");
            fmm_update_root(fmm[0], xy, qbase, f.p, fprev.p, q0);
            return;
        }
        forces(0);
        RedArgs a;
        a.tiles = red_tiles.p;
        a.tile_off = red_tile_off.p;
        a.ncomp = (int)(c1 - c0);
        a.f = f.p - (q0 - qbase);
        a.fprev = fprev.p - (q0 - qbase);
        a.mass = g->mass.p;
        a.qbase = qbase;
        a.variant = p->swing_variant;
        a.tau = p->tau;
        a.partial = partial.p;
        a.sg = sg.p;
        a.counter = counter.p;
        a.stats = d_stats;
        a.iter = iter.p;
        {
            BGL_RANGE("ForceAtlas2: swing and traction (Section 3.2)");
            swing_traction_kernel<<<n_red_tiles, 256, 0, s>>>(a);
            BGL_LAUNCH_CHECK();
        }
        BGL_RANGE("ForceAtlas2: node update (Section 3.2)");
        update_kernel<<<nblocks(q1 - q0, 256), 256, 0, s>>>(f.p - (q0 - qbase), fprev.p - (q0 - qbase), xy,
                                                            g->node_comp.p, sg.p, q0, q1, qbase, c0, (float)p->ks,
                                                            (float)p->ksmax, g->ctx->d_flag + 1);
        BGL_LAUNCH_CHECK();
    }
};

namespace {

// End of a loop iteration: count it and keep looping while below `iters`.
__global__ void loop_ctrl_kernel(cudaGraphConditionalHandle h, int *count, int iters) {
    const int k = ++*count;
    cudaGraphSetConditional(h, k < iters ? 1u : 0u);
}

}  // namespace

// With BGL_HOST_LOOP=1 in the environment, the iterations are launched
// from the host as one captured-iteration graph each instead of a device-side
// loop: profilers that cannot look inside graphs with conditional nodes can
// then see every kernel.  The results are the same.
static bool host_loop() {
    const char *v = std::getenv("BGL_HOST_LOOP");
    return v && v[0] == '1';
}

static void run_iterations_host(Fa2Run &run, int iters, double *d_stats, const SideWork &side) {
    bgl_ctx *ctx = run.g->ctx;
    cudaStream_t s = ctx->stream;
    cudaEvent_t side_done = nullptr;
    if (side) {
        // the side work on its own stream beside the iterations, joined after them
        BGL_CUDA(cudaEventCreateWithFlags(&side_done, cudaEventDisableTiming));
        BGL_CUDA(cudaEventRecord(run.ev_fork, s));
        BGL_CUDA(cudaStreamWaitEvent(run.side, run.ev_fork, 0));
        try {
            side(run.side);
            BGL_CUDA(cudaEventRecord(side_done, run.side));
        } catch (...) {
            cudaEventDestroy(side_done);
            throw;
        }
    }
    struct EventGuard {
        cudaEvent_t e;
        ~EventGuard() { if (e) cudaEventDestroy(e); }
    } side_guard{side_done};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int64_t before = launch_count();
    BGL_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    ctx->alloc->forbid = true;
    try {
        run.iteration(d_stats);
    } catch (...) {
        ctx->alloc->forbid = false;
        cudaGraph_t tmp = nullptr;
        cudaStreamEndCapture(s, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        throw;
    }
    ctx->alloc->forbid = false;
    BGL_CUDA(cudaStreamEndCapture(s, &graph));
    const int64_t per_iter = launch_count() - before;
    count_launches(-per_iter);
    try {
        BGL_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    } catch (...) {
        cudaGraphDestroy(graph);
        throw;
    }
    cudaGraphDestroy(graph);
    try {
        // a fused iteration finds the root square made by the previous one;
        // the first one's comes from the current positions
        if (run.fused) fmm_root(run.fmm[0], run.xy, run.qbase);
        for (int k = 0; k < iters; ++k) BGL_CUDA(cudaGraphLaunch(exec, s));
    } catch (...) {
        cudaGraphExecDestroy(exec);
        throw;
    }
    count_launches(per_iter * iters);
    if (side_done) BGL_CUDA(cudaStreamWaitEvent(s, side_done, 0));
    BGL_CUDA(cudaMemcpyAsync(ctx->h_flag + 1, ctx->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    cudaGraphExecDestroy(exec);
    run.check_fmm();
    if (ctx->h_flag[1]) fail(BGL_ENUMERIC, "fa2: a position became non-finite");
}

// All `iters` iterations of `run` in one graph launch: the graph holds a
// WHILE conditional node whose body is one captured iteration followed by a
// one-thread kernel that counts the iterations and clears the condition
// after the last, so the loop runs on the device without the host.
// Nothing may allocate while the capture is open.
static void run_iterations(Fa2Run &run, int iters, double *d_stats, const SideWork &side = SideWork()) {
    bgl_ctx *ctx = run.g->ctx;
    cudaStream_t s = ctx->stream;
    if (iters <= 0) {
        if (side) side(s);
        return;
    }
    BGL_CUDA(cudaMemsetAsync(ctx->d_flag + 1, 0, sizeof(int), s));
    BGL_CUDA(cudaMemsetAsync(run.iter.p, 0, sizeof(int), s));
    BGL_CUDA(cudaMemsetAsync(run.loop.p, 0, sizeof(int), s));
    run.enable_fuse(d_stats);
    if (host_loop()) {
        run_iterations_host(run, iters, d_stats, side);
        return;
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    BGL_CUDA(cudaGraphCreate(&graph, 0));
    int64_t kernels = 0;
    try {
        cudaGraphConditionalHandle h;
        BGL_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        BGL_CUDA(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        const int64_t before = launch_count();
        BGL_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        ctx->alloc->forbid = true;
        try {
            run.iteration(d_stats);
            loop_ctrl_kernel<<<1, 1, 0, s>>>(h, run.loop.p, iters);
            BGL_LAUNCH_CHECK();
        } catch (...) {
            ctx->alloc->forbid = false;
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(s, &tmp);
            throw;
        }
        ctx->alloc->forbid = false;
        cudaGraph_t captured = nullptr;
        BGL_CUDA(cudaStreamEndCapture(s, &captured));
        // captured launches run only when the graph does
        count_launches(before - launch_count());
        size_t nn = 0;
        BGL_CUDA(cudaGraphGetNodes(body, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) BGL_CUDA(cudaGraphGetNodes(body, nodes.data(), &nn));
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            BGL_CUDA(cudaGraphNodeGetType(nd, &t));
            if (t == cudaGraphNodeTypeKernel) ++kernels;
        }
        if (side) {
            // the side work, captured on the run's side stream (it may fork
            // to streams of its own), becomes a child graph beside the loop
            cudaGraph_t child = nullptr;
            BGL_CUDA(cudaStreamBeginCapture(run.side, cudaStreamCaptureModeThreadLocal));
            ctx->alloc->forbid = true;
            try {
                side(run.side);
            } catch (...) {
                ctx->alloc->forbid = false;
                cudaGraph_t tmp = nullptr;
                cudaStreamEndCapture(run.side, &tmp);
                if (tmp) cudaGraphDestroy(tmp);
                throw;
            }
            ctx->alloc->forbid = false;
            BGL_CUDA(cudaStreamEndCapture(run.side, &child));
            cudaGraphNode_t cn;
            const cudaError_t e = cudaGraphAddChildGraphNode(&cn, graph, nullptr, 0, child);
            cudaGraphDestroy(child);
            BGL_CUDA(e);
        }
        BGL_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    } catch (...) {
        cudaGraphDestroy(graph);
        throw;
    }
    cudaGraphDestroy(graph);
    count_launches(kernels * iters);
    try {
        if (run.fused) fmm_root(run.fmm[0], run.xy, run.qbase);
        BGL_CUDA(cudaGraphLaunch(exec, s));
    } catch (...) {
        cudaGraphExecDestroy(exec);
        throw;
    }
    BGL_CUDA(cudaMemcpyAsync(ctx->h_flag + 1, ctx->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    cudaGraphExecDestroy(exec);
    run.check_fmm();
    if (ctx->h_flag[1]) fail(BGL_ENUMERIC, "fa2: a position became non-finite");
}

void fa2_layout(bgl_graph *g, const bgl_params *p, float2 *xy, int64_t qbase, int64_t c0, int64_t c1, int iters,
                double *d_stats, const SideWork &side) {
    if (c1 <= c0 || iters <= 0) {
        if (side) side(g->ctx->stream);
        return;
    }
    BGL_RANGE("ForceAtlas2 iterations (Section 3.2)");
    Fa2Run run(g, p, xy, qbase, c0, c1);
    run_iterations(run, iters, d_stats, side);
}

// ---------------------------------------------------------------- resumable runs

namespace {

// 64-bit FNV-1a over a byte range
uint64_t fnv1a(uint64_t h, const void *data, size_t len) {
    const unsigned char *b = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < len; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

// Identity of component c of g: its size, position in the component order,
// node ids and adjacency rows (a checkpoint loads only into the same graph).
uint64_t component_fingerprint(bgl_graph *g, int64_t c) {
    const int64_t q0 = g->h_comp_off[c], q1 = g->h_comp_off[c + 1], n = q1 - q0;
    std::vector<int32_t> nodes(n);
    std::vector<int64_t> coff(n + 1);
    cudaStream_t s = g->ctx->stream;
    BGL_CUDA(cudaMemcpyAsync(nodes.data(), g->nodes.p + q0, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaMemcpyAsync(coff.data(), g->coff.p + q0, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    const int64_t e0 = coff[0], e1 = coff[n];
    std::vector<int32_t> cadj(e1 - e0);
    if (e1 > e0)
        BGL_CUDA(cudaMemcpyAsync(cadj.data(), g->cadj.p + e0, sizeof(int32_t) * (e1 - e0), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    for (auto &o : coff) o -= e0;
    uint64_t h = 0xcbf29ce484222325ull;
    const int64_t head[4] = {g->n, g->n_undir, c, n};
    h = fnv1a(h, head, sizeof(head));
    h = fnv1a(h, nodes.data(), sizeof(int32_t) * n);
    h = fnv1a(h, coff.data(), sizeof(int64_t) * (n + 1));
    h = fnv1a(h, cadj.data(), sizeof(int32_t) * cadj.size());
    return h;
}

// checkpoint layout: this header, then n float2 positions and n float2 F_{t-1}
struct StateHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int64_t n_nodes, n_undir, comp, comp_nodes;
    uint64_t fingerprint;
    int64_t iters_done;
    double sg;
    int32_t fmm_sortskip;          // FMM sort passes the next evaluation skips (-1: exact repulsion)
    int32_t pad;
    bgl_params params;
};
constexpr char STATE_MAGIC[8] = {'B', 'G', 'L', 'F', 'A', '2', 'S', 'T'};
constexpr uint32_t STATE_VERSION = 1;

}  // namespace

struct Fa2Session {
    bgl_graph *g = nullptr;
    bgl_params p;                  // owned copy (the run keeps a pointer to it)
    int64_t c = 0, q0 = 0, n = 0;
    int64_t iters_done = 0;
    uint64_t fingerprint = 0;
    DevBuf<float2> xy;             // positions, xy[q - q0]
    Fa2Run *run = nullptr;
    ~Fa2Session() { delete run; }
};

static Fa2Session *session_new(bgl_graph *g, const bgl_params *p, int64_t c) {
    Fa2Session *s = new Fa2Session();
    try {
        s->g = g;
        s->p = *p;
        s->c = c;
        s->q0 = g->h_comp_off[c];
        s->n = g->h_comp_off[c + 1] - s->q0;
        s->xy.reset(g->ctx->alloc, std::max<int64_t>(s->n, 1));
        s->run = new Fa2Run(g, &s->p, s->xy.p, s->q0, c, c + 1);
        s->fingerprint = component_fingerprint(g, c);
    } catch (...) {
        delete s;
        throw;
    }
    return s;
}

Fa2Session *fa2_session_create(bgl_graph *g, const bgl_params *p, int64_t c, const float2 *h_xy) {
    Fa2Session *s = session_new(g, p, c);
    try {
        BGL_CUDA(cudaMemcpyAsync(s->xy.p, h_xy, sizeof(float2) * s->n, cudaMemcpyHostToDevice, g->ctx->stream));
        BGL_CUDA(cudaStreamSynchronize(g->ctx->stream));
    } catch (...) {
        delete s;
        throw;
    }
    return s;
}

void fa2_session_destroy(Fa2Session *s) { delete s; }

void fa2_session_advance(Fa2Session *s, int iters, double *h_stats) {
    if (iters <= 0) return;
    bgl_ctx *ctx = s->g->ctx;
    DevBuf<double> st;
    if (h_stats) st.reset(ctx->alloc, 3 * (size_t)iters);
    run_iterations(*s->run, iters, h_stats ? st.p : nullptr);
    s->iters_done += iters;
    if (h_stats) {
        BGL_CUDA(cudaMemcpyAsync(h_stats, st.p, sizeof(double) * 3 * iters, cudaMemcpyDeviceToHost, ctx->stream));
        BGL_CUDA(cudaStreamSynchronize(ctx->stream));
    }
}

int64_t fa2_session_positions(Fa2Session *s, float2 *h_xy) {
    cudaStream_t st = s->g->ctx->stream;
    BGL_CUDA(cudaMemcpyAsync(h_xy, s->xy.p, sizeof(float2) * s->n, cudaMemcpyDeviceToHost, st));
    BGL_CUDA(cudaStreamSynchronize(st));
    return s->iters_done;
}

size_t fa2_session_state_bytes(const Fa2Session *s) { return sizeof(StateHeader) + 2 * sizeof(float2) * s->n; }

void fa2_session_save(Fa2Session *s, void *buf) {
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, STATE_MAGIC, 8);
    h.version = STATE_VERSION;
    h.header_bytes = (uint32_t)sizeof(StateHeader);
    h.n_nodes = s->g->n;
    h.n_undir = s->g->n_undir;
    h.comp = s->c;
    h.comp_nodes = s->n;
    h.fingerprint = s->fingerprint;
    h.iters_done = s->iters_done;
    h.params = s->p;
    h.fmm_sortskip = s->run->fmm.empty() ? -1 : fmm_sortskip(s->run->fmm[0]);
    cudaStream_t st = s->g->ctx->stream;
    BGL_CUDA(cudaMemcpyAsync(&h.sg, s->run->sg.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    char *out = static_cast<char *>(buf);
    float2 *xy = reinterpret_cast<float2 *>(out + sizeof(StateHeader));
    BGL_CUDA(cudaMemcpyAsync(xy, s->xy.p, sizeof(float2) * s->n, cudaMemcpyDeviceToHost, st));
    BGL_CUDA(cudaMemcpyAsync(xy + s->n, s->run->fprev.p, sizeof(float2) * s->n, cudaMemcpyDeviceToHost, st));
    BGL_CUDA(cudaStreamSynchronize(st));
    std::memcpy(out, &h, sizeof(h));
}

Fa2Session *fa2_session_load(bgl_graph *g, const void *buf, size_t len) {
    BGL_REQUIRE(len >= sizeof(StateHeader), "state: buffer shorter than the header");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, STATE_MAGIC, 8) != 0 || h.version != STATE_VERSION ||
        h.header_bytes != sizeof(StateHeader))
        fail(BGL_EINVAL, "state: not a ForceAtlas2 checkpoint of this library version");
    if (!g->has_comp) fail(BGL_ESTATE, "state: run bgl_components before loading a checkpoint");
    if (h.n_nodes != g->n || h.n_undir != g->n_undir || h.comp < 0 || h.comp >= g->n_comp ||
        h.comp_nodes != g->h_comp_off[h.comp + 1] - g->h_comp_off[h.comp])
        fail(BGL_EINVAL, "state: the checkpoint belongs to another graph");
    BGL_REQUIRE(len >= sizeof(StateHeader) + 2 * sizeof(float2) * (size_t)h.comp_nodes,
                "state: buffer shorter than the checkpoint");
    check_params(&h.params);
    Fa2Session *s = session_new(g, &h.params, h.comp);
    try {
        if (s->fingerprint != h.fingerprint) fail(BGL_EINVAL, "state: the checkpoint belongs to another graph");
        const float2 *xy = reinterpret_cast<const float2 *>(static_cast<const char *>(buf) + sizeof(StateHeader));
        cudaStream_t st = g->ctx->stream;
        BGL_CUDA(cudaMemcpyAsync(s->xy.p, xy, sizeof(float2) * s->n, cudaMemcpyHostToDevice, st));
        BGL_CUDA(cudaMemcpyAsync(s->run->fprev.p, xy + s->n, sizeof(float2) * s->n, cudaMemcpyHostToDevice, st));
        BGL_CUDA(cudaMemcpyAsync(s->run->sg.p, &h.sg, sizeof(double), cudaMemcpyHostToDevice, st));
        BGL_CUDA(cudaStreamSynchronize(st));
        if ((h.fmm_sortskip >= 0) != !s->run->fmm.empty()) fail(BGL_EINVAL, "state: repulsion kind mismatch");
        if (h.fmm_sortskip >= 0) fmm_set_sortskip(s->run->fmm[0], h.fmm_sortskip);
        s->iters_done = h.iters_done;
    } catch (...) {
        delete s;
        throw;
    }
    return s;
}

void fa2_forces(bgl_graph *g, const bgl_params *p, const float2 *xy, float2 *f, int64_t c, int what) {
    int64_t q0 = g->h_comp_off[c];
    Fa2Run run(g, p, const_cast<float2 *>(xy), q0, c, c + 1);
    run.forces(what);
    BGL_CUDA(cudaMemcpyAsync(f, run.f.p, sizeof(float2) * (run.q1 - run.q0), cudaMemcpyDeviceToDevice,
                             g->ctx->stream));
    BGL_CUDA(cudaStreamSynchronize(g->ctx->stream));
    run.check_fmm();
}

}  // namespace bgl
