// Allocation-free ForceAtlas2 iteration on caller-owned device arrays.
//
// Some callers cannot call cudaMalloc at the point where they want to run a
// layout step: a serving process that hands all of its device memory to
// its own pool at start-up has nothing left for a library to allocate, and
// a latency-bound loop cannot afford the device-wide synchronisation that
// cudaMalloc and cudaFree may cause.  bgl_fa2_iteration_noalloc serves them:
// the caller passes every input and output, and the only scratch the
// iteration needs -- the per-tile swing/traction partial sums and the
// arrival counter of their reduction -- lives in one file-scope device
// array of fixed size (NOALLOC_SCRATCH_BYTES), which every GPU that loads
// this library holds until the process exits.
//
// The kernels are variants of the ones in fa2.cu that need no host-built
// tile list and no per-call buffers: one component, targets tiled by block
// index, hub rows summed by the node's own thread.  The formulas of every
// force term, of the swing/traction sums and of the update are the same;
// the order and precision of the sums differ (here every thread sums its
// swing/traction terms in FP64 over tiles of 2,048 nodes and a hub's
// attraction in one loop, where fa2.cu sums in FP32 within a warp over tiles
// of 1,024 nodes and splits hub rows into 2,048-entry chunks), so the two
// agree within rounding, not bitwise.  A position that becomes non-finite
// sets the context's d_flag[2], which bgl_ctx_sync reports.
#include "bgl_internal.cuh"

namespace bgl {

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_R = 2;                           // targets per thread
constexpr int NA_TILE = NA_THREADS * NA_R;        // targets per block
constexpr int NA_STILE = 1024;                    // sources per shared-memory stage
constexpr int NA_RED_TILE = 2048;                 // nodes per swing/traction tile
constexpr int64_t NA_MAX_NODES = BGL_NOALLOC_MAX_NODES;
constexpr int NA_MAX_TILES = (int)(NA_MAX_NODES / NA_RED_TILE);
constexpr size_t NA_COUNTER_BYTES = 256;          // arrival counter, padded
constexpr size_t NOALLOC_SCRATCH_BYTES = NA_COUNTER_BYTES + sizeof(double2) * NA_MAX_TILES;

// The scratch of every call on this device: [0, 256) the arrival counter,
// then NA_MAX_TILES double2 partial sums.  Host code must not pass this
// symbol to a kernel; it passes the device address from
// cudaGetSymbolAddress (noalloc_scratch_address, stored in the context).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

__device__ __forceinline__ float na_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// repulsion of targets [blockIdx.x * NA_TILE, ...) from all n nodes
__global__ void __launch_bounds__(NA_THREADS) na_repulsion_kernel(const float2 *__restrict__ xy,
                                                                 const float *__restrict__ mass, int64_t n, float kr,
                                                                 float2 *__restrict__ f) {
    __shared__ float4 src[NA_STILE];
    const int64_t t0 = (int64_t)blockIdx.x * NA_TILE;
    float xi[NA_R], yi[NA_R], sx[NA_R], sy[NA_R], cx[NA_R], cy[NA_R];
#pragma unroll
    for (int r = 0; r < NA_R; ++r) {
        int64_t q = t0 + threadIdx.x + r * NA_THREADS;
        float2 p = q < n ? xy[q] : make_float2(0.f, 0.f);
        xi[r] = p.x;
        yi[r] = p.y;
        sx[r] = sy[r] = cx[r] = cy[r] = 0.f;
    }
    for (int64_t s0 = 0; s0 < n; s0 += NA_STILE) {
        const int cnt = (int)(n - s0 < NA_STILE ? n - s0 : NA_STILE);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += NA_THREADS) {
            float2 p = xy[s0 + k];
            src[k] = make_float4(p.x, p.y, mass[s0 + k], 0.f);
        }
        __syncthreads();
        float ax[NA_R], ay[NA_R];
#pragma unroll
        for (int r = 0; r < NA_R; ++r) ax[r] = ay[r] = 0.f;
#pragma unroll 4
        for (int j = 0; j < cnt; ++j) {
            const float4 s = src[j];
#pragma unroll
            for (int r = 0; r < NA_R; ++r) {
                float dx = xi[r] - s.x, dy = yi[r] - s.y;
                float r2 = fmaf(dx, dx, dy * dy);
                float w = s.z * na_rcp(fmaxf(r2, 1e-30f));   // the node itself adds 0
                ax[r] = fmaf(w, dx, ax[r]);
                ay[r] = fmaf(w, dy, ay[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NA_R; ++r) {   // compensated running total of the stage sums
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
    for (int r = 0; r < NA_R; ++r) {
        int64_t q = t0 + threadIdx.x + r * NA_THREADS;
        if (q >= n) continue;
        float km = kr * mass[q];
        f[q] = make_float2(km * sx[r], km * sy[r]);
    }
}

// attraction and gravity added to f, one thread per node
__global__ void na_attraction_gravity_kernel(const float2 *__restrict__ xy, const float *__restrict__ mass,
                                             const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                             int64_t n, float kg, float2 *__restrict__ f) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float2 p = xy[q];
    float ax = 0.f, ay = 0.f;
    for (int64_t e = off[q]; e < off[q + 1]; ++e) {
        float2 o = xy[adj[e]];
        ax -= p.x - o.x;
        ay -= p.y - o.y;
    }
    float km = kg * mass[q];
    float2 fr = f[q];
    f[q] = make_float2((fr.x + ax) - km * p.x, (fr.y + ay) - km * p.y);
}

// swing / traction partial sums per tile into the static scratch; the last
// block sums the tiles in order and sets s_G = min(tau trc / swg, 1.5 s_G)
__global__ void na_swing_traction_kernel(const float2 *__restrict__ f, const float2 *__restrict__ fprev,
                                         const float *__restrict__ mass, int64_t n, int variant, double tau,
                                         double *sg, unsigned char *scratch) {
    __shared__ double ws[32], wt[32];
    __shared__ bool last;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch);
    double2 *partial = reinterpret_cast<double2 *>(scratch + NA_COUNTER_BYTES);
    const int64_t t0 = (int64_t)blockIdx.x * NA_RED_TILE;
    const int64_t t1 = t0 + NA_RED_TILE < n ? t0 + NA_RED_TILE : n;
    double sw = 0.0, tr = 0.0;
    for (int64_t q = t0 + threadIdx.x; q < t1; q += blockDim.x) {
        float2 F = f[q], P = fprev[q];
        float s = sqrtf((F.x - P.x) * (F.x - P.x) + (F.y - P.y) * (F.y - P.y));
        float u = sqrtf((F.x + P.x) * (F.x + P.x) + (F.y + P.y) * (F.y + P.y));
        if (variant == 1) {
            float m = mass[q];
            sw += (double)m * s;
            tr += 0.5 * (double)m * u;
        } else {
            sw += s;
            tr += u;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        ws[warp] = sw;
        wt[warp] = tr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, u = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s += ws[w];
            u += wt[w];
        }
        partial[blockIdx.x] = make_double2(s, u);
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double swg = 0.0, trc = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
        double2 v = __ldcg(&partial[k]);
        swg += v.x;
        trc += v.y;
    }
    double g = *sg;
    double s_new = swg > 0.0 ? tau * trc / swg : 1.5 * g;
    if (s_new > 1.5 * g) s_new = 1.5 * g;
    *sg = s_new;
    *counter = 0u;
}

__global__ void na_update_kernel(const float2 *__restrict__ f, float2 *__restrict__ fprev, float2 *__restrict__ xy,
                                 const double *__restrict__ sg, int64_t n, float ks, float ksmax, int *bad) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float2 F = f[q], P = fprev[q];
    float g = (float)*sg;
    float sw = sqrtf((F.x - P.x) * (F.x - P.x) + (F.y - P.y) * (F.y - P.y));
    float s = ks * g / (1.f + g * sqrtf(sw));
    float fn = sqrtf(F.x * F.x + F.y * F.y);
    if (fn > 0.f && s > ksmax / fn) s = ksmax / fn;
    float2 p = xy[q];
    p.x += s * F.x;
    p.y += s * F.y;
    if (!isfinite(p.x) || !isfinite(p.y)) *bad = 1;
    xy[q] = p;
    fprev[q] = F;
}

inline unsigned na_blocks(int64_t n, int64_t per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

// Device address of the scratch array on the current device.  Called by
// bgl_ctx_create with the context's device current, so every context holds
// the address for its device (a context created after a device reset looks
// it up again).
void *noalloc_scratch_address() {
    void *ptr = nullptr;
    BGL_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    return ptr;
}

void fa2_iteration_noalloc(bgl_ctx *c, int64_t n, const int64_t *d_off, const int32_t *d_adj, const float *d_mass,
                           float2 *d_xy, float2 *d_fprev, float2 *d_f, double *d_sg, const bgl_params *p) {
    BGL_REQUIRE(n >= 0, "noalloc: n must be >= 0");
    BGL_REQUIRE(n <= NA_MAX_NODES, "noalloc: component has more than BGL_NOALLOC_MAX_NODES (2^20) nodes");
    if (n == 0) return;
    BGL_REQUIRE(d_off && d_adj && d_mass && d_xy && d_fprev && d_f && d_sg, "noalloc: a device array is NULL");
    unsigned char *scratch = c->noalloc_scratch;
    BGL_REQUIRE(scratch != nullptr, "noalloc: the context has no scratch address");
    cudaStream_t s = c->stream;
    // the arrival counter must start at zero; the partial sums are overwritten
    BGL_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned), s));
    na_repulsion_kernel<<<na_blocks(n, NA_TILE), NA_THREADS, 0, s>>>(d_xy, d_mass, n, (float)p->kr, d_f);
    BGL_LAUNCH_CHECK();
    na_attraction_gravity_kernel<<<na_blocks(n, 256), 256, 0, s>>>(d_xy, d_mass, d_off, d_adj, n, (float)p->kg, d_f);
    BGL_LAUNCH_CHECK();
    na_swing_traction_kernel<<<na_blocks(n, NA_RED_TILE), 256, 0, s>>>(d_f, d_fprev, d_mass, n, p->swing_variant,
                                                                       p->tau, d_sg, scratch);
    BGL_LAUNCH_CHECK();
    na_update_kernel<<<na_blocks(n, 256), 256, 0, s>>>(d_f, d_fprev, d_xy, d_sg, n, (float)p->ks, (float)p->ksmax,
                                                       c->d_flag + 2);
    BGL_LAUNCH_CHECK();
}

}  // namespace bgl
