// Device primitives: multi-block exclusive scan and stable LSD radix sort.
//
// Scan: reduce-then-scan over tiles of 4096 elements (512 threads x 8).
// Radix sort: 8-bit digits, tiles of 4096 keys (8 warps x 32 lanes x 16
// rounds).  Per pass: a per-tile digit histogram (shared-memory integer
// atomics), one exclusive scan of the digit-major histogram, and a scatter
// in which each warp ranks its keys with __match_any_sync so that equal
// digits keep their input order (stable).
#include <algorithm>

#include "bgl_internal.cuh"
#include "sort_hist.cuh"

namespace bgl {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_tot, T *total) {
    // exclusive scan of one value per thread across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? warp_tot[lane] : T(0);
        T s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nwarps) warp_tot[lane] = s - w;   // exclusive warp offsets
        if (lane == nwarps - 1) *total = s;
    }
    __syncthreads();
    T r = warp_tot[warp] + x - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void scan_reduce_kernel(const T *__restrict__ in, T *__restrict__ tile_sum, int64_t n) {
    __shared__ T red[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t k = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (k < n) s += in[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
        tile_sum[blockIdx.x] = t;
    }
}

// single block: exclusive scan of the tile sums, in place; total to *d_total
template <typename T>
__global__ void scan_tiles_kernel(T *tile_sum, int64_t ntiles, T *d_total) {
    __shared__ T wt[32];
    __shared__ T tot;
    T carry = 0;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        int64_t k = b + threadIdx.x;
        T v = k < ntiles ? tile_sum[k] : T(0);
        T e = block_exclusive_scan<T>(v, wt, &tot);
        if (k < ntiles) tile_sum[k] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

template <typename T>
__global__ void scan_apply_kernel(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ tile_off,
                                  int64_t n) {
    __shared__ T buf[SCAN_TILE];
    __shared__ T wt[32];
    __shared__ T tot;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int idx = i * SCAN_THREADS + threadIdx.x;
        int64_t k = base + idx;
        buf[idx] = k < n ? in[k] : T(0);
    }
    __syncthreads();
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = buf[threadIdx.x * SCAN_ITEMS + i];
        s += v[i];
    }
    T e = block_exclusive_scan<T>(s, wt, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        buf[threadIdx.x * SCAN_ITEMS + i] = e;
        e += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int idx = i * SCAN_THREADS + threadIdx.x;
        int64_t k = base + idx;
        if (k < n) out[k] = buf[idx];
    }
}

template <typename T>
void scan_exclusive(bgl_ctx *c, const T *in, T *out, int64_t n, T *d_total, T *tiles = nullptr) {
    if (n <= 0) {
        if (d_total) BGL_CUDA(cudaMemsetAsync(d_total, 0, sizeof(T), c->stream));
        return;
    }
    int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    DevBuf<T> own;
    if (!tiles) {
        own.reset(c->alloc, ntiles);
        tiles = own.p;
    }
    scan_reduce_kernel<T><<<(unsigned)ntiles, SCAN_THREADS, 0, c->stream>>>(in, tiles, n);
    BGL_LAUNCH_CHECK();
    scan_tiles_kernel<T><<<1, 1024, 0, c->stream>>>(tiles, ntiles, d_total);
    BGL_LAUNCH_CHECK();
    scan_apply_kernel<T><<<(unsigned)ntiles, SCAN_THREADS, 0, c->stream>>>(in, out, tiles, n);
    BGL_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

template <typename K>
__global__ void radix_hist_kernel(const K *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ hist,
                                  int64_t ntiles) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_ITEMS; ++i) {
        int64_t k = base + (int64_t)i * RS_THREADS + threadIdx.x;
        if (k < n) atomicAdd(&h[(unsigned)((keys[k] >> shift) & 0xFF)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) radix_scatter_kernel(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                              K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                              int64_t n, int shift,
                                                              const int32_t *__restrict__ offs, int64_t ntiles) {
    __shared__ int32_t cnt[RS_WARPS][256];
    __shared__ int32_t gbase[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&cnt[0][0])[i] = 0;
    gbase[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * 32 * RS_ITEMS;
    K key[RS_ITEMS];
    uint32_t val[RS_ITEMS];
    int32_t rank[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t k = wbase + r * 32 + lane;
        bool ok = k < n;
        key[r] = ok ? kin[k] : K(0);
        val[r] = (ok && vin) ? vin[k] : 0u;
        unsigned d = ok ? (unsigned)((key[r] >> shift) & 0xFF) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = __popc(peers & lt);
        int cur = ok ? cnt[warp][d] : 0;
        __syncwarp();
        if (ok && before == 0) cnt[warp][d] = cur + __popc(peers);
        __syncwarp();
        rank[r] = ok ? (cur + before) : -1;
    }
    __syncthreads();
    {   // exclusive prefix over warps for digit threadIdx.x
        int d = threadIdx.x;
        int s = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            int c = cnt[w][d];
            cnt[w][d] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        if (rank[r] < 0) continue;
        unsigned d = (unsigned)((key[r] >> shift) & 0xFF);
        int64_t dst = (int64_t)gbase[d] + cnt[warp][d] + rank[r];
        kout[dst] = key[r];
        if (vout) vout[dst] = val[r];
    }
}

template <typename K>
void radix_sort_buffers(bgl_ctx *c, K *keys, uint32_t *vals, int64_t n, int bits, K *ktmp, uint32_t *vtmp,
                        int32_t *hist, int32_t *tiles) {
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    K *ka = keys, *kb = ktmp;
    uint32_t *va = vals, *vb = vals ? vtmp : nullptr;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        radix_hist_kernel<K><<<(unsigned)ntiles, RS_THREADS, 0, c->stream>>>(ka, n, shift, hist, ntiles);
        BGL_LAUNCH_CHECK();
        scan_exclusive<int32_t>(c, hist, hist, 256 * ntiles, nullptr, tiles);
        radix_scatter_kernel<K><<<(unsigned)ntiles, RS_THREADS, 0, c->stream>>>(ka, va, kb, vb, n, shift, hist,
                                                                                ntiles);
        BGL_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {
        BGL_CUDA(cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, c->stream));
        if (vals) BGL_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
}

inline int64_t rs_tiles(int64_t n) { return (n + RS_TILE - 1) / RS_TILE; }
inline int64_t scan_tiles_for(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

template <typename K>
void radix_sort(bgl_ctx *c, K *keys, uint32_t *vals, int64_t n, int bits) {
    if (n <= 1 || bits <= 0) return;
    BGL_REQUIRE(n < (int64_t(1) << 31), "radix sort: more than 2^31 keys");
    const int64_t ntiles = rs_tiles(n);
    DevBuf<K> kt(c->alloc, n);
    DevBuf<uint32_t> vt;
    if (vals) vt.reset(c->alloc, n);
    DevBuf<int32_t> hist(c->alloc, 256 * ntiles), tiles(c->alloc, scan_tiles_for(256 * ntiles));
    radix_sort_buffers<K>(c, keys, vals, n, bits, kt.p, vals ? vt.p : nullptr, hist.p, tiles.p);
}

// ------------------------------------------------------------------ onesweep (32-bit keys)
//
// Four 8-bit digit passes.  One histogram kernel counts all four digit
// histograms at once and its last block turns them into global digit
// bases.  Each pass is then a single kernel: tiles take increasing indices
// from a ticket counter, rank their keys stably (per-warp __match_any_sync
// counts, warps in order), publish their per-digit counts, and look back
// over earlier tiles' published counts (decoupled look-back, Merrill and
// Garland) for their global offsets; keys are regrouped by digit in shared
// memory so each digit run is written with coalesced stores.  Waits are
// bounded; a wait that gives up records an error bit and the tile carries on.

// OS_THREADS, OS_ITEMS, OS_TILE: sort_hist.cuh (a caller's histogram kernel uses the same tiles)
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr uint32_t OS_AGG = 1u << 30, OS_INC = 2u << 30, OS_MASK = (1u << 30) - 1u;
constexpr long long OS_SPIN = 1ll << 24;
constexpr int OS_LB = 8;           // look-back window (predecessor tiles per step)

// digit histograms of the keys, OS_ITEMS per thread
__global__ void __launch_bounds__(OS_THREADS) os_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, OsHist h) {
    uint32_t k[OS_ITEMS];
    unsigned valid = 0;
    const int64_t i0 = (int64_t)blockIdx.x * OS_TILE + threadIdx.x;
#pragma unroll
    for (int r = 0; r < OS_ITEMS; ++r) {
        const int64_t i = i0 + (int64_t)r * OS_THREADS;
        k[r] = i < n ? keys[i] : 0u;
        if (i < n) valid |= 1u << r;
    }
    os_block_hist<OS_ITEMS>(k, valid, h);
}

// Buffers of pass d (0..3) when the first `skip` passes are skipped: the
// first active pass reads the input, the last writes the output, the ones
// between alternate between the two scratch pairs.
struct OsBufs {
    uint32_t *keys, *vals;      // input, and output of the last pass
    uint32_t *k0, *v0, *k1, *v1; // scratch
};

__global__ void __launch_bounds__(OS_THREADS, 2) os_scatter_kernel(OsBufs bf, int d, const int *d_skip, int64_t n,
                                                                 const uint32_t *__restrict__ base,
                                                                 uint32_t *status, unsigned *ticket, int *err,
                                                                 const float2 *__restrict__ gxy,
                                                                 const float *__restrict__ gmass,
                                                                 float4 *__restrict__ gpts, OsWait wait) {
    const int skip = d_skip ? *d_skip : 0;
    if (d < skip) return;
    const int shift = 8 * d;
    const uint32_t *__restrict__ kin = d == skip ? bf.keys : (((d - skip - 1) & 1) ? bf.k1 : bf.k0);
    const uint32_t *__restrict__ vin = d == skip ? bf.vals : (((d - skip - 1) & 1) ? bf.v1 : bf.v0);
    uint32_t *__restrict__ kout = d == 3 ? bf.keys : (((d - skip) & 1) ? bf.k1 : bf.k0);
    uint32_t *__restrict__ vout = d == 3 ? bf.vals : (((d - skip) & 1) ? bf.v1 : bf.v0);
    __shared__ int32_t cnt[OS_WARPS][256];
    __shared__ uint32_t gofs[256];
    __shared__ int32_t lstart[256];
    __shared__ int32_t wsum[OS_WARPS];
    __shared__ uint32_t skey[OS_TILE], sval[OS_TILE];
    __shared__ int tile_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // after a wait gave up (in an earlier pass, or in this one before the
    // block started) the keys are not sorted: blocks return before taking
    // a tile, so no tile is left waiting for one that nobody holds
    if (threadIdx.x == 0) tile_s = (*(volatile int *)err & 1) ? -1 : (int)atomicAdd(ticket, 1u);
    for (int i = threadIdx.x; i < OS_WARPS * 256; i += OS_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int tile = tile_s;
    if (tile < 0) return;
    const int64_t t0 = (int64_t)tile * OS_TILE;
    const int tcount = (int)(n - t0 < OS_TILE ? n - t0 : OS_TILE);
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wbase = t0 + (int64_t)warp * 32 * OS_ITEMS;
    uint32_t key[OS_ITEMS], val[OS_ITEMS];
    int32_t rank[OS_ITEMS];
    // all loads in flight before the ranking (whose warp barriers would
    // otherwise order them one after another)
#pragma unroll
    for (int r = 0; r < OS_ITEMS; ++r) {
        const int64_t k = wbase + r * 32 + lane;
        key[r] = k < n ? kin[k] : 0u;
        val[r] = k < n ? vin[k] : 0u;
    }
#pragma unroll
    for (int r = 0; r < OS_ITEMS; ++r) {
        const int64_t k = wbase + r * 32 + lane;
        const bool ok = k < n;
        const unsigned d = ok ? ((key[r] >> shift) & 0xFF) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before = __popc(peers & lt);
        const int cur = ok ? cnt[warp][d] : 0;
        __syncwarp();
        if (ok && before == 0) cnt[warp][d] = cur + __popc(peers);
        __syncwarp();
        rank[r] = ok ? cur + before : -1;
    }
    __syncthreads();
    {
        // thread = digit: prefix over warps, then an exclusive scan over digits
        // (tile-local start of each digit run), then the look-back for the
        // global offset of each digit run
        const int d = threadIdx.x;
        int s = 0;
#pragma unroll
        for (int w = 0; w < OS_WARPS; ++w) {
            const int c = cnt[w][d];
            cnt[w][d] = s;
            s += c;
        }
        int x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        volatile uint32_t *st = status;
        const uint32_t own = (uint32_t)s;
        uint32_t excl = 0;
        if (tile == 0) {
            if (!wait.stall_first) st[d] = OS_INC | own;
        } else {
            st[(int64_t)tile * 256 + d] = OS_AGG | own;
            // look back OS_LB predecessors per step: their status words are
            // loaded together, then taken newest first until an inclusive one
            bool done = false;
            for (int t = tile - 1; t >= 0 && !done; t -= OS_LB) {
                uint32_t v[OS_LB];
#pragma unroll
                for (int w = 0; w < OS_LB; ++w) v[w] = t - w >= 0 ? (uint32_t)st[(int64_t)(t - w) * 256 + d] : (uint32_t)OS_INC;
#pragma unroll
                for (int w = 0; w < OS_LB; ++w) {
                    if (done) break;
                    long long it = 0;
                    while ((v[w] & ~OS_MASK) == 0) {
                        if (++it > wait.spin) {
                            atomicOr(err, 1);
                            v[w] = OS_INC;
                            break;
                        }
                        __nanosleep(32);
                        v[w] = st[(int64_t)(t - w) * 256 + d];
                    }
                    excl += v[w] & OS_MASK;
                    if (v[w] & OS_INC) done = true;
                }
            }
            __threadfence();
            st[(int64_t)tile * 256 + d] = OS_INC | (excl + own);
        }
        gofs[d] = base[d] + excl;
        __syncthreads();
        int pre = 0;
        for (int w = 0; w < warp; ++w) pre += wsum[w];
        lstart[d] = pre + x - s;
    }
    __syncthreads();
    // keys to their tile-local sorted position, then coalesced runs to global
#pragma unroll
    for (int r = 0; r < OS_ITEMS; ++r) {
        if (rank[r] < 0) continue;
        const unsigned d = (key[r] >> shift) & 0xFF;
        const int lp = lstart[d] + cnt[warp][d] + rank[r];
        skey[lp] = key[r];
        sval[lp] = val[r];
    }
    __syncthreads();
    uint32_t dst[OS_ITEMS];
#pragma unroll
    for (int r = 0; r < OS_ITEMS; ++r) {
        const int i = r * OS_THREADS + threadIdx.x;
        key[r] = i < tcount ? skey[i] : 0u;
        val[r] = i < tcount ? sval[i] : 0u;
        const unsigned d = (key[r] >> shift) & 0xFF;
        dst[r] = gofs[d] + (uint32_t)(i - lstart[d]);
    }
    if (gpts) {
        // last pass with a gather: the sorted record {x, y, m, index}, all
        // gather loads issued before the stores
        float2 p[OS_ITEMS];
        float m[OS_ITEMS];
#pragma unroll
        for (int r = 0; r < OS_ITEMS; ++r) {
            const bool ok = r * OS_THREADS + (int)threadIdx.x < tcount;
            p[r] = ok ? gxy[val[r]] : make_float2(0.f, 0.f);
            m[r] = ok ? gmass[val[r]] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < OS_ITEMS; ++r) {
            if (r * OS_THREADS + (int)threadIdx.x >= tcount) continue;
            kout[dst[r]] = key[r];
            gpts[dst[r]] = make_float4(p[r].x, p[r].y, m[r], __int_as_float((int)val[r]));
        }
    } else {
#pragma unroll
        for (int r = 0; r < OS_ITEMS; ++r) {
            if (r * OS_THREADS + (int)threadIdx.x >= tcount) continue;
            kout[dst[r]] = key[r];
            vout[dst[r]] = val[r];
        }
    }
}

inline int64_t os_tiles(int64_t n) { return (n + OS_TILE - 1) / OS_TILE; }

}  // namespace

void scan_exclusive_i64(bgl_ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *d_total) {
    scan_exclusive<int64_t>(c, in, out, n, d_total);
}
void scan_exclusive_i32(bgl_ctx *c, const int32_t *in, int32_t *out, int64_t n, int32_t *d_total) {
    scan_exclusive<int32_t>(c, in, out, n, d_total);
}
void radix_sort_u64(bgl_ctx *c, uint64_t *keys, uint32_t *vals, int64_t n, int bits) {
    radix_sort<uint64_t>(c, keys, vals, n, bits);
}
void radix_sort_u32(bgl_ctx *c, uint32_t *keys, uint32_t *vals, int64_t n, int bits) {
    radix_sort<uint32_t>(c, keys, vals, n, bits);
}

void SortWorkspace::reserve(Allocator *a, int64_t n, cudaStream_t s) {
    if (n <= cap) return;
    keys.reset(a, n);
    vals.reset(a, n);
    keys2.reset(a, n);
    vals2.reset(a, n);
    // hist: 4 x 256 digit counts, 4 x 256 digit bases, 4 tickets, 1 counter, error word
    hist.reset(a, 8 * 256 + 8);
    BGL_CUDA(cudaMemsetAsync(hist.p, 0, hist.bytes(), s));
    tiles.reset(a, 4 * 256 * os_tiles(n));   // look-back status words, one block per pass
    cap = n;
}

OsHist radix_sort_u32_ws_begin(bgl_ctx *c, SortWorkspace &ws, int64_t n, bool clear) {
    BGL_REQUIRE(n <= ws.cap && n < (int64_t(1) << 30), "radix sort: workspace too small");
    cudaStream_t s = c->stream;
    const int64_t nt = os_tiles(n);
    OsHist h;
    h.hist = reinterpret_cast<uint32_t *>(ws.hist.p);
    h.base = h.hist + 4 * 256;
    unsigned *tickets = reinterpret_cast<unsigned *>(h.hist + 8 * 256);
    h.counter = tickets + 4;
    h.tickets = tickets;
    h.status = reinterpret_cast<uint32_t *>(ws.tiles.p);
    h.ntiles = nt;
    if (!clear) return h;
    // counts, pass tickets and look-back status words start at zero
    BGL_CUDA(cudaMemsetAsync(h.hist, 0, sizeof(uint32_t) * 4 * 256, s));
    BGL_CUDA(cudaMemsetAsync(tickets, 0, sizeof(unsigned) * 4, s));
    BGL_CUDA(cudaMemsetAsync(ws.tiles.p, 0, sizeof(uint32_t) * 4 * 256 * nt, s));
    return h;
}

void radix_sort_u32_ws_scatter(bgl_ctx *c, SortWorkspace &ws, uint32_t *keys, uint32_t *vals, int64_t n,
                               const float2 *gxy, const float *gmass, float4 *gpts, const int *d_skip, OsWait wait) {
    cudaStream_t s = c->stream;
    const int64_t nt = os_tiles(n);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws.hist.p);
    uint32_t *base = hist + 4 * 256;
    unsigned *tickets = reinterpret_cast<unsigned *>(hist + 8 * 256);
    int *err = wait.err ? wait.err : reinterpret_cast<int *>(tickets + 5);
    if (wait.spin <= 0) wait.spin = OS_SPIN;
    uint32_t *status = reinterpret_cast<uint32_t *>(ws.tiles.p);
    const OsBufs bf{keys, vals, ws.keys.p, ws.vals.p, ws.keys2.p, ws.vals2.p};
    for (int d = 0; d < 4; ++d) {
        const bool g = d == 3 && gpts;
        os_scatter_kernel<<<(unsigned)nt, OS_THREADS, 0, s>>>(bf, d, d_skip, n, base + 256 * d,
                                                              status + (int64_t)d * 256 * nt, tickets + d, err,
                                                              g ? gxy : nullptr, g ? gmass : nullptr,
                                                              g ? gpts : nullptr, wait);
        BGL_LAUNCH_CHECK();
    }
    // the sorted keys (and values unless gathered) are back in keys / vals
}

void radix_sort_u32_ws(bgl_ctx *c, SortWorkspace &ws, uint32_t *keys, uint32_t *vals, int64_t n, int bits,
                       const float2 *gxy, const float *gmass, float4 *gpts) {
    if (n <= 1 || bits <= 0) return;
    BGL_REQUIRE(bits == 32 && vals, "radix sort: the workspace sort takes 32-bit keys with values");
    const OsHist h = radix_sort_u32_ws_begin(c, ws, n);
    os_hist_kernel<<<(unsigned)os_tiles(n), OS_THREADS, 0, c->stream>>>(keys, n, h);
    BGL_LAUNCH_CHECK();
    radix_sort_u32_ws_scatter(c, ws, keys, vals, n, gxy, gmass, gpts);
}

int sort_workspace_error(bgl_ctx *c, SortWorkspace &ws) {
    int e = 0;
    int *err = reinterpret_cast<int *>(reinterpret_cast<unsigned *>(ws.hist.p + 8 * 256) + 5);
    BGL_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BGL_CUDA(cudaStreamSynchronize(c->stream));
    return e;
}

int bits_for(uint64_t v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

}  // namespace bgl
