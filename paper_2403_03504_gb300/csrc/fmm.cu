// Fast Multipole Method for the ForceAtlas2 repulsion (Section 3.2.1).
//
// Field of the repulsion: with z = x + i y and charges q_j = m_j,
//   E(z) = sum_j q_j / (z - z_j),    F_rep(i) = kr m_i conj(E(z_i)),
// the derivative of the 2-D Laplace potential sum_j q_j log(z - z_j).  The
// "two Taylor expansions" of Section 3.2.1 are taken as the complex Laurent
// (outgoing, multipole) and Taylor (incoming, local) expansions of that
// potential (Greengard and Rokhlin 1987), of order p, stored scaled by the
// box half-width r (a~_k = a_k / r^k, b~_l = b_l r^l) so that FP32 does not
// overflow and the translation operators do not depend on the level.
//
// One evaluation (all launches, no host synchronisation):
//   bbox      root square covering all points (FP32 min/max, FP64 geometry)
//   keys      16-bit quantised x, y interleaved into 32-bit Morton keys, with
//             the digit histograms of the sort in the same pass
//   sort      stable radix sort of (key, index), four onesweep passes over
//             tiles of 4,096 keys (the two low ones skipped when the last
//             tree was at most 8 levels deep); the last writes x, y, m in
//             key order
//   tree      adaptive quadtree: a box is split while it holds more than
//             leaf_size points (and is above level 16).  The leaf level of
//             point i is 1 + the deepest level at which some window of
//             leaf_size + 1 consecutive sorted points around i shares a key
//             prefix, so boxes are emitted in one pass, level by level, in
//             Morton order within a level, with their ends, parents and child
//             slots, and each box goes into a hash table keyed by (level,
//             Morton prefix) as it is emitted
//   lists     per box, by hash lookups of the 3x3 cells around it and its
//             parent: U (adjacent leaves, near field), V (children of the
//             parent's neighbours that are not adjacent: the "interacting
//             cells" of Section 3.2.1), W and X (the adaptive-tree lists of
//             Carrier, Greengard and Rokhlin that make every pair counted
//             exactly once)
//   up        P2M from the points for boxes of up to 512 points; M2M from
//             the 4 children for the larger ones, by the last child to finish
//   m2l       per box, independently: M2L over V + P2L over X (a partial
//             incoming expansion)
//   near      per leaf: the direct P2P sum over the points of U
//   far       per leaf: the incoming expansion composed from the partial
//             expansions of the leaf and all its ancestors (the L2L chain,
//             one shift per ancestor), L2P at the targets, M2P over W (a W
//             list longer than 16 entries: far_heavy, 16 warps per leaf)
//   combine   per point: the force from the near sum and the far field
// Near and far run concurrently (main and side stream); the combine pass
// joins them.
// Every sum has a fixed order, so results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cstdlib>

#include "fa2_update.cuh"
#include "fmm.cuh"
#include "p2p.cuh"
#include "sort_hist.cuh"

namespace bgl {

namespace {

constexpr int MAXLEV = 16;
constexpr int NLEV = MAXLEV + 1;
constexpr int TREE_TILE = 1024;
constexpr int TREE_THREADS = 256;
constexpr int BN = 49;                 // binomial table dimension (n <= 48)

// C(n, k) rounded to the nearest float (exact below 2^24), the value the
// table holds; with compile-time n and k (fully unrolled loops) it folds to
// an immediate operand
__host__ __device__ constexpr float binom_f(int n, int k) {
    unsigned long long v = 1;
    for (int j = 0; j < k; ++j) v = v * (unsigned long long)(n - j) / (unsigned long long)(j + 1);
    return (float)v;
}
constexpr int SRC_CAP = 2048;          // P2P sources staged per pass
constexpr int LEAF_THREADS = 128;
constexpr long long SPIN_LIMIT = 1ll << 24;
// per-evaluation work tickets, zeroed by the bounding-box kernel: [0, 8) the
// passes' own counters, [8, 24) the leaves in each near-field bucket
constexpr int NTICKETS = 24;
constexpr int NEAR_BUCKET_COUNTS = 8;
// Near-field tuning constants (compile-time): target lanes per warp,
// sources per stage, unroll of the source loop, whether the staging code is
// shared by the tile variants instead of inlined into each, whether the
// leaves are taken in buckets of equal tile shape (filled by the lists kernel),
// and how many pairs of a lane's targets are summed with packed FP32x2
// arithmetic (bitwise the same forces; the packed operations run on one of
// the SM's two FMA pipes, so the rest stay scalar to use the other).
#ifndef BGL_NEAR_LPS
#define BGL_NEAR_LPS 8
#endif
#ifndef BGL_NEAR_SRC
#define BGL_NEAR_SRC 128
#endif
#ifndef BGL_NEAR_UNROLL
#define BGL_NEAR_UNROLL 1
#endif
#ifndef BGL_NEAR_SHARED_STAGE
#define BGL_NEAR_SHARED_STAGE 0
#endif
#ifndef BGL_NEAR_BUCKETS
#define BGL_NEAR_BUCKETS 1
#endif
#ifndef BGL_NEAR_PACKED
#define BGL_NEAR_PACKED 1
#endif
constexpr int NEAR_SRC = BGL_NEAR_SRC;
constexpr int NEAR_WARPS = 1024 / NEAR_SRC;       // 32 KB of stage buffers per block
constexpr int NEAR_LPS = BGL_NEAR_LPS;            // target lanes
constexpr int NEAR_SPLIT = 32 / NEAR_LPS;         // source splits
constexpr int NEAR_RMAX = 64 / NEAR_LPS;          // targets per lane: 64 per tile
constexpr int NEAR_UNROLL = BGL_NEAR_UNROLL;

// tile shape class of a leaf of `points` points: targets per lane, 1..NEAR_RMAX
__host__ __device__ __forceinline__ int near_class(int points) {
    const int r = (points + NEAR_LPS - 1) / NEAR_LPS;
    return r < 1 ? 1 : (r > NEAR_RMAX ? NEAR_RMAX : r);
}


enum { ERR_SPIN = 1, ERR_LIST_OVERFLOW = 2, ERR_BOX_OVERFLOW = 4, ERR_BBOX = 8 };

// After a bounded wait of the sort gave up, the points are not sorted and the
// kernels that build on them return at once (the evaluation reports
// BGL_ETIMEOUT; its forces are not written).  The error word does not change
// while these kernels run (only the sort sets ERR_SPIN, earlier on the
// stream), so every thread of a launch takes the same branch.
__device__ __forceinline__ bool aborted(const int *err) { return (*err & ERR_SPIN) != 0; }

// Root square and the per-level box geometry in FP32 (GB300's FP64 rate is
// a small fraction of its FP32 rate, so nothing per point or per box uses it)
struct Root {
    double ox, oy, side;        // the square, as computed (FP64, once)
    float oxf, oyf, scale;      // origin and 65536 / side, for the keys
    float w[MAXLEV + 1];        // box side at each level
    float r[MAXLEV + 1];        // box half-width at each level
};

struct Tree {
    // sorted points
    const uint32_t *key;
    const float4 *pts;        // x, y, m, original local index (int bits)
    int n;
    // boxes
    int *bstart, *bend, *blevel, *bparent;
    uint32_t *bkey;
    int8_t *bleaf;
    int4 *bchild;
    int2 *bmeta;              // per box {x | y << 16 at its level, level | leaf << 8}: one load
    int *levoff;              // [NLEV + 1], levoff[NLEV] = number of boxes
    int *lofs;                // [5 * Bmax] per box: starts of U, V, W, X and the end, in lidx
    int *lidx;                // list entries (each box's lists in one chunk)
    int *pool;                // entries handed out so far (zero at the start of an evaluation)
    ulonglong2 *hkv;          // box hash table: {key tagged with the evaluation epoch, box index}
    int hmask;                // table size - 1 (a power of two)
    const unsigned *epoch;    // evaluation counter (1..2^24-1)
    int lcap;                 // capacity of lidx
    int Bmax;                 // capacity of the box arrays
    const Root *root;
    int *err;
    int *ncls;                // [NEAR_RMAX] leaves in each near-field bucket (zeroed per evaluation)
    int *cleaf;               // [NEAR_RMAX * Bmax] the leaves of each bucket
};

__device__ __forceinline__ uint32_t spread_bits(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__device__ __forceinline__ uint32_t compact_bits(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}

// number of leading 2-bit digits shared by two keys (16 if equal)
__device__ __forceinline__ int lcp_level(uint32_t a, uint32_t b) { return a == b ? MAXLEV : (__clz(a ^ b) >> 1); }

__device__ __forceinline__ uint32_t prefix_at(uint32_t key, int L) { return L == 0 ? 0u : key >> (32 - 2 * L); }

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

// bounded wait until *flag != 0; records ERR_SPIN and gives up after SPIN_LIMIT polls
__device__ __forceinline__ void wait_flag(const int *flag, int *err) {
    long long it = 0;
    while (ld_volatile(flag) == 0) {
        if (++it > SPIN_LIMIT) {
            atomicOr(err, ERR_SPIN);
            break;
        }
        __nanosleep(64);
    }
    __threadfence();
}

struct BoxGeo {
    float cx, cy, r;
};


// packed integer box coordinates (x | y << 16) at the box's level
__device__ __forceinline__ int mx_(int c) { return c & 0xFFFF; }
__device__ __forceinline__ int my_(int c) { return (int)((unsigned)c >> 16); }
__device__ __forceinline__ int pack_xy(uint32_t key) { return (int)(compact_bits(key) | (compact_bits(key >> 1) << 16)); }

// Box geometry is defined by the float origin and side: the centre of box
// (bx, by) at level L is origin + (2 bx + 1) r_L with r_L = side 2^-(L+1)
// (exact), evaluated with one rounding by a fused multiply-add.
__device__ __forceinline__ BoxGeo box_geo_xy(const Root *__restrict__ rt, int c, int L) {
    const float r = rt->r[L];
    BoxGeo g;
    g.cx = fmaf((float)(2 * mx_(c) + 1), r, rt->oxf);
    g.cy = fmaf((float)(2 * my_(c) + 1), r, rt->oyf);
    g.r = r;
    return g;
}

// closed squares of two distinct (non-nested) boxes (packed coordinates) touch or overlap
__device__ __forceinline__ bool adjacent_xy(int ca, int La, int cb, int Lb) {
    const int F = max(La, Lb);
    const int ax = mx_(ca) << (F - La), ay = my_(ca) << (F - La);
    const int bx = mx_(cb) << (F - Lb), by = my_(cb) << (F - Lb);
    const int aw = 1 << (F - La), bw = 1 << (F - Lb);
    return max(ax, bx) <= min(ax + aw, bx + bw) && max(ay, by) <= min(ay + aw, by + bw);
}


// ---------------------------------------------------------------- box hash table
//
// Keys: epoch (24 bits) << 40 | level << 35 | Morton prefix (32 bits).  A
// slot holding another epoch's key counts as empty, so the table is never
// cleared; linear probing.  A slot is {key, value} in 16 bytes, so a probe
// is one load; the value is written by the inserting thread and read only
// by later kernels.
__device__ __forceinline__ unsigned long long hash_key(unsigned epoch, int L, uint32_t prefix) {
    return ((unsigned long long)epoch << 40) | ((unsigned long long)L << 35) | (unsigned long long)prefix;
}

__device__ __forceinline__ unsigned hash_slot(unsigned long long k, int mask) {
    k ^= k >> 31;
    k *= 0x7fb5d329728ea185ull;
    k ^= k >> 27;
    return (unsigned)k & (unsigned)mask;
}

__device__ void hash_insert(ulonglong2 *hkv, int mask, unsigned epoch, int L, uint32_t prefix, int box, int *err) {
    const unsigned long long k = hash_key(epoch, L, prefix);
    unsigned s = hash_slot(k, mask);
    for (int probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = hkv[s].x;
        while ((cur >> 40) != epoch) {             // empty (stale): try to claim it
            const unsigned long long prev = atomicCAS(&hkv[s].x, cur, k);
            if (prev == cur) {
                hkv[s].y = (unsigned long long)(unsigned)box;
                return;
            }
            cur = prev;
        }
        s = (s + 1) & (unsigned)mask;
    }
    atomicOr(err, 4);                              // table full (cannot happen at twice the box capacity)
}

// box index of (L, prefix) in this evaluation, or -1
__device__ __forceinline__ int hash_find(const Tree &T, unsigned epoch, int L, uint32_t prefix) {
    const unsigned long long k = hash_key(epoch, L, prefix);
    unsigned s = hash_slot(k, T.hmask);
    for (int probe = 0; probe <= T.hmask; ++probe) {
        const ulonglong2 cur = __ldcg(&T.hkv[s]);
        if (cur.x == k) return (int)cur.y;
        if ((cur.x >> 40) != epoch) return -1;
        s = (s + 1) & (unsigned)T.hmask;
    }
    return -1;
}

// The box at level L covering cell (cx, cy) of level L, else the coarser
// leaf covering it, else -1 (empty cell or outside the root square).
__device__ int cover(const Tree &T, unsigned epoch, int L, int cx, int cy) {
    if (cx < 0 || cy < 0 || cx >= (1 << L) || cy >= (1 << L)) return -1;
    for (int l = L; l >= 0; --l) {
        const int d = L - l;
        const uint32_t pre = spread_bits((uint32_t)(cx >> d)) | (spread_bits((uint32_t)(cy >> d)) << 1);
        const int A = hash_find(T, epoch, l, pre);
        if (A < 0) continue;
        if (l == L) return A;
        return (T.bmeta[A].y & 256) ? A : -1;
    }
    return -1;
}

// ---------------------------------------------------------------- bbox, keys, gather

// This evaluation's work tickets, digit counts and sort pass tickets start
// at zero (block 0 of the kernel that opens the evaluation).
__device__ __forceinline__ void evaluation_clear(int *tickets, const OsHist &h) {
    if (blockIdx.x != 0) return;
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) h.hist[i] = 0u;
    if (threadIdx.x < NTICKETS) tickets[threadIdx.x] = 0;
    if (threadIdx.x < 4) h.tickets[threadIdx.x] = 0u;
}

// The bounding box from each thread's (min x, max x, min y, max y): block
// partials, and the last block to arrive makes the root square of the
// quadtree (reading 15), resets the arrival counter and advances the epoch.
// Every thread of the block calls it.
__device__ void bbox_reduce_root(float mnx, float mxx, float mny, float mxy, float4 *__restrict__ part,
                                 unsigned *counter, Root *root, int *err, unsigned *epoch) {
    __shared__ float4 wred[32];
    __shared__ bool last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wred[warp] = make_float4(mnx, mxx, mny, mxy);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 a = wred[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            float4 b = wred[w];
            a = make_float4(fminf(a.x, b.x), fmaxf(a.y, b.y), fminf(a.z, b.z), fmaxf(a.w, b.w));
        }
        part[blockIdx.x] = a;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float4 a = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        float4 c = __ldcg(&part[b]);
        a = make_float4(fminf(a.x, c.x), fmaxf(a.y, c.y), fminf(a.z, c.z), fmaxf(a.w, c.w));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.x = fminf(a.x, __shfl_xor_sync(0xffffffffu, a.x, o));
        a.y = fmaxf(a.y, __shfl_xor_sync(0xffffffffu, a.y, o));
        a.z = fminf(a.z, __shfl_xor_sync(0xffffffffu, a.z, o));
        a.w = fmaxf(a.w, __shfl_xor_sync(0xffffffffu, a.w, o));
    }
    __syncthreads();
    if (lane == 0) wred[warp] = a;
    __syncthreads();
    if (threadIdx.x != 0) return;
    a = wred[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        float4 c = wred[w];
        a = make_float4(fminf(a.x, c.x), fmaxf(a.y, c.y), fminf(a.z, c.z), fmaxf(a.w, c.w));
    }
    double w = fmax((double)a.y - (double)a.x, (double)a.w - (double)a.z);
    double side = w * (1.0 + 0x1.0p-20);
    if (!isfinite(side)) {
        atomicOr(err, ERR_BBOX);
        side = 1.0;
    }
    if (!(side > 0.0)) side = 1.0;     // all points coincide
    Root r;
    r.side = side;
    r.ox = 0.5 * ((double)a.x + (double)a.y) - 0.5 * side;
    r.oy = 0.5 * ((double)a.z + (double)a.w) - 0.5 * side;
    if (!isfinite(r.ox) || !isfinite(r.oy)) {
        atomicOr(err, ERR_BBOX);
        r.ox = r.oy = 0.0;
    }
    r.oxf = (float)r.ox;
    r.oyf = (float)r.oy;
    const float sidef = (float)(side * (1.0 + 0x1.0p-22));   // rounding up keeps every point inside
    r.scale = 65536.0f / sidef;
    for (int L = 0; L <= MAXLEV; ++L) {
        r.w[L] = ldexpf(sidef, -L);
        r.r[L] = ldexpf(sidef, -(L + 1));
    }
    *root = r;
    *counter = 0u;
    *epoch = (*epoch % 0xFFFFFEu) + 1u;   // 1 .. 2^24 - 2; 0 never tags a live key
}

__global__ void bbox_kernel(const float2 *__restrict__ xy, int n, float4 *__restrict__ part, unsigned *counter,
                            Root *root, int *err, unsigned *epoch, int *tickets, OsHist h) {
    evaluation_clear(tickets, h);
    float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
        float2 p[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) p[r] = i + r * stride < n ? xy[i + r * stride] : xy[i];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            mnx = fminf(mnx, p[r].x);
            mxx = fmaxf(mxx, p[r].x);
            mny = fminf(mny, p[r].y);
            mxy = fmaxf(mxy, p[r].y);
        }
    }
    bbox_reduce_root(mnx, mxx, mny, mxy, part, counter, root, err, epoch);
}

constexpr int KEY_ITEMS = OS_ITEMS;      // one key block per radix tile

__global__ void __launch_bounds__(256) keys_kernel(const float2 *__restrict__ xy, int n, const Root *__restrict__ root,
                                                   uint32_t *__restrict__ key, uint32_t *__restrict__ idx, OsHist h) {
    const float ox = root->oxf, oy = root->oyf, sc = root->scale;
    const int i0 = blockIdx.x * 256 * KEY_ITEMS + threadIdx.x;
    uint32_t k[KEY_ITEMS];
    unsigned valid = 0;
    float2 p[KEY_ITEMS];
#pragma unroll
    for (int r = 0; r < KEY_ITEMS; ++r) {
        const int i = i0 + r * 256;
        p[r] = i < n ? xy[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < KEY_ITEMS; ++r) {
        const int i = i0 + r * 256;
        const float fx = floorf((p[r].x - ox) * sc), fy = floorf((p[r].y - oy) * sc);
        const int qx = (int)fminf(fmaxf(fx, 0.f), 65535.f), qy = (int)fminf(fmaxf(fy, 0.f), 65535.f);
        k[r] = spread_bits((uint32_t)qx) | (spread_bits((uint32_t)qy) << 1);
        if (i < n) {
            key[i] = k[r];
            idx[i] = (uint32_t)i;
            valid |= 1u << r;
        }
    }
    static_assert(256 * KEY_ITEMS == OS_TILE, "a key block is one radix tile");
    os_clear_status(h, blockIdx.x);
    os_block_hist<KEY_ITEMS>(k, valid, h);
}


// ---------------------------------------------------------------- tree build

// per point: c(i) = shared levels with point i-1 (-1 for i = 0), lambda(i) =
// level of its leaf; per tile and level: number of boxes that start in the tile
__global__ void __launch_bounds__(TREE_THREADS) tree_count_kernel(const uint32_t *__restrict__ key, int n, int S,
                                                                 int8_t *__restrict__ cl, int8_t *__restrict__ lam,
                                                                 int *__restrict__ tcnt, int ntiles,
                                                                 const int *__restrict__ sortskip, int *gmax,
                                                                 const int *err) {
    if (aborted(err)) return;
    // keys sorted on their top 16 bits only (two radix passes skipped):
    // boxes stop at level 8
    const int cap = *sortskip == 2 ? 8 : MAXLEV;
    __shared__ uint32_t sk[TREE_TILE + 2 * 256];
    __shared__ int8_t g[TREE_TILE + 256];
    __shared__ int cnt[NLEV];
    const int t0 = blockIdx.x * TREE_TILE;
    const int lo = t0 - S;                           // smem index 0 <-> point lo
    const int span = TREE_TILE + 2 * S;
    for (int k = threadIdx.x; k < span; k += TREE_THREADS) {
        int i = lo + k;
        sk[k] = (i >= 0 && i < n) ? key[i] : 0u;
    }
    if (threadIdx.x < NLEV) cnt[threadIdx.x] = 0;
    __syncthreads();
    // g(j) = lcp(key[j], key[j + S]) for windows j in [t0 - S, t0 + TILE)
    const int ng = TREE_TILE + S;
    for (int k = threadIdx.x; k < ng; k += TREE_THREADS) {
        int j = lo + k;
        g[k] = (j >= 0 && j + S < n) ? (int8_t)lcp_level(sk[k], sk[k + S]) : (int8_t)-1;
    }
    __syncthreads();
    // maxima of g over runs of P entries, P the largest power of two <= S + 1
    // (doubling: after the pass with step h, g[k] = max g[k .. k + 2h - 1])
    int P = 1;
    while (2 * P <= S + 1) P *= 2;
    constexpr int GM = (TREE_TILE + 256 + TREE_THREADS - 1) / TREE_THREADS;
    for (int h = 1; h < P; h *= 2) {
        int8_t v[GM];
#pragma unroll
        for (int m = 0; m < GM; ++m) {
            const int k = threadIdx.x + m * TREE_THREADS;
            v[m] = k < ng ? (int8_t)max((int)g[k], k + h < ng ? (int)g[k + h] : -1) : (int8_t)-1;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < GM; ++m) {
            const int k = threadIdx.x + m * TREE_THREADS;
            if (k < ng) g[k] = v[m];
        }
        __syncthreads();
    }
    int local[NLEV];
#pragma unroll
    for (int L = 0; L < NLEV; ++L) local[L] = 0;
    int gm = -1;
    for (int r = 0; r < TREE_TILE / TREE_THREADS; ++r) {
        int i = t0 + r * TREE_THREADS + threadIdx.x;
        if (i >= n) break;
        int k = i - lo;
        int c = i == 0 ? -1 : lcp_level(sk[k - 1], sk[k]);
        // windows j in [i - S, i] (g is -1 where a window does not fit): two
        // runs of P cover them
        const int G = max((int)g[k - S], (int)g[k - P + 1]);
        gm = max(gm, G);
        int la = min(cap, G + 1);
        cl[i] = (int8_t)c;
        lam[i] = (int8_t)la;
#pragma unroll
        for (int L = 0; L < NLEV; ++L) local[L] += (c < L && L <= la) ? 1 : 0;
    }
#pragma unroll
    for (int L = 0; L < NLEV; ++L)
        if (local[L]) atomicAdd(&cnt[L], local[L]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if ((threadIdx.x & 31) == 0 && gm >= 0) atomicMax(gmax, gm);
    __syncthreads();
    if (threadIdx.x < NLEV) tcnt[threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of the (level, tile) counts (one block of SCAN_THREADS,
// counts staged in shared memory with coalesced loads, SCAN_ITEMS
// consecutive counts per thread); level offsets.
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;

// Also picks the radix passes of the next evaluation: when no window of
// leaf_size + 1 points shares 8 or more levels (the tree is at most 8 levels
// deep), the next sort orders the top 16 key bits only.
__global__ void __launch_bounds__(SCAN_THREADS) tree_scan_kernel(int *tcnt, int ntiles, int *levoff, int Bmax,
                                                                 int *err, const int *gmax, int *sortskip) {
    if (aborted(err)) return;
    __shared__ int sv[SCAN_THREADS * SCAN_ITEMS];
    __shared__ int wsum[32];
    __shared__ int carry_s;
    const int total = NLEV * ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < total; base += SCAN_THREADS * SCAN_ITEMS) {
        const int m = min(SCAN_THREADS * SCAN_ITEMS, total - base);
        for (int i = threadIdx.x; i < SCAN_THREADS * SCAN_ITEMS; i += SCAN_THREADS) sv[i] = i < m ? tcnt[base + i] : 0;
        __syncthreads();
        int v[SCAN_ITEMS];
        int s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            v[k] = sv[threadIdx.x * SCAN_ITEMS + k];
            s += v[k];
        }
        int x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int w = wsum[lane];
            int t = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t - w;
            if (lane == 31) carry_s = t;
        }
        __syncthreads();
        int e = carry + wsum[warp] + x - s;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            sv[threadIdx.x * SCAN_ITEMS + k] = e;
            e += v[k];
        }
        carry += carry_s;
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += SCAN_THREADS) tcnt[base + i] = sv[i];
        __syncthreads();
    }
    if (threadIdx.x <= NLEV) {
        const int L = threadIdx.x;
        levoff[L] = L < NLEV ? tcnt[L * ntiles] : carry;
    }
    if (threadIdx.x == 0 && carry > Bmax) atomicOr(err, ERR_BOX_OVERFLOW);
    if (threadIdx.x == 0) *sortskip = *gmax <= 7 ? 2 : 0;
}

// Boxes of the tile, level by level in point order.  Warp w owns the
// contiguous points [t0 + w * PW, t0 + (w + 1) * PW) in rounds of 32, so a
// box's rank in its level is the tile's level offset + the counts of the
// earlier warps (one barrier) + the earlier rounds and lanes of its warp
// (ballots).  With before_L(i) = boxes of level L that start before point
// i, at point i:
//   a box of level L starts (c(i) < L <= lambda(i)): index before_L(i);
//     its parent is the box of level L - 1 holding point i: index
//     before_{L-1}(i) if that one starts at i too, else before_{L-1}(i) - 1;
//   the box of level L holding point i - 1 ends (c(i) < L <= lambda(i-1)):
//     index before_L(i) - 1, end i; every box holding point n - 1 ends at n.
// Each new box also takes its child slot in the parent and its entry in
// the hash table.  Levels above the deepest leaf level met in the tile
// (of its points and of the point before it) hold no box start or end.
__global__ void __launch_bounds__(TREE_THREADS) tree_emit_kernel(Tree T, const int8_t *__restrict__ cl,
                                                                const int8_t *__restrict__ lam,
                                                                const int *__restrict__ tcnt, int ntiles, int Bmax) {
    if (aborted(T.err)) return;
    constexpr int NW = TREE_THREADS / 32;
    constexpr int R = TREE_TILE / TREE_THREADS;        // rounds per warp
    constexpr int PW = TREE_TILE / NW;                 // points per warp
    __shared__ int wcount[NLEV][NW];
    __shared__ int smax;
    __shared__ int stc[NLEV];          // the tile's offset at every level, loaded once
    if (threadIdx.x == 0) smax = 0;
    if (threadIdx.x < NLEV) stc[threadIdx.x] = tcnt[threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const unsigned epoch = *T.epoch;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t0 = blockIdx.x * TREE_TILE;
    const unsigned lt = (1u << lane) - 1u;
    int c[R], la[R], lp[R];
    uint32_t k[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t0 + warp * PW + r * 32 + lane;
        const bool ok = i < T.n;
        c[r] = ok ? cl[i] : 99;
        la[r] = ok ? lam[i] : -99;
        lp[r] = ok && i > 0 ? lam[i - 1] : -99;      // leaf level of point i - 1
        k[r] = ok ? T.key[i] : 0u;
    }
    {
        int m = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) m = max(m, max(la[r], lp[r]));
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) atomicMax(&smax, m);
    }
    __syncthreads();
    const int Lmax = min(smax, NLEV - 1);
    // levels at which a box starts or ends among the warp's points (a box of
    // level L starts at i for c(i) < L <= lambda(i), one holding point i - 1
    // ends there for c(i) < L <= lambda(i - 1), and every box holding the
    // last point ends at n); at the other levels the warp has nothing to do
    unsigned lm = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int lo = c[r] + 1, hi = max(la[r], lp[r]);
        if (lo <= hi && hi < NLEV) lm |= ((2u << hi) - 1u) & ~((1u << lo) - 1u);
        if (t0 + warp * PW + r * 32 + lane == T.n - 1 && la[r] >= 0) lm |= (2u << la[r]) - 1u;
    }
    lm = __reduce_or_sync(0xffffffffu, lm);
    // per-warp totals of every level
    for (int L = 0; L <= Lmax; ++L) {
        if (!((lm >> L) & 1u)) {
            if (lane == 0) wcount[L][warp] = 0;
            continue;
        }
        int tot = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) tot += __popc(__ballot_sync(0xffffffffu, c[r] < L && L <= la[r]));
        if (lane == 0) wcount[L][warp] = tot;
    }
    __syncthreads();
    int pb[R];            // before_{L-1}(i), then whether a box of level L - 1 starts at i
    bool pf[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        pb[r] = 0;
        pf[r] = false;
    }
    for (int L = 0; L <= Lmax; ++L) {
        int base = stc[L];
        for (int w = 0; w < warp; ++w) base += wcount[L][w];
        if (!((lm >> L) & 1u)) {
            // no start or end at this level: before_L(i) = base for every point
#pragma unroll
            for (int r = 0; r < R; ++r) {
                pb[r] = base;
                pf[r] = false;
            }
            continue;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = t0 + warp * PW + r * 32 + lane;
            const bool f = c[r] < L && L <= la[r];
            const unsigned bl = __ballot_sync(0xffffffffu, f);
            const int before = base + __popc(bl & lt);
            if (f && before < Bmax) {
                const int b = before;
                const uint32_t P = prefix_at(k[r], L);
                T.bstart[b] = i;
                T.blevel[b] = L;
                T.bkey[b] = P;
                T.bleaf[b] = (int8_t)(L == la[r]);
                T.bmeta[b] = make_int2(pack_xy(P), L | ((L == la[r]) ? 256 : 0));
                int par = -1;
                if (L >= 1) {
                    par = pf[r] ? pb[r] : pb[r] - 1;
                    if (par >= 0 && par < b) ((int *)&T.bchild[par])[P & 3u] = b;
                    else atomicOr(T.err, ERR_BOX_OVERFLOW);
                }
                T.bparent[b] = par;
                hash_insert(T.hkv, T.hmask, epoch, L, P, b, T.err);
            }
            // the box of level L holding point i - 1 ends at i
            if (i < T.n && c[r] < L && L <= lp[r] && before >= 1 && before - 1 < Bmax) T.bend[before - 1] = i;
            // every box holding the last point ends at n
            if (i == T.n - 1 && L <= la[r] && before + (f ? 0 : -1) >= 0 && before + (f ? 0 : -1) < Bmax)
                T.bend[before + (f ? 0 : -1)] = T.n;
            pb[r] = before;
            pf[r] = f;
            base += __popc(bl);
        }
    }
}


// ---------------------------------------------------------------- neighbour tables and lists

__device__ __forceinline__ int meta_level(int2 m) { return m.y & 255; }
__device__ __forceinline__ bool meta_leaf(int2 m) { return (m.y & 256) != 0; }

// Contribution of neighbour cell k (0..8, k = 4 is the box itself) to the
// interaction lists of box b.  Each builder counts when out is null and
// writes otherwise, in a fixed order.
//   U (b a leaf): b itself (k = 4); the leaf at b's level or coarser covering
//      cell k (once, if no earlier cell had it); or, for an internal box at
//      cell k, the leaves inside it that touch b;
//   W (b a leaf): the children met in that descent that do not touch b;
//   V (level >= 2): children of the parent's neighbour box at cell k (at the
//      parent's level) that do not touch b, with their offset class
//      (dx + 3) * 7 + (dy + 3);
//   X (level >= 2): the leaf at the parent's level or coarser covering the
//      parent's cell k, if it does not touch b (once).
__device__ void lists_uw(const Tree &T, int b, int2 mb, const int *nbb, int k, int *ou, int *ow, int &cu, int &cw) {
    cu = cw = 0;
    if (!meta_leaf(mb)) return;
    if (k == 4) {
        if (ou) ou[0] = b;
        cu = 1;
        return;
    }
    const int A = nbb[k];
    if (A < 0) return;
    for (int k2 = 0; k2 < k; ++k2)
        if (k2 != 4 && nbb[k2] == A) return;
    const int2 ma = T.bmeta[A];
    if (meta_leaf(ma)) {
        if (ou) ou[0] = A;
        cu = 1;
        return;
    }
    const int cb = mb.x;
    const int L = meta_level(mb);
    int stack[4 * MAXLEV + 4];
    int sp = 0;
    stack[sp++] = A;
    while (sp > 0) {
        const int D = stack[--sp];
        const int4 ch = T.bchild[D];
        const int cs[4] = {ch.x, ch.y, ch.z, ch.w};
        int2 mc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) mc[q] = cs[q] >= 0 ? T.bmeta[cs[q]] : make_int2(0, 0);
        for (int q = 3; q >= 0; --q) {
            const int C = cs[q];
            if (C < 0) continue;
            if (adjacent_xy(mc[q].x, meta_level(mc[q]), cb, L)) {
                if (meta_leaf(mc[q])) {
                    if (ou) ou[cu] = C;
                    ++cu;
                } else if (sp < 4 * MAXLEV + 4) {
                    stack[sp++] = C;
                } else {
                    atomicOr(T.err, ERR_LIST_OVERFLOW);
                }
            } else {
                if (ow) ow[cw] = C;
                ++cw;
            }
        }
    }
}

// (ov[q] for child q, -1 where it is absent or adjacent; cv = how many are set)
__device__ __forceinline__ void lists_v(const Tree &T, int2 mb, int A, int k, int (&ov)[4], int &cv) {
    cv = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) ov[q] = -1;
    const int L = meta_level(mb);
    if (L < 2 || k == 4) return;
    if (A < 0) return;
    const int2 ma = T.bmeta[A];
    if (meta_level(ma) != L - 1 || meta_leaf(ma)) return;
    const int bx = mx_(mb.x), by = my_(mb.x);
    const int4 ch = T.bchild[A];
    const int cs[4] = {ch.x, ch.y, ch.z, ch.w};
    int cc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) cc[q] = cs[q] >= 0 ? T.bmeta[cs[q]].x : 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int C = cs[q];
        if (C < 0) continue;
        const int dx = mx_(cc[q]) - bx, dy = my_(cc[q]) - by;
        if (abs(dx) <= 1 && abs(dy) <= 1) continue;
        ov[q] = (C << 6) | ((dx + 3) * 7 + (dy + 3));
        ++cv;
    }
}

// (dup: an earlier cell of the parent had the same box)
__device__ void lists_x(const Tree &T, int2 mb, int A, int k, bool dup, int *ox, int &cx) {
    cx = 0;
    const int L = meta_level(mb);
    if (L < 2 || k == 4) return;
    if (A < 0 || dup) return;
    const int2 ma = T.bmeta[A];
    if (!meta_leaf(ma)) return;
    if (adjacent_xy(ma.x, meta_level(ma), mb.x, L)) return;
    if (ox) ox[0] = A;
    cx = 1;
}

// Warp-wide breadth-first descent from the internal same-level neighbours
// of leaf (cb, L) (front[0 .. nf)): every child that touches the leaf is a
// U entry if it is a leaf and joins the next frontier otherwise; every child
// that does not touch it is a W entry.  The frontier is taken 32 boxes at a
// time, a lane per box; one warp scan of packed class counts orders the
// outputs (level by level, frontier order, child order).  Entries go to
// su[nu ..] and sw[nw ..] while they fit in LST_CAP; returns false if any
// list or frontier exceeded its staging capacity (the counts stay exact).
constexpr int LST_CAP = 256;
constexpr int FRONT_CAP = 128;

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ bool descend(const Tree &T, int cb, int L, int *front, int nf, int *su, int &nu, int *sw, int &nw,
                        int lane) {
    int *cur = front, *nxt = front + FRONT_CAP;
    bool ok = true;
    while (nf > 0) {
        int nn = 0;
        for (int base = 0; base < nf; base += 32) {
            const int i = base + lane;
            int cs[4] = {-1, -1, -1, -1};
            unsigned cls = 0;       // 2 bits per child: 0 none, 1 U, 2 W, 3 frontier
            if (i < nf) {
                const int4 ch = T.bchild[cur[i]];
                cs[0] = ch.x;
                cs[1] = ch.y;
                cs[2] = ch.z;
                cs[3] = ch.w;
                int2 mc[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) mc[q] = cs[q] >= 0 ? T.bmeta[cs[q]] : make_int2(0, 0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (cs[q] < 0) continue;
                    const unsigned c = adjacent_xy(mc[q].x, mc[q].y & 255, cb, L) ? (mc[q].y & 256 ? 1u : 3u) : 2u;
                    cls |= c << (2 * q);
                }
            }
            // counts packed 10 bits per class (at most 4 per lane, 128 per warp)
            int cnt = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned c = (cls >> (2 * q)) & 3u;
                cnt += c == 1u ? 1 : (c == 2u ? (1 << 10) : (c == 3u ? (1 << 20) : 0));
            }
            const int inc = warp_incl_scan(cnt);
            const int tot = __shfl_sync(0xffffffffu, inc, 31);
            int pu = nu + ((inc - cnt) & 1023), pw = nw + (((inc - cnt) >> 10) & 1023), pf = nn + ((inc - cnt) >> 20);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned c = (cls >> (2 * q)) & 3u;
                if (c == 1u) {
                    if (pu < LST_CAP) su[pu] = cs[q];
                    ++pu;
                } else if (c == 2u) {
                    if (pw < LST_CAP) sw[pw] = cs[q];
                    ++pw;
                } else if (c == 3u) {
                    if (pf < FRONT_CAP) nxt[pf] = cs[q];
                    ++pf;
                }
            }
            nu += tot & 1023;
            nw += (tot >> 10) & 1023;
            nn += tot >> 20;
        }
        __syncwarp();
        int *t = cur;
        cur = nxt;
        nxt = t;
        nf = nn;
        if (nf > FRONT_CAP) {
            ok = false;
            break;
        }
    }
    return ok && nu <= LST_CAP && nw <= LST_CAP;
}

// Neighbour cells and interaction lists, one warp per box (no waits).
// Lanes 0-8 look up the 3x3 cells around the box (k = (dy + 1) * 3 + dx + 1:
// the box at its level covering the cell, else the coarser leaf covering it,
// else -1), lanes 9-17 those around its parent.  Then lanes 9-17 form V and
// lanes 18-26 X for the parent's cells (in registers); for a leaf, lanes 0-8
// give the direct U entries (the box itself, coarser or same-level leaves)
// and the internal same-level neighbours, from which the warp descends to
// the finer U entries and the W entries (staged in shared memory).  One
// atomic reserves the box's chunk of lidx; the order inside every list is
// fixed.  A box whose lists overflow the staging falls back to a per-lane
// walk, run once to count and once to write.
constexpr int LIST_WARPS = 8;

__global__ void __launch_bounds__(LIST_WARPS * 32) nbr_lists_kernel(Tree T) {
    if (aborted(T.err)) return;
    __shared__ int s_u[LIST_WARPS][LST_CAP], s_w[LIST_WARPS][LST_CAP];
    __shared__ int s_front[LIST_WARPS][2 * FRONT_CAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int role = lane / 9, k = lane % 9;
    const unsigned lt = (1u << lane) - 1u;
    int *su = s_u[wib], *sw = s_w[wib], *front = s_front[wib];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int B = min(T.levoff[NLEV], T.Bmax);
    const unsigned epoch = *T.epoch;
    for (int b = gw; b < B; b += nwarps) {
        const int2 mb = T.bmeta[b];
        const int L = meta_level(mb);
        const bool leaf = meta_leaf(mb);
        const int bx = mx_(mb.x), by = my_(mb.x);
        const int p = b == 0 ? -1 : T.bparent[b];
        int mine = -1;
        if (lane < 9) {
            mine = lane == 4 ? b : cover(T, epoch, L, bx + lane % 3 - 1, by + lane / 3 - 1);
        } else if (lane < 18 && p >= 0) {
            const int j = lane - 9;
            mine = j == 4 ? p : cover(T, epoch, L - 1, (bx >> 1) + j % 3 - 1, (by >> 1) + j / 3 - 1);
        }
        // lane (role, k): the box of cell k around b (role 0) or around its parent (roles 1, 2)
        const int A = __shfl_sync(0xffffffffu, mine, role == 0 ? k : 9 + k);
        // a cell whose box an earlier cell of the same group already had (k = 4 excluded)
        const bool grp = role <= 2 && k != 4 && A >= 0;
        const unsigned long long tag =
            grp ? ((unsigned long long)role << 32) | (unsigned)A : (1ull << 40) + (unsigned)lane;
        const bool dup = (__match_any_sync(0xffffffffu, tag) & lt) != 0u;
        // V (lanes 9-17, up to 4 each) and X (lanes 18-26, up to 1 each) in registers
        int ve[4] = {-1, -1, -1, -1};
        int cv = 0, xe = -1;
        if (role == 1 && p >= 0) lists_v(T, mb, A, k, ve, cv);
        else if (role == 2 && p >= 0) {
            int cx = 0;
            lists_x(T, mb, A, k, dup, &xe, cx);
            if (!cx) xe = -1;
        }
        // direct U entries and the frontier (lanes 0-8 of a leaf)
        int du = -1, fr = -1;
        if (leaf && role == 0) {
            if (k == 4) du = b;
            else if (A >= 0 && !dup) {
                if (meta_leaf(T.bmeta[A])) du = A;
                else fr = A;
            }
        }
        const unsigned bu = __ballot_sync(0xffffffffu, du >= 0), bf = __ballot_sync(0xffffffffu, fr >= 0);
        if (du >= 0) su[__popc(bu & lt)] = du;
        if (fr >= 0) front[__popc(bf & lt)] = fr;
        int nu = __popc(bu), nw = 0;
        __syncwarp();
        const bool staged = bf == 0u || descend(T, mb.x, L, front, __popc(bf), su, nu, sw, nw, lane);
        int nbb[9];
        if (!staged) {
            // overflow: exact counts by the per-lane walk
#pragma unroll
            for (int j = 0; j < 9; ++j) nbb[j] = __shfl_sync(0xffffffffu, mine, j);
            int cu = 0, cw = 0;
            if (role == 0) lists_uw(T, b, mb, nbb, k, nullptr, nullptr, cu, cw);
            nu = __shfl_sync(0xffffffffu, warp_incl_scan(cu), 31);
            nw = __shfl_sync(0xffffffffu, warp_incl_scan(cw), 31);
        }
        const int iv = warp_incl_scan(cv);
        const int tv = __shfl_sync(0xffffffffu, iv, 31);
        const unsigned bx_ = __ballot_sync(0xffffffffu, xe >= 0);
        const int tx = __popc(bx_);
        const int total = nu + tv + nw + tx;
        int base = 0;
        if (lane == 0) {
            base = atomicAdd(T.pool, total);
            if (base + total > T.lcap) {
                atomicOr(T.err, ERR_LIST_OVERFLOW);
                base = -1;
            }
        }
        base = __shfl_sync(0xffffffffu, base, 0);
#if BGL_NEAR_BUCKETS
        if (lane == 0 && leaf) {
            const int cls = near_class(T.bend[b] - T.bstart[b]);
            const int pos = atomicAdd(T.ncls + cls - 1, 1);
            T.cleaf[(size_t)(cls - 1) * T.Bmax + pos] = b;
        }
#endif
        if (base < 0) {
            if (lane < 5) T.lofs[5 * b + lane] = 0;
            __syncwarp();
            continue;
        }
        if (lane == 0) {
            T.lofs[5 * b] = base;
            T.lofs[5 * b + 1] = base + nu;
            T.lofs[5 * b + 2] = base + nu + tv;
            T.lofs[5 * b + 3] = base + nu + tv + nw;
            T.lofs[5 * b + 4] = base + total;
        }
        int *out = T.lidx + base;
        {
            int c = nu + iv - cv;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (ve[q] >= 0) out[c++] = ve[q];
        }
        if (xe >= 0) out[nu + tv + nw + __popc(bx_ & lt)] = xe;
        if (staged) {
            for (int i = lane; i < nu; i += 32) out[i] = su[i];
            for (int i = lane; i < nw; i += 32) out[nu + tv + i] = sw[i];
        } else {
            int cu = 0, cw = 0;
            if (role == 0) lists_uw(T, b, mb, nbb, k, nullptr, nullptr, cu, cw);
            const int iu = warp_incl_scan(cu), iw = warp_incl_scan(cw);
            int d0, d1;
            if (role == 0) lists_uw(T, b, mb, nbb, k, out + (iu - cu), out + nu + tv + (iw - cw), d0, d1);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- expansions

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 crcp(float2 a) {
    float d = 1.0f / (a.x * a.x + a.y * a.y);
    return make_float2(a.x * d, -a.y * d);
}
// 1 / a with the MUFU reciprocal (about one rounding of error more than crcp)
__device__ __forceinline__ float2 crcp_fast(float2 a) {
    const float d = rcp_approx(fmaf(a.x, a.x, a.y * a.y));
    return make_float2(a.x * d, -a.y * d);
}

// Warp sum of the 2 (PT + 1) floats of a (real and imaginary parts
// interleaved, float f = part f & 1 of coefficient f / 2), scattered: on
// return out[c] of lane L holds the total of float 32 c + L.  Recursive
// halving: at each step a lane keeps one half of its values, sends the
// other half to its partner and adds what it receives, so a chunk of 32
// floats takes 16 + 8 + 4 + 2 + 1 = 31 shuffles (a butterfly on every
// float takes 5 per float).  The order of the additions is fixed.
template <int PT>
__host__ __device__ constexpr int scatter_chunks() { return (2 * (PT + 1) + 31) / 32; }

template <int PT>
__device__ __forceinline__ void warp_sum_scatter(const float2 (&a)[PT + 1], int lane, float (&out)[scatter_chunks<PT>()]) {
    constexpr int NF = 2 * (PT + 1);
#pragma unroll
    for (int c = 0; c < scatter_chunks<PT>(); ++c) {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int f = 32 * c + i;
            v[i] = f < NF ? ((f & 1) ? a[f >> 1].y : a[f >> 1].x) : 0.f;
        }
#pragma unroll
        for (int h = 16; h > 0; h >>= 1) {
            const bool up = (lane & h) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float send = up ? v[i] : v[i + h];
                const float keep = up ? v[i + h] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
            }
        }
        out[c] = v[0];
    }
}


struct ExpArgs {
    Tree T;
    float2 *M;            // multipole  [(PT + 1) * Bmax]
    float2 *Lc;           // local      [(PT + 1) * Bmax]
    int *arrive;          // [Bmax], zero between evaluations (reset by the last arriver)
    int *done;            // [Bmax]
    int *ticket;
    const float *binom;   // [BN * BN]
    int p;
    const float *vout;    // BF16 M2L: the translated expansion of every V entry (null: M2L in FP32 here)
    const int *vbase;     //   row of box b's first V entry in vout
};

// ---------------------------------------------------------------- M2L on tensor cores (BF16)
//
// A V entry of offset class c translates the source's scaled outgoing
// expansion by a fixed matrix T_c (scaled coefficients make it the same at
// every level): in real form, rows (l, re/im) for l = 0..p, columns (k,
// re/im), blocks [[t_r, -t_i], [t_i, t_r]] of
//   t(l, 0) = -w^-l / l,  t(l, k) = (-1)^k C(l+k-1, k-1) w^-(l+k),  l >= 1,
// w = 2 (dx + i dy); row l = 0 is zero (b~_0 is not used).  With p <= 15 the
// matrix fits 32 x 32.  The entries are bucketed by class; a warp takes 8
// entries of one class at a time: B = their source vectors, each divided by
// its largest component (per-box scaling) and rounded to BF16; A = T_c in
// BF16 (precomputed as mma fragments); mma.m16n8k16 with FP32 accumulate,
// 2 row tiles x 2 depth tiles; the results, multiplied back by the scales,
// go to row vbase[b] + j of vout for the j-th V entry of box b.  The M2L +
// P2L kernel then sums a box's rows in list order, so the result does not
// depend on the bucketing order.
constexpr int VCLS = 49;              // offset classes (dx, dy) in [-3, 3]^2, 40 of them used
constexpr int VROWS = 32;             // rows of a translated expansion in vout

// rows of vout for every box's V entries (the order of boxes in vout is
// immaterial: each box reads back its own rows)
__global__ void vbase_kernel(Tree T, int *vtot, int cap, int *vbase) {
    if (aborted(T.err)) return;
    const int B = min(T.levoff[NLEV], T.Bmax);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const int nv = T.lofs[5 * b + 2] - T.lofs[5 * b + 1];
        int base = 0;
        if (nv > 0) {
            base = atomicAdd(vtot, nv);
            if (base + nv > cap) {
                atomicOr(T.err, ERR_LIST_OVERFLOW);
                base = 0;
            }
        }
        vbase[b] = base;
    }
}

__global__ void vclass_count_kernel(Tree T, int *count) {
    if (aborted(T.err)) return;
    __shared__ int sc[VCLS];
    for (int i = threadIdx.x; i < VCLS; i += blockDim.x) sc[i] = 0;
    __syncthreads();
    const int B = min(T.levoff[NLEV], T.Bmax);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
        for (int e = T.lofs[5 * b + 1]; e < T.lofs[5 * b + 2]; ++e) atomicAdd(&sc[T.lidx[e] & 63], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < VCLS; i += blockDim.x)
        if (sc[i]) atomicAdd(&count[i], sc[i]);
}

// bucket starts (exclusive scan of the 49 counts, rounded up to tiles of 8);
// the padding slots of every bucket hold {-1, -1}
__global__ void vclass_scan_kernel(const int *count, int *start, int *cursor, int cap, int2 *pairs, int *err) {
    if (aborted(err)) return;
    if (threadIdx.x != 0) return;
    int acc = 0;
    for (int c = 0; c < VCLS; ++c) {
        start[c] = acc;
        cursor[c] = acc;
        const int padded = (count[c] + 7) & ~7;
        for (int j = acc + count[c]; j < acc + padded && j < cap; ++j) pairs[j] = make_int2(-1, -1);
        acc += padded;
    }
    start[VCLS] = acc;
    if (acc > cap) atomicOr(err, ERR_LIST_OVERFLOW);
}

// pairs[pos] = {V entry index in lidx, its row in vout}; slots are claimed
// per block (shared counters, one global atomic per class and round)
__global__ void vclass_scatter_kernel(Tree T, int *cursor, const int *vbase, int cap, int2 *pairs) {
    if (aborted(T.err)) return;
    __shared__ int sc[VCLS], sb[VCLS];
    const int B = min(T.levoff[NLEV], T.Bmax);
    for (int r0 = blockIdx.x * blockDim.x; r0 < B; r0 += gridDim.x * blockDim.x) {
        for (int i = threadIdx.x; i < VCLS; i += blockDim.x) sc[i] = 0;
        __syncthreads();
        const int b = r0 + threadIdx.x;
        const int vs = b < B ? T.lofs[5 * b + 1] : 0, ve = b < B ? T.lofs[5 * b + 2] : 0;
        for (int e = vs; e < ve; ++e) atomicAdd(&sc[T.lidx[e] & 63], 1);
        __syncthreads();
        for (int i = threadIdx.x; i < VCLS; i += blockDim.x) {
            sb[i] = sc[i] ? atomicAdd(&cursor[i], sc[i]) : 0;
            sc[i] = 0;
        }
        __syncthreads();
        for (int e = vs; e < ve; ++e) {
            const int c = T.lidx[e] & 63;
            const int pos = sb[c] + atomicAdd(&sc[c], 1);
            if (pos < cap) pairs[pos] = make_int2(e, vbase[b] + (e - vs));
        }
        __syncthreads();
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// one warp per tile of 8 entries of one class
__global__ void __launch_bounds__(256) m2l_bf16_kernel(Tree T, const float2 *__restrict__ M, int PT1, int p,
                                                       const int *__restrict__ start, const int2 *__restrict__ pairs,
                                                       const uint4 *__restrict__ tfrag, int cap, float *vout) {
    if (aborted(T.err)) return;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    // buckets past the capacity were not filled (the overflow is flagged): translate nothing
    const int total = start[VCLS] <= cap ? start[VCLS] : 0;
    const int gid = lane >> 2, tig = lane & 3;
    for (int t0 = gw * 8; t0 < total; t0 += nw * 8) {
        // class of this tile (tiles never straddle buckets)
        int c = 0;
        while (c + 1 < VCLS && start[c + 1] <= t0) ++c;
        const int2 pr = pairs[t0 + gid];            // entry of column gid (-1: padding)
        const bool live = pr.x >= 0 && pr.x < T.lcap && pr.y >= 0 && pr.y < cap;
        const int e = live ? pr.y : -1;              // its row in vout
        const int D = live ? (T.lidx[pr.x] >> 6) : -1;
        // B fragments: rows k = kt * 16 + tig * 2 (+1, +8, +9) of column gid
        float v[2][4];
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            const int k0 = kt * 8 + tig, k1 = k0 + 4;       // coefficient indices
            const float2 a0 = (D >= 0 && k0 <= p) ? M[(size_t)D * PT1 + k0] : make_float2(0.f, 0.f);
            const float2 a1 = (D >= 0 && k1 <= p) ? M[(size_t)D * PT1 + k1] : make_float2(0.f, 0.f);
            v[kt][0] = a0.x;
            v[kt][1] = a0.y;
            v[kt][2] = a1.x;
            v[kt][3] = a1.y;
        }
        // per-column scale: the largest component (the 4 lanes of a column)
        float mx = 0.f;
#pragma unroll
        for (int kt = 0; kt < 2; ++kt)
#pragma unroll
            for (int j = 0; j < 4; ++j) mx = fmaxf(mx, fabsf(v[kt][j]));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        const float inv = mx > 0.f ? 1.0f / mx : 0.f;
        uint32_t b[2][2];
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            b[kt][0] = pack_bf16x2(v[kt][0] * inv, v[kt][1] * inv);
            b[kt][1] = pack_bf16x2(v[kt][2] * inv, v[kt][3] * inv);
        }
        float acc[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[mt][j] = 0.f;
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                const uint4 af = tfrag[((size_t)(c * 2 + mt) * 2 + kt) * 32 + lane];
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                    "{%8, %9}, {%0, %1, %2, %3};\n"
                    : "+f"(acc[mt][0]), "+f"(acc[mt][1]), "+f"(acc[mt][2]), "+f"(acc[mt][3])
                    : "r"(af.x), "r"(af.y), "r"(af.z), "r"(af.w), "r"(b[kt][0]), "r"(b[kt][1]));
            }
        }
        // C: rows mt * 16 + gid (+8), columns tig * 2, tig * 2 + 1; scale back per column
        int ec[2];
        float sc[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            ec[j] = __shfl_sync(0xffffffffu, e, (tig * 2 + j) * 4);
            sc[j] = __shfl_sync(0xffffffffu, mx, (tig * 2 + j) * 4);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (ec[j] < 0) continue;
            float *o = vout + (size_t)ec[j] * VROWS;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                o[mt * 16 + gid] = acc[mt][j] * sc[j];
                o[mt * 16 + gid + 8] = acc[mt][2 + j] * sc[j];
            }
        }
    }
}

// Outgoing expansions of the boxes of level >= 2 (the only ones any list
// uses).  A box of at most P2M_MAX points gets its expansion directly from
// its points (P2M, one warp, fixed-order warp sum).  The few larger boxes near
// the root get theirs by M2M from their four children, computed by the last
// child to finish (an arrival count per box), so no warp waits.
constexpr int P2M_MAX = 512;

template <int PT>
__global__ void __launch_bounds__(256) up_kernel(ExpArgs a) {
    if (aborted(a.T.err)) return;
    __shared__ float sbin[BN * BN];
    __shared__ float2 stage[8][4][PT + 1];
    for (int i = threadIdx.x; i < BN * BN; i += blockDim.x) sbin[i] = a.binom[i];
    __syncthreads();
    const Tree &T = a.T;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int B = min(T.levoff[NLEV], T.Bmax);
    const int b0 = min(T.levoff[2], B);
    const Root *rt = T.root;
    const int p = a.p;
    for (int b = b0 + gw; b < B; b += nw) {
        const int s = T.bstart[b], e = T.bend[b];
        const int2 mb = T.bmeta[b];
        if (e - s > P2M_MAX && !meta_leaf(mb)) continue;   // filled by M2M below
        // whether the parent is filled by M2M (loaded ahead of the P2M sum)
        const int pb0 = T.bparent[b];
        const bool up0 = pb0 >= 0 && (T.bmeta[pb0].y & 255) >= 2 && T.bend[pb0] - T.bstart[pb0] > P2M_MAX;
        const BoxGeo g = box_geo_xy(rt, mb.x, mb.y & 255);
        const float ir = 1.0f / g.r;
        float2 acc[PT + 1];
#pragma unroll
        for (int k = 0; k <= PT; ++k) acc[k] = make_float2(0.f, 0.f);
        for (int j = s + lane; j < e; j += 32) {
            const float4 q = T.pts[j];
            const float2 w = make_float2((q.x - g.cx) * ir, (q.y - g.cy) * ir);
            float2 pw = w;
            acc[0].x += q.z;
#pragma unroll
            for (int k = 1; k <= PT; ++k) {
                acc[k].x = fmaf(q.z, pw.x, acc[k].x);
                acc[k].y = fmaf(q.z, pw.y, acc[k].y);
                pw = cmul(pw, w);
            }
        }
        float tot[scatter_chunks<PT>()];
        warp_sum_scatter<PT>(acc, lane, tot);
        // a~_0 = sum q, a~_k = -sum q w^k / k
#pragma unroll
        for (int c = 0; c < scatter_chunks<PT>(); ++c) {
            const int f = 32 * c + lane, k = f >> 1;
            if (k <= p) reinterpret_cast<float *>(a.M)[(size_t)b * (PT + 1) * 2 + f] =
                k > 0 ? tot[c] * (-1.0f / (float)k) : tot[c];
        }
        // only a box whose parent is filled by M2M publishes its expansion (a
        // fence, then the parent's arrival count)
        int child = b;
        for (bool up = up0;;) {
            if (!up) break;
            const int pb = T.bparent[child];
            __threadfence();        // every lane's expansion writes, before lane 0's count
            __syncwarp();
            int last = 0;
            const int4 ch = T.bchild[pb];
            const int cs[4] = {ch.x, ch.y, ch.z, ch.w};
            if (lane == 0) {
                const int nch = (ch.x >= 0) + (ch.y >= 0) + (ch.z >= 0) + (ch.w >= 0);
                const int old = atomicAdd(&a.arrive[pb], 1);
                last = old == nch - 1;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (!last) break;
            __threadfence();
            if (lane == 0) a.arrive[pb] = 0;
            // stage the children's coefficients (one coalesced load per lane and child)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (cs[q] >= 0 && lane <= p) stage[wib][q][lane] = __ldcg(&a.M[(size_t)cs[q] * (PT + 1) + lane]);
            __syncwarp();
            // M2M: b~_l = -a~_0 u^l / l + sum_{k=1}^{l} a~_k 2^-k u^(l-k) C(l-1, k-1)
            float2 out = make_float2(0.f, 0.f);
            if (lane <= p) {
                const int l = lane;
                for (int q = 0; q < 4; ++q) {
                    if (cs[q] < 0) continue;
                    const float2 u = make_float2((q & 1) ? 0.5f : -0.5f, (q & 2) ? 0.5f : -0.5f);
                    const float2 a0 = stage[wib][q][0];
                    if (l == 0) {
                        out = cadd(out, a0);
                        continue;
                    }
                    float2 pw = make_float2(1.f, 0.f);
                    float2 sum = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = PT; k >= 1; --k) {
                        if (k <= l) {
                            const float cb = sbin[(l - 1) * BN + (k - 1)] * ldexpf(1.0f, -k);
                            sum = cadd(sum, cscale(cmul(stage[wib][q][k], pw), cb));
                            pw = cmul(pw, u);
                        }
                    }
                    sum = cadd(sum, cscale(cmul(a0, pw), -1.0f / (float)l));   // pw = u^l
                    out = cadd(out, sum);
                }
                a.M[(size_t)pb * (PT + 1) + l] = out;
            }
            __syncwarp();
            child = pb;
            const int gp = T.bparent[child];
            up = gp >= 0 && (T.bmeta[gp].y & 255) >= 2 && T.bend[gp] - T.bstart[gp] > P2M_MAX;
        }
    }
}

// Incoming expansion of every box of level >= 2 from its own interaction
// lists only (no parent term): M2L over V and P2L over X, one warp per box,
// lanes over the V entries and over the points of X leaves, a
// fixed-order warp sum to combine.  Boxes are independent, so the pass has no waits;
// the parents' contributions are folded in at the leaves (far_kernel).
// (at PT = 8 the kernel fits 64 registers and at PT = 12 128: four and two
// blocks per SM hide more of the latency of the list and expansion loads)
template <int PT, bool TC>
__global__ void __launch_bounds__(256, PT == 8 ? 4 : (PT == 12 ? 2 : 1)) m2l_kernel(ExpArgs a) {
    if (aborted(a.T.err)) return;
    const Tree &T = a.T;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int B = min(T.levoff[NLEV], T.Bmax);
    const int b0 = min(T.levoff[2], B);            // boxes of levels 0 and 1 have empty lists
    const Root *rt = T.root;
    const int p = a.p;
    for (int b = b0 + gw; b < B; b += nw) {
        float2 acc[PT + 1];
#pragma unroll
        for (int k = 0; k <= PT; ++k) acc[k] = make_float2(0.f, 0.f);
        // M2L: b~_l += w^-l ( -a~_0 / l + sum_k (-1)^k a~_k w^-k C(l+k-1, k-1) ), w = 2 (dx + i dy)
        const int vs = T.lofs[5 * b + 1], ve = T.lofs[5 * b + 2];
        if constexpr (TC) {
            // translated on the tensor cores: lane l sums coefficient l over the entries in order
            if (lane >= 1 && lane <= p)
                for (int e = vs; e < ve; ++e) {
                    const float *o = a.vout + (size_t)(a.vbase[b] + (e - vs)) * VROWS + 2 * lane;
                    acc[0].x += o[0];
                    acc[0].y += o[1];
                }
        }
        for (int e = vs + lane; !TC && e < ve; e += 32) {
            const int ent = T.lidx[e];
            const int D = ent >> 6, cls = ent & 63;
            const float2 w = make_float2(2.0f * (float)(cls / 7 - 3), 2.0f * (float)(cls % 7 - 3));
            const float2 iw = crcp_fast(w);
            const float2 *md = a.M + (size_t)D * (PT + 1);
            const float2 a0 = md[0];
            float2 ap[PT + 1];
            float2 pw = iw;
#pragma unroll
            for (int k = 1; k <= PT; ++k) {
                float2 v = k <= p ? md[k] : make_float2(0.f, 0.f);
                v = cmul(v, pw);
                ap[k] = (k & 1) ? make_float2(-v.x, -v.y) : v;
                pw = cmul(pw, iw);
            }
            float2 pl = iw;
#pragma unroll
            for (int l = 1; l <= PT; ++l) {
                const float nil = -1.0f / (float)l;          // l is a compile-time constant here
                float2 s = make_float2(a0.x * nil, a0.y * nil);
#pragma unroll
                for (int k = 1; k <= PT; ++k) {
                    const float cb = binom_f(l + k - 1, k - 1);
                    s.x = fmaf(cb, ap[k].x, s.x);
                    s.y = fmaf(cb, ap[k].y, s.y);
                }
                acc[l] = cadd(acc[l], cmul(s, pl));
                pl = cmul(pl, iw);
            }
        }
        // P2L: b~_l += -q t^l / l, t = r / (z_j - c)
        const int2 mb = T.bmeta[b];
        const BoxGeo g = box_geo_xy(rt, mb.x, mb.y & 255);
        const int xs = T.lofs[5 * b + 3], xe = T.lofs[5 * b + 4];
        for (int e = xs; e < xe; ++e) {
            const int C = T.lidx[e];
            for (int j = T.bstart[C] + lane; j < T.bend[C]; j += 32) {
                const float4 s = T.pts[j];
                const float2 t = cscale(crcp_fast(make_float2(s.x - g.cx, s.y - g.cy)), g.r);
                float2 pw = t;
#pragma unroll
                for (int l = 1; l <= PT; ++l) {
                    const float c = s.z * (-1.0f / (float)l);
                    acc[l].x = fmaf(c, pw.x, acc[l].x);
                    acc[l].y = fmaf(c, pw.y, acc[l].y);
                    pw = cmul(pw, t);
                }
            }
        }
        float2 tc = make_float2(0.f, 0.f);
        if constexpr (TC) {
            // acc[0] of lane l holds its coefficient's tensor-core sum
            tc = acc[0];
            acc[0] = make_float2(0.f, 0.f);
        }
        float tot[scatter_chunks<PT>()];
        warp_sum_scatter<PT>(acc, lane, tot);
#pragma unroll
        for (int c = 0; c < scatter_chunks<PT>(); ++c) {
            const int f = 32 * c + lane, k = f >> 1;
            float v = tot[c];
            if constexpr (TC) {
                const float tx = __shfl_sync(0xffffffffu, tc.x, k & 31), ty = __shfl_sync(0xffffffffu, tc.y, k & 31);
                v += (f & 1) ? ty : tx;
            }
            if (k <= p) reinterpret_cast<float *>(a.Lc)[(size_t)b * (PT + 1) * 2 + f] = k == 0 ? 0.f : v;
        }
    }
}


struct LeafArgs {
    ExpArgs e;
    float2 *f;           // f[q - fbase]: near-field sums, then the final forces
    const float2 *fa;    // fa[q - fbase] added to the final force, or null
    float2 *ef;          // far field E(z) of every point, by component-local index
    const float *mass;   // mass[o], component-local index
    int64_t q0, fbase;
    float kr;
    int *ticket;
    int *heavy, *nheavy;  // leaves whose W list the far_heavy kernel takes, and their count
    int heavy_cap;
    // fused swing/traction (null fprev: not fused)
    const float2 *fprev;  // fprev[q - fbase]
    int variant;
    double tau;
    double *sg, *stats;
    int *iter;
    double2 *spart;       // per combine block
    unsigned *scount;     // arrival count of the combine blocks
};

// Near field: the direct sum over the points of U for every target of a
// leaf.  One warp per leaf, the leaves taken through a ticket counter bucket
// by bucket (the lists kernel files every leaf under its tile shape, the
// most targets per lane first), so that the warps of an SM run one or two of
// the unrolled tile variants at a time and the instruction cache holds them
// (taken in box order instead, with all variants interleaved on every SM,
// the same kernel ran 12 % slower).  The
// sources are staged NEAR_SRC at a time in the warp's own shared memory
// with asynchronous 16-byte copies (cp.async), double-buffered: the copies
// of the next chunk are in flight while the current chunk is summed; each
// chunk is padded to a multiple of NEAR_SPLIT with zero-mass sources, which
// add exactly 0.  The warp's lanes form NEAR_LPS target lanes times
// NEAR_SPLIT source splits: lane (t, h) owns the R = ceil(targets / 8)
// targets t, t + 8, ... of the leaf (at most 7 padded target slots) and
// every NEAR_SPLIT-th staged source from h, so each shared-memory load of a
// source serves R pairs; the splits combine by a fixed butterfly.  Writes
// the raw sum sum_j m_j (p_i - p_j) / |p_i - p_j|^2 to f (the combine pass
// completes it).  Measured on the 554k-node giant component's final layout:
// four target lanes (up to sixteen targets each, fewer padded slots) ran 8 %
// slower, as did unrolling the source loop (the code of the variants
// outgrows the instruction cache).

static_assert(NEAR_LPS * NEAR_RMAX == 64, "a near tile covers a full leaf of 64 points");
static_assert(NEAR_WARPS >= 1 && NEAR_WARPS * NEAR_SRC * 2 * 16 == 32768, "stage buffers");
static_assert(NEAR_SRC % NEAR_SPLIT == 0, "chunks split evenly");

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Issue the copies of the next chunk (up to NEAR_SRC sources of the U list
// from entry *ui, offset *off) into buf and zero-mass padding up to a
// multiple of NEAR_SPLIT; returns the padded chunk size.
#if BGL_NEAR_SHARED_STAGE
__device__ __noinline__
#else
__device__ __forceinline__
#endif
int stage_chunk(const Tree &T, float4 *buf, int &ui, int &off, int ue, int lane) {
    int cnt = 0;
    while (ui < ue && cnt < NEAR_SRC) {
        const int C = T.lidx[ui];
        const int cs = T.bstart[C], ce = T.bend[C];
        const int take = min(ce - cs - off, NEAR_SRC - cnt);
        for (int k = lane; k < take; k += 32) cp_async16(buf + cnt + k, T.pts + cs + off + k);
        cnt += take;
        off += take;
        if (off == ce - cs) {
            ++ui;
            off = 0;
        }
    }
    cp_async_commit();
    const int padded = (cnt + NEAR_SPLIT - 1) & ~(NEAR_SPLIT - 1);
    if (lane < padded - cnt) buf[cnt + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    return padded;
}

// Pairs of the targets tb + t + 8 r (r < R) of lane (t, h) with the staged
// sources h, h + NEAR_SPLIT, ...
template <int R>
__device__ __forceinline__ void near_tile(const Tree &T, LeafArgs &la, float4 (*buf)[NEAR_SRC], int tb, int ntc,
                                          int us, int ue, int lane) {
    const int t = lane % NEAR_LPS, h = lane / NEAR_LPS;
    float zx[R], zy[R], fx[R], fy[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t + r * NEAR_LPS;
        const float4 z = i < ntc ? T.pts[tb + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        zx[r] = z.x;
        zy[r] = z.y;
        fx[r] = fy[r] = 0.f;
    }
#if BGL_NEAR_PACKED
    // targets 2k, 2k + 1 (k < R2) negated and packed, with their negated
    // sums; targets from 2 R2 on stay scalar
    constexpr int R2 = R / 2 < BGL_NEAR_PACKED ? R / 2 : BGL_NEAR_PACKED;
    float2 nzx[R2 > 0 ? R2 : 1], nzy[R2 > 0 ? R2 : 1], gx[R2 > 0 ? R2 : 1], gy[R2 > 0 ? R2 : 1];
#pragma unroll
    for (int k = 0; k < R2; ++k) {
        nzx[k] = make_float2(-zx[2 * k], -zx[2 * k + 1]);
        nzy[k] = make_float2(-zy[2 * k], -zy[2 * k + 1]);
        gx[k] = gy[k] = make_float2(0.f, 0.f);
    }
#endif
    int ui = us, off = 0, cur = 0;
    int cnt = stage_chunk(T, buf[0], ui, off, ue, lane);
    while (cnt > 0) {
        // next chunk in flight while this one is summed
        const int nxt = ui < ue ? stage_chunk(T, buf[cur ^ 1], ui, off, ue, lane) : (cp_async_commit(), 0);
        cp_async_wait_one();
        __syncwarp();
        const float4 *src = buf[cur] + h;
        const int steps = cnt / NEAR_SPLIT;
#pragma unroll NEAR_UNROLL
        for (int j = 0; j < steps; ++j) {
            const float4 q = src[j * NEAR_SPLIT];
#if BGL_NEAR_PACKED
#pragma unroll
            for (int k = 0; k < R2; ++k) p2p_pair2(nzx[k], nzy[k], q, gx[k], gy[k]);
#pragma unroll
            for (int r = 2 * R2; r < R; ++r) p2p_pair(zx[r], zy[r], q, fx[r], fy[r]);
#else
#pragma unroll
            for (int r = 0; r < R; ++r) p2p_pair(zx[r], zy[r], q, fx[r], fy[r]);
#endif
        }
        __syncwarp();
        cur ^= 1;
        cnt = nxt;
    }
#if BGL_NEAR_PACKED
#pragma unroll
    for (int k = 0; k < R2; ++k) {
        fx[2 * k] = -gx[k].x;
        fx[2 * k + 1] = -gx[k].y;
        fy[2 * k] = -gy[k].x;
        fy[2 * k + 1] = -gy[k].y;
    }
#endif
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float sx = fx[r], sy = fy[r];
#pragma unroll
        for (int o = NEAR_LPS; o < 32; o <<= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        // every lane now holds the sums of its target lane; split h stores
        // the targets r = h (mod NEAR_SPLIT)
        const int i = t + r * NEAR_LPS;
        if (r % NEAR_SPLIT == h && i < ntc) {
            const int zi = __float_as_int(T.pts[tb + i].w);
            la.f[la.q0 + zi - la.fbase] = make_float2(sx, sy);
        }
    }
}

// The near and far fields are computed by two kernels that may run at the
// same time (the near sum into f, the far field into ef, both by the
// point's component-local index); once both are done, one coalesced pass
// writes the force of every point:
//   F_rep(o) = kr m_o (near(o) + conj(E(z_o))) (+ fa(o))
// It also empties the child slots of this evaluation's boxes for the next
// tree (the emit kernel fills only the slots of children that exist; the
// plan starts with all slots empty).
__global__ void combine_kernel(LeafArgs la, int n) {
    if (aborted(la.e.T.err)) return;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const Tree &T = la.e.T;
    for (int b = o, B = min(T.levoff[NLEV], T.Bmax); b < B; b += gridDim.x * blockDim.x)
        T.bchild[b] = make_int4(-1, -1, -1, -1);
    float sw = 0.f, tr = 0.f;
    if (o < n) {
        const int64_t q = la.q0 + o - la.fbase;
        const float2 nr = la.f[q];
        const float2 E = la.ef[o];
        const float km = la.kr * la.mass[o];
        const float2 a = la.fa ? la.fa[q] : make_float2(0.f, 0.f);
        const float2 F = make_float2(fmaf(km, nr.x + E.x, a.x), fmaf(km, nr.y - E.y, a.y));
        la.f[q] = F;
        if (la.fprev) fa2_swing_terms(F, la.fprev[q], la.mass[o], la.variant, sw, tr);
    }
    if (!la.fprev) return;
    // swing/traction of the iteration (Section 3.2): FP32 within a warp, FP64
    // across warps and blocks, blocks summed in order by the last to arrive
    __shared__ double ws[32], wt[32];
    __shared__ bool last;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, k);
        tr += __shfl_xor_sync(0xffffffffu, tr, k);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        ws[warp] = (double)sw;
        wt[warp] = (double)tr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, u = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s += ws[w];
            u += wt[w];
        }
        la.spart[blockIdx.x] = make_double2(s, u);
        __threadfence();
        last = atomicAdd(la.scount, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block: thread t sums the partials t, t + blockDim, ... (fixed
    // order), then the block's sums in warp order
    double swg = 0.0, trc = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        const double2 v = __ldcg(&la.spart[k]);
        swg += v.x;
        trc += v.y;
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        swg += __shfl_xor_sync(0xffffffffu, swg, k);
        trc += __shfl_xor_sync(0xffffffffu, trc, k);
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
        const double s_new = fa2_global_speed(swg, trc, *la.sg, la.tau);
        *la.sg = s_new;
        if (la.stats) {
            const int it = *la.iter;
            la.stats[3 * it] = swg;
            la.stats[3 * it + 1] = trc;
            la.stats[3 * it + 2] = s_new;
        }
        *la.iter += 1;
        *la.scount = 0u;
    }
}

// Fused update: every point moves by s F (Section 3.2) and F_{t-1} <- F;
// the new positions give the next evaluation's root square, and block 0
// clears the next evaluation's tickets and counts (what bbox_kernel does).
__global__ void update_root_kernel(float2 *xy, const float2 *__restrict__ f, float2 *fprev, int n, const double *sg,
                                   float ks, float ksmax, int *bad, float4 *__restrict__ part, unsigned *counter,
                                   Root *root, int *err, unsigned *epoch, int *tickets, OsHist h) {
    evaluation_clear(tickets, h);
    const float g = (float)*sg;
    float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // one point per thread
    if (i < n) {
        const float2 F = f[i], P = fprev[i];
        const float2 p = fa2_move(xy[i], F, P, g, ks, ksmax);
        if (!isfinite(p.x) || !isfinite(p.y)) *bad = 1;
        xy[i] = p;
        fprev[i] = F;
        mnx = fminf(mnx, p.x);
        mxx = fmaxf(mxx, p.x);
        mny = fminf(mny, p.y);
        mxy = fmaxf(mxy, p.y);
    }
    bbox_reduce_root(mnx, mxx, mny, mxy, part, counter, root, err, epoch);
}

// the tile variant with R targets per lane
template <int R>
__device__ __forceinline__ void near_dispatch(int r, const Tree &T, LeafArgs &la, float4 (*buf)[NEAR_SRC], int tb,
                                              int ntc, int us, int ue, int lane) {
    if constexpr (R > 1) {
        if (r < R) {
            near_dispatch<R - 1>(r, T, la, buf, tb, ntc, us, ue, lane);
            return;
        }
    }
    near_tile<R>(T, la, buf, tb, ntc, us, ue, lane);
}

__global__ void __launch_bounds__(NEAR_WARPS * 32) near_kernel(LeafArgs la) {
    if (aborted(la.e.T.err)) return;
    const Tree &T = la.e.T;
    __shared__ __align__(16) float4 stage[NEAR_WARPS][2][NEAR_SRC];
    const int lane = threadIdx.x & 31;
    float4(*buf)[NEAR_SRC] = stage[threadIdx.x >> 5];
#if BGL_NEAR_BUCKETS
    // leaves bucket by bucket, the most targets per lane first
    int cnt_l = lane < NEAR_RMAX ? T.ncls[lane] : 0;
    int total = cnt_l;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(la.ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) return;
        int cls = NEAR_RMAX;
        for (;; --cls) {
            const int c = __shfl_sync(0xffffffffu, cnt_l, cls - 1);
            if (t < c) break;
            t -= c;
        }
        const int b = T.cleaf[(size_t)(cls - 1) * T.Bmax + t];
#else
    const int B = min(T.levoff[NLEV], T.Bmax);
    for (;;) {
        int b = 0;
        if (lane == 0) b = atomicAdd(la.ticket, 1);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= B) return;
        if (!T.bleaf[b]) continue;
#endif
        const int s = T.bstart[b], e = T.bend[b];
        const int us = T.lofs[5 * b], ue = T.lofs[5 * b + 1];
        for (int tb = s; tb < e; tb += NEAR_LPS * NEAR_RMAX) {
            const int ntc = min(NEAR_LPS * NEAR_RMAX, e - tb);
            near_dispatch<NEAR_RMAX>((ntc + NEAR_LPS - 1) / NEAR_LPS, T, la, buf, tb, ntc, us, ue, lane);
        }
    }
}

// Far field of every target of a leaf (one warp per leaf).  First the
// leaf's incoming expansion: the sum over its ancestors A of levels >= 2
// (and itself) of A's M2L + P2L expansion shifted from c_A to the leaf
// centre -- the chain of L2L shifts of the downward pass composed into one
// shift per ancestor (ancestors found by independent hash lookups):
//   b~_m(leaf) += 2^(-D m) sum_{l >= m} b~_l(A) C(l, m) t^(l-m),
//   t = (c_leaf - c_A) / r_A, D = level(leaf) - level(A);
// lane m computes coefficient m.  Then, a lane per target: L2P of that
// expansion and M2P over W (W boxes staged in shared memory), the field E
// stored for the combine pass; a longer W list is far_heavy_kernel's.
constexpr int FAR_WARPS = 4;
constexpr int FAR_W = 16;        // W entries staged in shared memory
constexpr int FAR_HEAVY = 16;    // longer W lists: the M2P goes to far_heavy_kernel (sixteen warps per leaf)
static_assert(FAR_HEAVY <= FAR_W, "every W list the far kernel keeps fits its staging");

// M2P of W entry k at z: E += (a~_0 - sum_k k a~_k t^k) / (z - c_D), t = r_D / (z - c_D)
template <int PT>
__device__ __forceinline__ float2 m2p_term(const Tree &T, const Root *rt, const float2 *M, int p, int k, float4 z) {
    const int Dx = T.lidx[k];
    const int2 md_ = T.bmeta[Dx];
    const BoxGeo gd = box_geo_xy(rt, md_.x, md_.y & 255);
    const float2 dz = make_float2(z.x - gd.cx, z.y - gd.cy);
    const float id2 = rcp_approx(fmaf(dz.x, dz.x, dz.y * dz.y));
    const float2 idz = make_float2(dz.x * id2, -dz.y * id2);
    const float2 tt2 = cscale(idz, gd.r);
    const float2 *md = M + (size_t)Dx * (PT + 1);
    float2 hs = make_float2(0.f, 0.f);
#pragma unroll
    for (int kk = PT; kk >= 1; --kk) {
        if (kk <= p) hs = cadd(cmul(hs, tt2), cscale(md[kk], (float)kk));
    }
    hs = cmul(hs, tt2);
    const float2 a0 = md[0];
    return cmul(make_float2(a0.x - hs.x, a0.y - hs.y), idz);
}

template <int PT>
__global__ void __launch_bounds__(FAR_WARPS * 32, 12) far_kernel(LeafArgs la) {
    if (aborted(la.e.T.err)) return;
    __shared__ float sbin[(PT + 1) * (PT + 1)];   // C(l, m), l, m <= PT
    __shared__ float2 loc[FAR_WARPS][PT + 1];
    __shared__ float2 ancl[FAR_WARPS][MAXLEV - 1][PT + 1];
    __shared__ float2 part_[FAR_WARPS][MAXLEV - 1][PT + 1];
    __shared__ int s_anc[FAR_WARPS][MAXLEV - 1];
    __shared__ float2 s_t[FAR_WARPS][MAXLEV - 1];
    __shared__ float4 s_wg[FAR_WARPS][FAR_W];             // W box centre and half-width
    __shared__ float2 s_wm[FAR_WARPS][FAR_W][PT + 1];     // W box outgoing expansion
    for (int i = threadIdx.x; i < (PT + 1) * (PT + 1); i += blockDim.x)
        sbin[i] = la.e.binom[(i / (PT + 1)) * BN + i % (PT + 1)];
    __syncthreads();
    const Tree &T = la.e.T;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int B = min(T.levoff[NLEV], T.Bmax);
    const Root *rt = T.root;
    const int p = la.e.p;
    const unsigned epoch = *T.epoch;
    for (int b = gw; b < B; b += nw) {
        const int2 mb = T.bmeta[b];
        if (!meta_leaf(mb)) continue;
        const int Lb = mb.y & 255;
        const uint32_t kb = T.bkey[b];
        const int s = T.bstart[b], e = T.bend[b];
        const int ws = T.lofs[5 * b + 2], we = T.lofs[5 * b + 3];
        const int nW = we - ws;
        // a W list longer than the staging is left to far_heavy_kernel, which spreads it over warps
        const bool heavy = nW > FAR_HEAVY;
        const bool wst = !heavy;
        if (heavy && lane == 0) {
            const int h = atomicAdd(la.nheavy, 1);
            if (h < la.heavy_cap) la.heavy[h] = b;
            else atomicOr(T.err, ERR_LIST_OVERFLOW);
        }
        // a short W list: its boxes' geometry and expansions in shared memory
        if (wst && lane < nW) {
            const int Dx = T.lidx[ws + lane];
            const int2 md_ = T.bmeta[Dx];
            const BoxGeo gd = box_geo_xy(rt, md_.x, md_.y & 255);
            s_wg[wib][lane] = make_float4(gd.cx, gd.cy, gd.r, __int_as_float(Dx));
        }
        // ancestors of levels >= 2 (lane j: level Lb - j, key kb >> 2j), found by
        // independent hash lookups, and the shift t_j = (c_leaf - c_A) / r_A
        const int nA = Lb >= 2 ? Lb - 1 : 0;
        if (lane < nA) {
            s_anc[wib][lane] = lane == 0 ? b : hash_find(T, epoch, Lb - lane, kb >> (2 * lane));
            const uint32_t ka = kb >> (2 * lane);
            const float sc = ldexpf(1.0f, -lane);
            const float sx = (float)((int)(2 * compact_bits(kb) + 1) - (int)(2 * compact_bits(ka) + 1) * (1 << lane));
            const float sy =
                (float)((int)(2 * compact_bits(kb >> 1) + 1) - (int)(2 * compact_bits(ka >> 1) + 1) * (1 << lane));
            s_t[wib][lane] = make_float2(sx * sc, sy * sc);
        }
        __syncwarp();
        // their partial local expansions (M2L + P2L) staged in shared memory
        for (int it = lane; it < nA * (PT + 1); it += 32) {
            const int j = it / (PT + 1), l = it - j * (PT + 1);
            const int A = s_anc[wib][j];
            ancl[wib][j][l] = A >= 0 && l <= p ? la.e.Lc[(size_t)A * (PT + 1) + l] : make_float2(0.f, 0.f);
        }
        if (wst) {
            for (int it = lane; it < nW * (PT + 1); it += 32) {
                const int i = it / (PT + 1), k = it - i * (PT + 1);
                const int Dx = __float_as_int(s_wg[wib][i].w);
                // k a~_k (a~_0 for k = 0): the weights of the M2P Horner sum
                const float2 mk = k <= p ? la.e.M[(size_t)Dx * (PT + 1) + k] : make_float2(0.f, 0.f);
                s_wm[wib][i][k] = k == 0 ? mk : cscale(mk, (float)k);
            }
        }
        __syncwarp();
        // incoming expansion of the leaf: items (ancestor j, coefficient m)
        // spread over all lanes, each a Horner sum in t_j, then each
        // coefficient summed over j in order:
        //   b~_m(leaf) += 2^(-j m) sum_{l >= m} b~_l(A_j) C(l, m) t_j^(l-m)
        for (int it = lane; it < nA * PT; it += 32) {
            const int j = it / PT, m = it - j * PT + 1;
            float2 sres = make_float2(0.f, 0.f);
            if (m <= p) {
                const float2 t = s_t[wib][j];
                for (int l = p; l >= m; --l) sres = cadd(cmul(sres, t), cscale(ancl[wib][j][l], sbin[l * (PT + 1) + m]));
            }
            part_[wib][j][m] = make_float2(ldexpf(sres.x, -j * m), ldexpf(sres.y, -j * m));
        }
        __syncwarp();
        float2 mine = make_float2(0.f, 0.f);
        if (lane >= 1 && lane <= p)
            for (int j = 0; j < nA; ++j) mine = cadd(mine, part_[wib][j][lane]);
        if (lane <= PT) loc[wib][lane] = cscale(mine, (float)lane);     // l b~_l, the L2P weights
        __syncwarp();
        const BoxGeo g = box_geo_xy(rt, mb.x, Lb);
        const float ir = 1.0f / g.r;
        for (int tt = s + lane; tt < e; tt += 32) {
            const float4 z = T.pts[tt];
            float2 E;
            // L2P: E = (1/r) sum_l l b~_l v^(l-1), v = (z - c) / r
            {
                const float2 v = make_float2((z.x - g.cx) * ir, (z.y - g.cy) * ir);
                float2 hs = make_float2(0.f, 0.f);
#pragma unroll
                for (int l = PT; l >= 1; --l) {
                    if (l <= p) hs = cadd(cmul(hs, v), loc[wib][l]);
                }
                E = cscale(hs, ir);
            }
            // M2P: E += (a~_0 - sum_k k a~_k t^k) / (z - c_D), t = r_D / (z - c_D)
            // (a list longer than the staging is far_heavy_kernel's)
            if (!heavy) {
                for (int i = 0; i < nW; ++i) {
                    const float4 gd = s_wg[wib][i];
                    const float2 dz = make_float2(z.x - gd.x, z.y - gd.y);
                    const float id2 = rcp_approx(fmaf(dz.x, dz.x, dz.y * dz.y));
                    const float2 idz = make_float2(dz.x * id2, -dz.y * id2);
                    const float2 tt2 = cscale(idz, gd.z);
                    float2 hs = make_float2(0.f, 0.f);
#pragma unroll
                    for (int kk = PT; kk >= 1; --kk) {
                        if (kk <= p) hs = cadd(cmul(hs, tt2), s_wm[wib][i][kk]);
                    }
                    hs = cmul(hs, tt2);
                    const float2 a0 = s_wm[wib][i][0];
                    E = cadd(E, cmul(make_float2(a0.x - hs.x, a0.y - hs.y), idz));
                }
            }
            la.ef[__float_as_int(z.w)] = E;
        }
    }
}

// The M2P of the leaves with more than FAR_HEAVY W entries (a leaf next to a
// finely divided region can have hundreds, which one warp reading them from
// global memory would take alone long after the rest of the far field is
// done): one block of HEAVY_WARPS warps per leaf, warp w taking the entries
// w, w + HEAVY_WARPS, ..., lanes over 32 targets at a time; warp 0 then adds
// the partial sums in warp order to the L2P value that far_kernel stored.
constexpr int HEAVY_WARPS = 16;

template <int PT>
__global__ void __launch_bounds__(HEAVY_WARPS * 32) far_heavy_kernel(LeafArgs la) {
    if (aborted(la.e.T.err)) return;
    __shared__ float2 part[HEAVY_WARPS][32];
    const Tree &T = la.e.T;
    const Root *rt = T.root;
    const int p = la.e.p;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nh = min(*la.nheavy, la.heavy_cap);
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int b = la.heavy[h];
        const int s = T.bstart[b], e = T.bend[b];
        const int ws = T.lofs[5 * b + 2], we = T.lofs[5 * b + 3];
        for (int t0 = s; t0 < e; t0 += 32) {
            const int tt = t0 + lane;
            float2 acc = make_float2(0.f, 0.f);
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (tt < e) {
                z = T.pts[tt];
                for (int k = ws + warp; k < we; k += HEAVY_WARPS) acc = cadd(acc, m2p_term<PT>(T, rt, la.e.M, p, k, z));
            }
            part[warp][lane] = acc;
            __syncthreads();
            if (warp == 0 && tt < e) {
                const int o = __float_as_int(z.w);
                float2 E = la.ef[o];
#pragma unroll
                for (int w = 0; w < HEAVY_WARPS; ++w) E = cadd(E, part[w][lane]);
                la.ef[o] = E;
            }
            __syncthreads();
        }
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

// float -> bf16 bits, round to nearest even (finite inputs)
static uint16_t bf16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(r >> 16);
}

// mma.m16n8k16 A fragments (row-major 16 x 16 tiles, BF16) of the real M2L
// matrices of the 49 offset classes for expansion order p <= 15; layout
// [class][row tile][depth tile][lane] -> 4 x 32 bits
static std::vector<uint4> m2l_fragments(int p) {
    std::vector<uint4> out((size_t)VCLS * 2 * 2 * 32);
    std::vector<double> R(32 * 32);
    std::vector<double> binom(64 * 64, 0.0);
    for (int i = 0; i < 64; ++i) {
        binom[i * 64] = 1.0;
        for (int k = 1; k <= i; ++k)
            binom[i * 64 + k] = binom[(i - 1) * 64 + k - 1] + (k <= i - 1 ? binom[(i - 1) * 64 + k] : 0.0);
    }
    for (int c = 0; c < VCLS; ++c) {
        std::fill(R.begin(), R.end(), 0.0);
        const double wr = 2.0 * (c / 7 - 3), wi = 2.0 * (c % 7 - 3);
        const double w2 = wr * wr + wi * wi;
        if (w2 > 0.0) {
            // powers of 1/w
            std::vector<double> pr(2 * p + 2), pi(2 * p + 2);
            pr[0] = 1.0;
            pi[0] = 0.0;
            const double ir = wr / w2, ii = -wi / w2;
            for (int j = 1; j <= 2 * p + 1; ++j) {
                pr[j] = pr[j - 1] * ir - pi[j - 1] * ii;
                pi[j] = pr[j - 1] * ii + pi[j - 1] * ir;
            }
            for (int l = 1; l <= p; ++l) {
                for (int k = 0; k <= p; ++k) {
                    double tr, ti;
                    if (k == 0) {
                        tr = -pr[l] / l;
                        ti = -pi[l] / l;
                    } else {
                        const double cf = ((k & 1) ? -1.0 : 1.0) * binom[(l + k - 1) * 64 + (k - 1)];
                        tr = cf * pr[l + k];
                        ti = cf * pi[l + k];
                    }
                    R[(2 * l) * 32 + 2 * k] = tr;
                    R[(2 * l) * 32 + 2 * k + 1] = -ti;
                    R[(2 * l + 1) * 32 + 2 * k] = ti;
                    R[(2 * l + 1) * 32 + 2 * k + 1] = tr;
                }
            }
        }
        auto pk = [&](int r, int col) {
            return (uint32_t)bf16_bits((float)R[r * 32 + col]) |
                   ((uint32_t)bf16_bits((float)R[r * 32 + col + 1]) << 16);
        };
        for (int mt = 0; mt < 2; ++mt)
            for (int kt = 0; kt < 2; ++kt)
                for (int lane = 0; lane < 32; ++lane) {
                    const int gid = lane >> 2, tig = lane & 3;
                    const int r0 = mt * 16 + gid, r1 = r0 + 8, c0 = kt * 16 + tig * 2;
                    out[(((size_t)c * 2 + mt) * 2 + kt) * 32 + lane] =
                        make_uint4(pk(r0, c0), pk(r1, c0), pk(r0, c0 + 8), pk(r1, c0 + 8));
                }
    }
    return out;
}

struct FmmPlan {
    bgl_graph *g = nullptr;
    OsWait wait;           // bounded waits of the sort: error word, poll limit, test stall
    bool fused = false;    // fused ForceAtlas2 iteration (fmm_fuse): no bounding-box kernel, swing in combine
    FmmFuse fz;
    DevBuf<double2> spart; // swing/traction partial sums of the combine blocks
    DevBuf<unsigned> scount;
    int64_t c = 0, q0 = 0;
    int n = 0, p = 8, PT = 8, S = 64, Bmax = 1, ntiles = 1, lcap = 1, grid_p = 1;
    float kr = 1.f;
    DevBuf<Root> root;
    DevBuf<float4> part;
    DevBuf<unsigned> counter;
    DevBuf<uint32_t> key, idx;
    DevBuf<float4> pts;
    DevBuf<int8_t> cl, lam, bleaf;
    DevBuf<int> tcnt, levoff, bstart, bend, blevel, bparent, lofs, lidx;
    DevBuf<int> cleaf;     // near-field buckets of leaves (with BGL_NEAR_BUCKETS)
    DevBuf<uint32_t> bkey;
    DevBuf<int4> bchild;
    DevBuf<int2> bmeta;
    DevBuf<float2> M, Lc;
    DevBuf<int> arrive, tickets, err;
    DevBuf<int> sortskip;     // radix passes the next sort skips (0 or 2), set by the tree of the last evaluation
    // BF16 tensor-core M2L
    bool bf16 = false;
    int vcap = 0;
    DevBuf<uint4> tfrag;      // [VCLS][2][2][32] mma fragments of the translation matrices
    DevBuf<int> vbase, vclass;    // [Bmax]; counts, starts, cursors of the class buckets
    DevBuf<int2> vpairs;      // [vcap]
    DevBuf<float> vout;       // [vcap * VROWS]
    DevBuf<float2> ef;
    DevBuf<int> heavy;        // [Bmax] leaves handed to far_heavy_kernel
    DevBuf<ulonglong2> hkv;
    DevBuf<unsigned> epoch;
    int hmask = 0;
    DevBuf<float> binom;
    SortWorkspace sortws;
    cudaStream_t side = nullptr;          // second stream for the concurrent branch
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ~FmmPlan() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        if (side) cudaStreamDestroy(side);
    }
};

FmmPlan *fmm_create(bgl_graph *g, const bgl_params *p, int64_t c) {
    bgl_ctx *ctx = g->ctx;
    Allocator *A = ctx->alloc;
    cudaStream_t s = ctx->stream;
    FmmPlan *pl = new FmmPlan();
    try {
        pl->g = g;
        pl->c = c;
        pl->q0 = g->h_comp_off[c];
        const int64_t n64 = g->h_comp_off[c + 1] - pl->q0;
        BGL_REQUIRE(n64 < (int64_t(1) << 30), "fmm: component too large");
        pl->n = (int)n64;
        pl->p = p->fmm_p;
        pl->PT = p->fmm_p <= 8 ? 8 : (p->fmm_p <= 12 ? 12 : (p->fmm_p <= 16 ? 16 : 24));
        pl->S = p->leaf_size;
        pl->kr = (float)p->kr;
        const int n = std::max(pl->n, 1);
        // boxes: internal boxes hold > S points, at most n/(S+1) per level for
        // levels 0..15; every other box is a child of one
        int64_t bmax = 1 + 4 * (int64_t)MAXLEV * (n / (pl->S + 1) + 1);
        bmax = std::min<int64_t>(bmax, (int64_t)NLEV * n + 1);
        pl->Bmax = (int)bmax;
        pl->ntiles = (n + TREE_TILE - 1) / TREE_TILE;
        // list entries: U <= 17 per leaf, V <= 27, W and X <= 8 per box
        pl->lcap = (int)std::min<int64_t>((int64_t)60 * bmax + 64, (int64_t)1 << 30);
        pl->root.reset(A, 1);
        pl->part.reset(A, std::max<int64_t>(1024, nblk(pl->n, 256)));   // bounding-box partials, one per block
        pl->counter.reset(A, 1);
        pl->key.reset(A, n);
        pl->idx.reset(A, n);
        pl->pts.reset(A, n);
        pl->cl.reset(A, n);
        pl->lam.reset(A, n);
        pl->tcnt.reset(A, (size_t)NLEV * pl->ntiles + 1);
        pl->levoff.reset(A, NLEV + 1);
        pl->bstart.reset(A, bmax);
        pl->bend.reset(A, bmax);
        pl->blevel.reset(A, bmax);
        pl->bparent.reset(A, bmax);
        pl->bkey.reset(A, bmax);
        pl->bleaf.reset(A, bmax);
        pl->bchild.reset(A, bmax);
        BGL_CUDA(cudaMemsetAsync(pl->bchild.p, 0xFF, sizeof(int4) * bmax, s));
        pl->bmeta.reset(A, bmax);
        pl->lofs.reset(A, 5 * bmax);
        if (BGL_NEAR_BUCKETS) pl->cleaf.reset(A, (size_t)NEAR_RMAX * bmax);
        pl->lidx.reset(A, pl->lcap);
        pl->M.reset(A, (size_t)(pl->PT + 1) * bmax);
        pl->Lc.reset(A, (size_t)(pl->PT + 1) * bmax);
        pl->arrive.reset(A, bmax);
        pl->sortskip.reset(A, 1);
        BGL_CUDA(cudaMemsetAsync(pl->sortskip.p, 0, sizeof(int), s));
        if (p->m2l_bf16) {
            BGL_REQUIRE(pl->p <= 15, "fmm: the BF16 tensor-core M2L takes expansion orders up to 15");
            pl->bf16 = true;
            // V entries: at most 27 per box, with at most n / 2 + 4096 boxes (beyond that
            // the overflow is flagged and the evaluation fails); whole tiles of 8
            pl->vcap = (int)(std::min<int64_t>(std::min<int64_t>(pl->lcap, 27 * ((int64_t)n / 2 + 4096)) + 8 * VCLS,
                                               (int64_t)1 << 30) & ~int64_t(7));
            pl->vbase.reset(A, bmax);
            pl->vclass.reset(A, 3 * VCLS + 1);
            pl->vpairs.reset(A, pl->vcap);
            pl->vout.reset(A, (size_t)pl->vcap * VROWS);
            std::vector<uint4> frag = m2l_fragments(pl->p);
            pl->tfrag.reset(A, frag.size());
            BGL_CUDA(cudaMemcpyAsync(pl->tfrag.p, frag.data(), sizeof(uint4) * frag.size(), cudaMemcpyHostToDevice, s));
        }
        pl->ef.reset(A, n);
        pl->heavy.reset(A, bmax);
        int64_t hs = 1;
        while (hs < 2 * bmax) hs <<= 1;
        pl->hmask = (int)(hs - 1);
        pl->hkv.reset(A, hs);
        pl->epoch.reset(A, 1);
        BGL_CUDA(cudaMemsetAsync(pl->hkv.p, 0, sizeof(ulonglong2) * hs, s));
        BGL_CUDA(cudaMemsetAsync(pl->epoch.p, 0, sizeof(unsigned), s));
        pl->tickets.reset(A, NTICKETS);
        pl->err.reset(A, 1);
        pl->wait.err = pl->err.p;
        {
            // test aid for the failure path: BGL_TEST_SORT_STALL=1 makes the
            // sort's first tile withhold its counts and the waits on it give
            // up after 4,096 polls, so the evaluation reports BGL_ETIMEOUT
            const char *v = std::getenv("BGL_TEST_SORT_STALL");
            if (v && v[0] == '1') {
                pl->wait.stall_first = 1;
                pl->wait.spin = 1 << 12;
            }
        }
        pl->sortws.reserve(A, n, s);
        BGL_CUDA(cudaMemsetAsync(pl->counter.p, 0, sizeof(unsigned), s));
        BGL_CUDA(cudaMemsetAsync(pl->arrive.p, 0, sizeof(int) * bmax, s));
        BGL_CUDA(cudaMemsetAsync(pl->err.p, 0, sizeof(int), s));
        std::vector<float> bn(BN * BN, 0.f);
        for (int i = 0; i < BN; ++i) {
            double v = 1.0;
            for (int k = 0; k <= i; ++k) {
                bn[i * BN + k] = (float)v;
                v = v * (double)(i - k) / (double)(k + 1);
            }
        }
        pl->binom.reset(A, BN * BN);
        BGL_CUDA(cudaMemcpyAsync(pl->binom.p, bn.data(), sizeof(float) * bn.size(), cudaMemcpyHostToDevice, s));
        BGL_CUDA(cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking));
        for (auto &e : pl->ev) BGL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        BGL_CUDA(cudaStreamSynchronize(s));
        pl->grid_p = ctx->num_sms * 8;
    } catch (...) {
        delete pl;
        throw;
    }
    return pl;
}

void fmm_destroy(FmmPlan *pl) { delete pl; }

static Tree make_tree(FmmPlan *pl) {
    Tree T;
    T.key = pl->key.p;
    T.pts = pl->pts.p;
    T.n = pl->n;
    T.bstart = pl->bstart.p;
    T.bend = pl->bend.p;
    T.blevel = pl->blevel.p;
    T.bparent = pl->bparent.p;
    T.bkey = pl->bkey.p;
    T.bleaf = pl->bleaf.p;
    T.bchild = pl->bchild.p;
    T.bmeta = pl->bmeta.p;
    T.levoff = pl->levoff.p;
    T.lofs = pl->lofs.p;
    T.lidx = pl->lidx.p;
    T.pool = pl->tickets.p + 3;
    T.hkv = pl->hkv.p;
    T.hmask = pl->hmask;
    T.epoch = pl->epoch.p;
    T.lcap = pl->lcap;
    T.Bmax = pl->Bmax;
    T.root = pl->root.p;
    T.err = pl->err.p;
    T.ncls = pl->tickets.p + NEAR_BUCKET_COUNTS;
    T.cleaf = pl->cleaf.p;
    return T;
}

static ExpArgs exp_args(FmmPlan *pl, const Tree &T) {
    ExpArgs a;
    a.T = T;
    a.M = pl->M.p;
    a.Lc = pl->Lc.p;
    a.arrive = pl->arrive.p;
    a.done = nullptr;
    a.ticket = pl->tickets.p + 1;
    a.binom = pl->binom.p;
    a.p = pl->p;
    a.vout = pl->bf16 ? pl->vout.p : nullptr;
    a.vbase = pl->bf16 ? pl->vbase.p : nullptr;
    return a;
}

static LeafArgs leaf_args(FmmPlan *pl, const ExpArgs &a, float2 *f, int64_t fbase, const float2 *fa) {
    LeafArgs la;
    la.e = a;
    la.f = f;
    la.fa = fa;
    la.q0 = pl->q0;
    la.fbase = fbase;
    la.kr = pl->kr;
    la.ticket = pl->tickets.p + 2;
    la.ef = pl->ef.p;
    la.mass = pl->g->mass.p + pl->q0;
    la.heavy = pl->heavy.p;
    la.nheavy = pl->tickets.p + 4;
    la.heavy_cap = pl->Bmax;
    la.fprev = pl->fused ? pl->fz.fprev : nullptr;      // indexed like f
    la.variant = pl->fz.variant;
    la.tau = pl->fz.tau;
    la.sg = pl->fz.sg;
    la.stats = pl->fz.stats;
    la.iter = pl->fz.iter;
    la.spart = pl->spart.p;
    la.scount = pl->scount.p;
    return la;
}

static unsigned bbox_blocks(const FmmPlan *pl) {
    return (unsigned)std::min<int64_t>(2 * pl->g->ctx->num_sms, nblk(pl->n, 256));
}

// points: bounding box, keys, sort, gather (also clears the tickets and the list pool)
static void phase_points(FmmPlan *pl, const float2 *xl, cudaStream_t s) {
    bgl_ctx *ctx = pl->g->ctx;
    const int n = pl->n;
    const float *ml = pl->g->mass.p + pl->q0;
    cudaStream_t keep = ctx->stream;
    ctx->stream = s;
    try {
        // tickets, digit counts and look-back words are zeroed by bbox_kernel
        // (by update_root_kernel in a fused iteration, which also made the root)
        // and keys_kernel
        const OsHist h = radix_sort_u32_ws_begin(ctx, pl->sortws, n, false);
        if (!pl->fused) {
            bbox_kernel<<<bbox_blocks(pl), 256, 0, s>>>(xl, n, pl->part.p, pl->counter.p, pl->root.p, pl->err.p,
                                                       pl->epoch.p, pl->tickets.p, h);
            BGL_LAUNCH_CHECK();
        }
        keys_kernel<<<nblk(n, 256 * KEY_ITEMS), 256, 0, s>>>(xl, n, pl->root.p, pl->key.p, pl->idx.p, h);
        BGL_LAUNCH_CHECK();
        radix_sort_u32_ws_scatter(ctx, pl->sortws, pl->key.p, pl->idx.p, n, xl, ml, pl->pts.p, pl->sortskip.p,
                                  pl->wait);
    } catch (...) {
        ctx->stream = keep;
        throw;
    }
    ctx->stream = keep;
}

// tree: boxes in level order, ends, parents, children
static void phase_tree(FmmPlan *pl, const Tree &T, cudaStream_t s) {
    tree_count_kernel<<<pl->ntiles, TREE_THREADS, 0, s>>>(pl->key.p, pl->n, pl->S, pl->cl.p, pl->lam.p, pl->tcnt.p,
                                                          pl->ntiles, pl->sortskip.p, pl->tickets.p + 6, pl->err.p);
    BGL_LAUNCH_CHECK();
    tree_scan_kernel<<<1, SCAN_THREADS, 0, s>>>(pl->tcnt.p, pl->ntiles, pl->levoff.p, pl->Bmax, pl->err.p,
                                                pl->tickets.p + 6, pl->sortskip.p);
    BGL_LAUNCH_CHECK();
    tree_emit_kernel<<<pl->ntiles, TREE_THREADS, 0, s>>>(T, pl->cl.p, pl->lam.p, pl->tcnt.p, pl->ntiles, pl->Bmax);
    BGL_LAUNCH_CHECK();
}

// neighbour tables and interaction lists
static void phase_lists(FmmPlan *pl, const Tree &T, cudaStream_t s) {
    nbr_lists_kernel<<<pl->grid_p, 256, 0, s>>>(T);
    BGL_LAUNCH_CHECK();
}

template <int PT>
static void launch_up(FmmPlan *pl, const ExpArgs &a, cudaStream_t s) {
    up_kernel<PT><<<pl->grid_p, 256, 0, s>>>(a);
    BGL_LAUNCH_CHECK();
}
template <int PT>
static void launch_down(FmmPlan *pl, const ExpArgs &a, cudaStream_t s) {
    if (pl->bf16) {
        int *cnt = pl->vclass.p, *start = cnt + VCLS, *cursor = start + VCLS + 1;
        BGL_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * VCLS, s));
        vbase_kernel<<<pl->grid_p / 4, 256, 0, s>>>(a.T, pl->tickets.p + 7, pl->vcap, pl->vbase.p);
        BGL_LAUNCH_CHECK();
        vclass_count_kernel<<<pl->grid_p / 4, 256, 0, s>>>(a.T, cnt);
        BGL_LAUNCH_CHECK();
        vclass_scan_kernel<<<1, 32, 0, s>>>(cnt, start, cursor, pl->vcap, pl->vpairs.p, pl->err.p);
        BGL_LAUNCH_CHECK();
        vclass_scatter_kernel<<<pl->grid_p / 4, 256, 0, s>>>(a.T, cursor, pl->vbase.p, pl->vcap, pl->vpairs.p);
        BGL_LAUNCH_CHECK();
        m2l_bf16_kernel<<<pl->grid_p, 256, 0, s>>>(a.T, a.M, PT + 1, pl->p, start, pl->vpairs.p, pl->tfrag.p, pl->vcap,
                                                   pl->vout.p);
        BGL_LAUNCH_CHECK();
    }
    if (pl->bf16)
        m2l_kernel<PT, true><<<pl->grid_p, 256, 0, s>>>(a);
    else
        m2l_kernel<PT, false><<<pl->grid_p, 256, 0, s>>>(a);
    BGL_LAUNCH_CHECK();
}
// Persistent near-field grid: every resident block of every SM when the
// near field runs alone, one block per SM fewer when the far-field kernels
// run beside it on the side stream.  Four near blocks take nearly all of an
// SM's registers, so the latency-bound far-field kernels beside them found
// no room until near blocks retired (bench step 149.3 ms with four near
// blocks per SM, 147.7 with three, 154.3 with two).  BGL_NEAR_BLOCKS_PER_SM
// (read once per process) sets the count for both cases, up to the
// resident maximum.
static int near_blocks_per_sm(bool beside) {
    static const int full = [] {
        int b = 0;
        BGL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, near_kernel, NEAR_WARPS * 32, 0));
        return b > 0 ? b : 1;
    }();
    static const int forced = [] {
        const char *v = std::getenv("BGL_NEAR_BLOCKS_PER_SM");
        return v ? std::atoi(v) : 0;
    }();
    if (forced > 0) return std::min(forced, full);
    return beside && full > 1 ? full - 1 : full;
}
static void launch_near(FmmPlan *pl, const LeafArgs &la, cudaStream_t s, bool beside) {
    near_kernel<<<pl->g->ctx->num_sms * near_blocks_per_sm(beside), NEAR_WARPS * 32, 0, s>>>(la);
    BGL_LAUNCH_CHECK();
}
template <int PT>
static void launch_far(FmmPlan *pl, const LeafArgs &la, cudaStream_t s) {
    far_kernel<PT><<<2 * pl->grid_p, FAR_WARPS * 32, 0, s>>>(la);
    BGL_LAUNCH_CHECK();
    far_heavy_kernel<PT><<<pl->g->ctx->num_sms, HEAVY_WARPS * 32, 0, s>>>(la);
    BGL_LAUNCH_CHECK();
}
static void launch_combine(FmmPlan *pl, const LeafArgs &la, cudaStream_t s) {
    combine_kernel<<<nblk(pl->n, 256), 256, 0, s>>>(la, pl->n);
    BGL_LAUNCH_CHECK();
}

// Whole evaluation.  With `concurrent`, the upward and downward passes and
// the far field run on the plan's side stream while the near field runs on
// the main stream; the combine pass joins them:
//   main: points, tree --+-- lists ----+-- near ---------------------+-- combine
//   side:                +-- up -------+-- (lists) down -- far ------+
// ev (timing events, 7, may be null) forces one stream and marks the phases.
template <int PT>
static void evaluate(FmmPlan *pl, const float2 *xl, float2 *f, int64_t fbase, bool concurrent, cudaEvent_t *ev,
                     const float2 *fa = nullptr, cudaEvent_t fa_ready = nullptr) {
    cudaStream_t s = pl->g->ctx->stream;
    const Tree T = make_tree(pl);
    const ExpArgs a = exp_args(pl, T);
    const LeafArgs la = leaf_args(pl, a, f, fbase, fa);
    if (ev) BGL_CUDA(cudaEventRecord(ev[0], s));
    phase_points(pl, xl, s);
    if (ev) BGL_CUDA(cudaEventRecord(ev[1], s));
    phase_tree(pl, T, s);
    if (ev) BGL_CUDA(cudaEventRecord(ev[2], s));
    if (!concurrent) {
        phase_lists(pl, T, s);
        if (ev) BGL_CUDA(cudaEventRecord(ev[3], s));
        launch_up<PT>(pl, a, s);
        if (ev) BGL_CUDA(cudaEventRecord(ev[4], s));
        launch_down<PT>(pl, a, s);
        if (ev) BGL_CUDA(cudaEventRecord(ev[5], s));
        launch_near(pl, la, s, false);
        if (ev) BGL_CUDA(cudaEventRecord(ev[6], s));
        launch_far<PT>(pl, la, s);
        if (fa_ready) BGL_CUDA(cudaStreamWaitEvent(s, fa_ready, 0));
        launch_combine(pl, la, s);
        if (ev) BGL_CUDA(cudaEventRecord(ev[7], s));
        return;
    }
    cudaStream_t t = pl->side;
    BGL_CUDA(cudaEventRecord(pl->ev[0], s));           // tree built
    BGL_CUDA(cudaStreamWaitEvent(t, pl->ev[0], 0));
    launch_up<PT>(pl, a, t);
    phase_lists(pl, T, s);
    BGL_CUDA(cudaEventRecord(pl->ev[1], s));           // lists built
    launch_near(pl, la, s, true);
    BGL_CUDA(cudaStreamWaitEvent(t, pl->ev[1], 0));
    launch_down<PT>(pl, a, t);
    launch_far<PT>(pl, la, t);
    BGL_CUDA(cudaEventRecord(pl->ev[2], t));           // far field done
    BGL_CUDA(cudaStreamWaitEvent(s, pl->ev[2], 0));
    if (fa_ready) BGL_CUDA(cudaStreamWaitEvent(s, fa_ready, 0));
    launch_combine(pl, la, s);
}

static void evaluate_any(FmmPlan *pl, const float2 *xl, float2 *f, int64_t fbase, bool concurrent, cudaEvent_t *ev,
                         const float2 *fa = nullptr, cudaEvent_t fa_ready = nullptr) {
    if (pl->PT == 8) evaluate<8>(pl, xl, f, fbase, concurrent, ev, fa, fa_ready);
    else if (pl->PT == 12) evaluate<12>(pl, xl, f, fbase, concurrent, ev, fa, fa_ready);
    else if (pl->PT == 16) evaluate<16>(pl, xl, f, fbase, concurrent, ev, fa, fa_ready);
    else evaluate<24>(pl, xl, f, fbase, concurrent, ev, fa, fa_ready);
}

void fmm_repulsion(FmmPlan *pl, const float2 *xy, int64_t qbase, float2 *f, int64_t fbase, const float2 *fa,
                   cudaEvent_t fa_ready) {
    if (pl->n <= 0) return;
    evaluate_any(pl, xy + (pl->q0 - qbase), f, fbase, true, nullptr, fa, fa_ready);
}

namespace {

// interaction counts: P2P pairs, M2P and P2L point-box terms
__global__ void count_kernel(Tree T, unsigned long long *out) {
    if (aborted(T.err)) return;
    const int B = min(T.levoff[NLEV], T.Bmax);
    unsigned long long p2p = 0, m2p = 0, p2l = 0, leaves = 0, depth = 0, m2l = 0, heavy = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        depth = max(depth, (unsigned long long)T.blevel[b]);
        m2l += (unsigned long long)(T.lofs[5 * b + 2] - T.lofs[5 * b + 1]);
        const int X0 = T.lofs[5 * b + 3], X1 = T.lofs[5 * b + 4];
        for (int e = X0; e < X1; ++e) {
            const int C = T.lidx[e];
            p2l += (unsigned long long)(T.bend[C] - T.bstart[C]);
        }
        if (!T.bleaf[b]) continue;
        ++leaves;
        const unsigned long long nt = (unsigned long long)(T.bend[b] - T.bstart[b]);
        unsigned long long ns = 0;
        for (int e = T.lofs[5 * b]; e < T.lofs[5 * b + 1]; ++e) {
            const int C = T.lidx[e];
            ns += (unsigned long long)(T.bend[C] - T.bstart[C]);
        }
        p2p += nt * ns;
        m2p += nt * (unsigned long long)(T.lofs[5 * b + 3] - T.lofs[5 * b + 2]);
        heavy += (T.lofs[5 * b + 3] - T.lofs[5 * b + 2]) > FAR_HEAVY ? 1ull : 0ull;
    }
    atomicAdd(&out[0], p2p);
    atomicAdd(&out[1], m2p);
    atomicAdd(&out[2], p2l);
    atomicAdd(&out[3], leaves);
    atomicMax(&out[4], depth);
    atomicAdd(&out[5], m2l);
    atomicAdd(&out[6], heavy);
}

}  // namespace

void fmm_profile(FmmPlan *pl, const float2 *xy, int64_t qbase, int reps, double *out) {
    bgl_ctx *ctx = pl->g->ctx;
    cudaStream_t s = ctx->stream;
    const float2 *xl = xy + (pl->q0 - qbase);
    const Tree T = make_tree(pl);
    DevBuf<float2> f(ctx->alloc, std::max(pl->n, 1));
    std::vector<float2> f_first(pl->n), f_last(pl->n);
    cudaEvent_t ev[8], c0, c1;
    for (auto &e : ev) BGL_CUDA(cudaEventCreate(&e));
    BGL_CUDA(cudaEventCreate(&c0));
    BGL_CUDA(cudaEventCreate(&c1));
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    try {
        const int R = std::max(reps, 1);
        for (int r = 0; r < R; ++r) {
            evaluate_any(pl, xl, f.p, pl->q0, false, ev);
            BGL_CUDA(cudaEventSynchronize(ev[7]));
            float ms;
            for (int k = 0; k < 7; ++k) {
                BGL_CUDA(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
                acc[k] += ms;
            }
            if (r == 0 && pl->n > 0)
                BGL_CUDA(cudaMemcpy(f_first.data(), f.p, sizeof(float2) * pl->n, cudaMemcpyDeviceToHost));
        }
        // the concurrent schedule used inside ForceAtlas2 iterations
        for (int r = 0; r < R; ++r) {
            BGL_CUDA(cudaEventRecord(c0, s));
            evaluate_any(pl, xl, f.p, pl->q0, true, nullptr);
            BGL_CUDA(cudaEventRecord(c1, s));
            BGL_CUDA(cudaEventSynchronize(c1));
            float ms;
            BGL_CUDA(cudaEventElapsedTime(&ms, c0, c1));
            acc[7] += ms;
        }
    } catch (...) {
        for (auto &e : ev) cudaEventDestroy(e);
        cudaEventDestroy(c0);
        cudaEventDestroy(c1);
        throw;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    cudaEventDestroy(c0);
    cudaEventDestroy(c1);
    // the first evaluation (sorting all key bits) against the last (with the
    // radix passes the plan chose from the tree): largest difference relative
    // to the largest force
    const int skip_last = fmm_sortskip(pl);
    if (pl->n > 0) BGL_CUDA(cudaMemcpy(f_last.data(), f.p, sizeof(float2) * pl->n, cudaMemcpyDeviceToHost));
    double dmax = 0.0, fmax = 0.0;
    for (int i = 0; i < pl->n; ++i) {
        dmax = std::max(dmax, (double)std::hypot(f_last[i].x - f_first[i].x, f_last[i].y - f_first[i].y));
        fmax = std::max(fmax, (double)std::hypot(f_first[i].x, f_first[i].y));
    }
    DevBuf<unsigned long long> cnt(ctx->alloc, 7);
    BGL_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * 7, s));
    count_kernel<<<pl->grid_p, 256, 0, s>>>(T, cnt.p);
    BGL_LAUNCH_CHECK();
    unsigned long long h[7];
    int lev[NLEV + 1];
    BGL_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaMemcpyAsync(lev, pl->levoff.p, sizeof(lev), cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    const double R = std::max(reps, 1);
    out[0] = std::min(lev[NLEV], pl->Bmax);
    out[1] = (double)h[3];
    out[2] = (double)h[4];
    out[3] = (double)h[0];
    out[4] = (double)h[5];
    out[5] = (double)h[1];
    out[6] = (double)h[2];
    for (int k = 0; k < 8; ++k) out[7 + k] = acc[k] / R;
    out[15] = fmax > 0.0 ? dmax / fmax : 0.0;
    out[16] = (double)skip_last;
    out[17] = (double)h[6];
}

void fmm_fuse(FmmPlan *pl, const FmmFuse &fz) {
    bgl_ctx *ctx = pl->g->ctx;
    pl->fz = fz;
    if (!pl->spart.p) {
        pl->spart.reset(ctx->alloc, nblk(pl->n, 256));
        pl->scount.reset(ctx->alloc, 1);
        BGL_CUDA(cudaMemsetAsync(pl->scount.p, 0, sizeof(unsigned), ctx->stream));
    }
    pl->fused = true;
}

void fmm_root(FmmPlan *pl, const float2 *xy, int64_t qbase) {
    bgl_ctx *ctx = pl->g->ctx;
    const OsHist h = radix_sort_u32_ws_begin(ctx, pl->sortws, pl->n, false);
    bbox_kernel<<<bbox_blocks(pl), 256, 0, ctx->stream>>>(xy + (pl->q0 - qbase), pl->n, pl->part.p, pl->counter.p,
                                                          pl->root.p, pl->err.p, pl->epoch.p, pl->tickets.p, h);
    BGL_LAUNCH_CHECK();
}

void fmm_update_root(FmmPlan *pl, float2 *xy, int64_t qbase, const float2 *f, float2 *fprev, int64_t fbase) {
    bgl_ctx *ctx = pl->g->ctx;
    const OsHist h = radix_sort_u32_ws_begin(ctx, pl->sortws, pl->n, false);
    update_root_kernel<<<nblk(pl->n, 256), 256, 0, ctx->stream>>>(
        xy + (pl->q0 - qbase), f + (pl->q0 - fbase), fprev + (pl->q0 - fbase), pl->n, pl->fz.sg, pl->fz.ks,
        pl->fz.ksmax, pl->fz.bad, pl->part.p, pl->counter.p, pl->root.p, pl->err.p, pl->epoch.p, pl->tickets.p, h);
    BGL_LAUNCH_CHECK();
}

int fmm_sortskip(FmmPlan *pl) {
    int v = 0;
    BGL_CUDA(cudaMemcpyAsync(&v, pl->sortskip.p, sizeof(int), cudaMemcpyDeviceToHost, pl->g->ctx->stream));
    BGL_CUDA(cudaStreamSynchronize(pl->g->ctx->stream));
    return v;
}

void fmm_set_sortskip(FmmPlan *pl, int skip) {
    BGL_REQUIRE(skip == 0 || skip == 2, "fmm: sort pass skip must be 0 or 2");
    BGL_CUDA(cudaMemcpyAsync(pl->sortskip.p, &skip, sizeof(int), cudaMemcpyHostToDevice, pl->g->ctx->stream));
    BGL_CUDA(cudaStreamSynchronize(pl->g->ctx->stream));
}

int fmm_error(FmmPlan *pl) {
    int e = 0;
    BGL_CUDA(cudaMemcpyAsync(&e, pl->err.p, sizeof(int), cudaMemcpyDeviceToHost, pl->g->ctx->stream));
    BGL_CUDA(cudaStreamSynchronize(pl->g->ctx->stream));
    if (sort_workspace_error(pl->g->ctx, pl->sortws)) e |= ERR_SPIN;
    // a failed evaluation may have stopped before its combine pass: empty
    // every child slot again so that the plan stays usable
    if (e) {
        BGL_CUDA(cudaMemsetAsync(pl->bchild.p, 0xFF, sizeof(int4) * pl->Bmax, pl->g->ctx->stream));
        BGL_CUDA(cudaStreamSynchronize(pl->g->ctx->stream));
    }
    return e;
}

}  // namespace bgl
