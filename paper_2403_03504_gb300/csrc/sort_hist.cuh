// Block-level digit histograms for the onesweep radix sort (sort.cu).
#pragma once
#include "bgl_internal.cuh"

namespace bgl {

// Radix tiles: OS_THREADS threads x OS_ITEMS keys.  A caller's histogram
// kernel (os_block_hist, os_clear_status) runs one block per tile.
#ifndef BGL_OS_ITEMS
#define BGL_OS_ITEMS 16
#endif
constexpr int OS_THREADS = 256;
constexpr int OS_ITEMS = BGL_OS_ITEMS;
static_assert(OS_ITEMS >= 1 && OS_ITEMS <= 32, "a thread's keys are tracked in a 32-bit mask");
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;

// Adds the block's keys (key[r] for the bits r of `valid`) to the four 8-bit
// digit histograms of h (shared-memory counts, then one global atomic per
// non-empty bin); the last block to arrive writes the exclusive digit bases
// and resets the arrival count.  Every thread of a 256-thread block calls it.
template <int ITEMS>
__device__ void os_block_hist(const uint32_t (&key)[ITEMS], unsigned valid, OsHist h) {
    __shared__ uint32_t sh[4][256];
    __shared__ uint32_t ws[8];
    __shared__ bool last;
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        if (!((valid >> r) & 1u)) continue;
#pragma unroll
        for (int d = 0; d < 4; ++d) atomicAdd(&sh[d][(key[r] >> (8 * d)) & 0xFFu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x)
        if ((&sh[0][0])[i]) atomicAdd(&h.hist[i], (&sh[0][0])[i]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(h.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // exclusive scan of each digit histogram (thread = bin)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = 0; d < 4; ++d) {
        const uint32_t v = __ldcg(&h.hist[d * 256 + threadIdx.x]);
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; ++w) pre += ws[w];
        h.base[d * 256 + threadIdx.x] = pre + x - v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *h.counter = 0u;
}

// The look-back status words of tile `tile` for the four passes to zero
// (every thread of a 256-thread block calls it).
__device__ __forceinline__ void os_clear_status(const OsHist &h, int64_t tile) {
#pragma unroll
    for (int d = 0; d < 4; ++d) h.status[((int64_t)d * h.ntiles + tile) * 256 + threadIdx.x] = 0u;
}

}  // namespace bgl
