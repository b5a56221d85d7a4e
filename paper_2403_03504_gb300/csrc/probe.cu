// Throughput probes behind the ALU roofline of the pair kernels (the
// all-pairs repulsion of Section 3.2, exact and FMM near field).
//
// Four kernels, each one 1,024-thread block per SM running eight
// independent chains per thread, timed by clock64() inside the block, so
// the rates come out per SM clock whatever the clock frequency was:
//   0  FP32 pipe: fmaf chains                       -> FP32 lanes / clk / SM
//   1  MUFU: chains x <- rcp.approx(x) + 0.5 (the add keeps the chain from
//      being an involution that the compiler may fold away; it runs on the
//      FP32 pipe at 1/8 of that pipe's rate)  -> reciprocals / clk / SM
//   2  the pair itself (p2p_pair: 7 FP32 operations and one reciprocal)
//      on register-resident sources                 -> pairs / clk / SM
//   3  two pairs at a time (p2p_pair2: 7 packed FP32x2 operations and two
//      reciprocals, the source broadcast into both halves) -> pairs / clk / SM
// The pair rates are the ceilings of the near-field and exact kernels' inner
// loops without their shared-memory loads and loop control.
#include <algorithm>
#include <vector>

#include "bgl_internal.cuh"
#include "p2p.cuh"

namespace bgl {

namespace {

constexpr int PROBE_THREADS = 1024;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_ITERS = 4096;

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS, 1) probe_kernel(int iters, float seed, float *sink,
                                                                 long long *cycles) {
    float a[PROBE_CHAINS], b[PROBE_CHAINS];
    float2 ga[PROBE_CHAINS], gb[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) {
        a[k] = seed + 1e-3f * (float)(k + 1) + 1e-6f * (float)threadIdx.x;
        b[k] = seed - 1e-3f * (float)(k + 1);
        ga[k] = make_float2(a[k], b[k]);
        gb[k] = make_float2(b[k], a[k]);
    }
    // the chains start after the first clock read and end before the second
    // by data dependence: their inputs take a term of the first clock value
    // (zero in practice, unknown to the compiler), and their sum is stored to
    // shared memory before the barrier that precedes the second read
    __shared__ float red[32];
    __syncthreads();
    const long long t0 = clock64();
    const float z = (float)(t0 >> 62);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) {
        a[k] += z;
        b[k] += z;
        ga[k].x += z;
        gb[k].y += z;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) {
            if (KIND == 0) {
                a[k] = fmaf(a[k], 0.9999f, 1e-4f);
            } else if (KIND == 1) {
                a[k] = rcp_approx(a[k]) + 0.5f;   // converges to (1 + sqrt(17)) / 4
            } else if (KIND == 2) {
                // the source follows the chain's own sums, so every pair
                // depends on the previous one of its chain
                const float4 q = make_float4(a[k], b[k], 1.0f, 0.f);
                p2p_pair(seed, -seed, q, a[k], b[k]);
            } else {
                const float4 q = make_float4(ga[k].x, gb[k].y, 1.0f, 0.f);
                p2p_pair2(make_float2(-seed, -1.5f * seed), make_float2(seed, 0.5f * seed), q, ga[k], gb[k]);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += KIND == 3 ? (ga[k].x + ga[k].y) + (gb[k].x + gb[k].y) : a[k] + b[k];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < PROBE_THREADS / 32; ++w) tot += red[w];
        if (tot == 1234.5f) sink[0] = tot;   // keeps the chains live
    }
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int KIND>
double probe_rate(bgl_ctx *c, int nsm, float *sink, long long *cyc) {
    cudaStream_t s = c->stream;
    // warm-up launch, then the measured one
    for (int rep = 0; rep < 2; ++rep) {
        probe_kernel<KIND><<<nsm, PROBE_THREADS, 0, s>>>(PROBE_ITERS, 1.25f, sink, cyc);
        BGL_LAUNCH_CHECK();
    }
    std::vector<long long> h(nsm);
    BGL_CUDA(cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * nsm, cudaMemcpyDeviceToHost, s));
    BGL_CUDA(cudaStreamSynchronize(s));
    std::sort(h.begin(), h.end());
    const double ops = (double)PROBE_THREADS * PROBE_ITERS * PROBE_CHAINS * (KIND == 3 ? 2 : 1);
    return ops / (double)std::max<long long>(h[nsm / 2], 1);   // median block
}

}  // namespace

void peak_probe(bgl_ctx *c, double *out) {
    const int nsm = c->num_sms;
    DevBuf<float> sink(c->alloc, 1);
    DevBuf<long long> cyc(c->alloc, nsm);
    out[0] = probe_rate<0>(c, nsm, sink.p, cyc.p);
    out[1] = probe_rate<1>(c, nsm, sink.p, cyc.p);
    out[2] = probe_rate<2>(c, nsm, sink.p, cyc.p);
    out[3] = (double)nsm;
    out[4] = probe_rate<3>(c, nsm, sink.p, cyc.p);
}

}  // namespace bgl
