// Device pieces shared by the Kamada-Kawai kernels (Section 3.1) and the
// assembly of component layouts (Section 4): the SplitMix64 generator of
// the initial positions and the safeguarded 2x2 Newton-Raphson step.
#pragma once
#include <cstdint>

namespace bgl {

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

// hardware reciprocal and square root (one MUFU operation each, about one
// rounding of error): the step below is a safeguarded Newton move whose
// rounding the sweeps do not amplify
__device__ __forceinline__ float kk_rcp(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float kk_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// Safeguarded Newton-Raphson step (Section 3.1) in FP32: with
// H = l1 P1 + l2 P2 (l1 >= l2, P1 + P2 = I), delta = -(P1 g / e1 + P2 g / e2)
// where e_i = l_i for positive curvature and max(|l_i|, 0.1 max|l|) otherwise;
// steps longer than l are shortened to l.  Returns false for H = 0.
__device__ __forceinline__ bool kk_step(float gx, float gy, float a, float b, float c, float l, float *dx,
                                        float *dy) {
    // positive definite with both eigenvalues above 1e-12 of the larger (tr
    // > 0 and det > 4e-12 tr^2 imply it: l2 = det / l1 > 4e-12 tr^2 / (2 tr)
    // >= 1e-12 l1 since l1 <= 2 tr): then e_i = l_i and the step is -H^-1 g
    const float tr2 = a + c;
    const float det = fmaf(a, c, -b * b);
    if (tr2 > 0.f && det > 1e-12f * tr2 * tr2) {
        const float id = kk_rcp(det);
        float sx = -(c * gx - b * gy) * id;
        float sy = -(a * gy - b * gx) * id;
        const float len2 = fmaf(sx, sx, sy * sy);
        if (len2 > l * l) {
            const float sc = l * rsqrtf(len2);
            sx *= sc;
            sy *= sc;
        }
        *dx = sx;
        *dy = sy;
        return true;
    }
    const float h = 0.5f * (a - c);
    const float dd = kk_sqrt(fmaf(h, h, b * b));
    const float tr = 0.5f * (a + c);
    const float l1 = tr + dd, l2 = tr - dd;
    const float big = fmaxf(fabsf(l1), fabsf(l2));
    if (big == 0.0f) return false;
    const float fl = 0.1f * big;
    const float e1 = l1 > 1e-12f * big ? l1 : fmaxf(fabsf(l1), fl);
    const float e2 = l2 > 1e-12f * big ? l2 : fmaxf(fabsf(l2), fl);
    float sx, sy;
    const float ie1 = kk_rcp(e1), ie2 = kk_rcp(e2);
    if (dd == 0.0f) {
        sx = -gx * ie1;
        sy = -gy * ie1;
    } else {
        const float i2d = kk_rcp(2.0f * dd);
        const float p1x = ((h + dd) * gx + b * gy) * i2d;
        const float p1y = (b * gx + (dd - h) * gy) * i2d;
        sx = -(p1x * ie1 + (gx - p1x) * ie2);
        sy = -(p1y * ie1 + (gy - p1y) * ie2);
    }
    const float len2 = sx * sx + sy * sy;
    if (len2 > l * l) {
        const float sc = l * rsqrtf(len2);
        sx *= sc;
        sy *= sc;
    }
    *dx = sx;
    *dy = sy;
    return true;
}

}  // namespace bgl
