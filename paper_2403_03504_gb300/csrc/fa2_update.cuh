// Device pieces of the ForceAtlas2 update (Section 3.2) shared by the
// iteration kernels of fa2.cu and the FMM's fused combine and update
// kernels (fmm.cu), so both apply the same formulas:
//   swing  |F_t - F_{t-1}|, traction |F_t + F_{t-1}| (weighted by m and the
//          traction halved in variant 1);
//   s_G = min(tau trc / swg, 1.5 s_G) (1.5 s_G when swg = 0);
//   s_n = ks s_G / (1 + s_G sqrt(swing_n)), at most ksmax / |F_t(n)|;
//   p_n += s_n F_t(n).
#pragma once

namespace bgl {

// swing and traction terms of one node
__device__ __forceinline__ void fa2_swing_terms(float2 F, float2 P, float m, int variant, float &sw, float &tr) {
    const float s = sqrtf((F.x - P.x) * (F.x - P.x) + (F.y - P.y) * (F.y - P.y));
    const float u = sqrtf((F.x + P.x) * (F.x + P.x) + (F.y + P.y) * (F.y + P.y));
    if (variant == 1) {
        sw = m * s;
        tr = 0.5f * m * u;
    } else {
        sw = s;
        tr = u;
    }
}

// the global speed after an iteration with sums swg, trc
__device__ __forceinline__ double fa2_global_speed(double swg, double trc, double g, double tau) {
    double s_new = swg > 0.0 ? tau * trc / swg : 1.5 * g;
    if (s_new > 1.5 * g) s_new = 1.5 * g;
    return s_new;
}

// the node's new position
__device__ __forceinline__ float2 fa2_move(float2 p, float2 F, float2 P, float g, float ks, float ksmax) {
    const float sw = sqrtf((F.x - P.x) * (F.x - P.x) + (F.y - P.y) * (F.y - P.y));
    float s = ks * g / (1.f + g * sqrtf(sw));
    const float fn = sqrtf(F.x * F.x + F.y * F.y);
    if (fn > 0.f && s > ksmax / fn) s = ksmax / fn;
    p.x += s * F.x;
    p.y += s * F.y;
    return p;
}

}  // namespace bgl
