// Pair kernel of the direct repulsion sum (Section 3.2), shared by the
// exact comparator and the near field of the FMM.
#pragma once

namespace bgl {

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One pair of the direct sum: f += m_j (z - z_j) / (|z - z_j|^2 + 1e-30) for
// the target (zx, zy) and the source q = (x_j, y_j, m_j, .).  A coincident
// pair (the target itself) has dx = dy = 0 and adds exactly 0; for any other
// pair of FP32 points the 1e-30 shift is far below one rounding of r^2.
// Costs 7 FP32 operations and one MUFU reciprocal.
__device__ __forceinline__ void p2p_pair(float zx, float zy, const float4 &q, float &fx, float &fy) {
    const float dx = zx - q.x, dy = zy - q.y;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, 1e-30f));
    const float w = q.z * rcp_approx(r2);
    fx = fmaf(w, dx, fx);
    fy = fmaf(w, dy, fy);
}

// Two targets against one source with the packed FP32x2 instructions of
// sm_100 and later (one issue slot for two lanes' worth of add, multiply or
// FMA): 7 packed operations and two reciprocals for two pairs.  The targets
// come negated (nzx = -zx) and the accumulators hold the negated sums,
// g += m_j (z_j - z) / (|z_j - z|^2 + 1e-30): each operation is the sign
// mirror of p2p_pair's (round-to-nearest is symmetric in sign), so -g equals,
// bit for bit, what p2p_pair accumulates in the same order.
__device__ __forceinline__ void p2p_pair2(float2 nzx, float2 nzy, const float4 &q, float2 &gx, float2 &gy) {
    const float2 dx = __fadd2_rn(make_float2(q.x, q.x), nzx);
    const float2 dy = __fadd2_rn(make_float2(q.y, q.y), nzy);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, make_float2(1e-30f, 1e-30f)));
    const float2 w = __fmul2_rn(make_float2(q.z, q.z), make_float2(rcp_approx(r2.x), rcp_approx(r2.y)));
    gx = __ffma2_rn(w, dx, gx);
    gy = __ffma2_rn(w, dy, gy);
}

}  // namespace bgl
