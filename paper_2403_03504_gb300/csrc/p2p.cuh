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

}  // namespace bgl
