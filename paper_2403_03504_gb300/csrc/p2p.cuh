// Pair kernel of the direct repulsion sum (Section 3.2), shared by the
// exact comparator and the near field of the FMM.
#pragma once

namespace bgl {

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed FP32 pairs (two lanes of one 64-bit register, f32x2 instructions):
// one instruction applies the same operation to two sources.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f2x v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
    f2x d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Target (zx, zy) = (x, x), (y, y) against the two sources (qx, qy, qm):
//   f += m_j (z - z_j) / (|z - z_j|^2 + 1e-30)
// A coincident pair (the target itself) has dx = dy = 0 and adds exactly 0;
// for any other pair of FP32 points the 1e-30 shift is far below one
// rounding of r^2.  Padding sources carry m = 0 and finite coordinates.
__device__ __forceinline__ void p2p_pair2(f2x zx, f2x zy, f2x qx, f2x qy, f2x qm, f2x &fx, f2x &fy) {
    const f2x eps = 0x0DA24260'0DA24260ull;   // 1e-30f in both halves
    const f2x dx = sub2(zx, qx), dy = sub2(zy, qy);
    const f2x r2 = fma2(dx, dx, fma2(dy, dy, eps));
    float a, b;
    upk2(r2, a, b);
    const f2x w = mul2(qm, pk2(rcp_approx(a), rcp_approx(b)));
    fx = fma2(w, dx, fx);
    fy = fma2(w, dy, fy);
}

}  // namespace bgl
