// packed.cuh -- a pair of FP32 lanes evaluated by Blackwell's packed FP32
// instructions (two FMAs, adds or multiplies per instruction), so the
// per-node arithmetic of rlbm_device.cuh runs for two nodes at once.  Only
// + - * and fused multiply-add are packed; reciprocals, square roots and
// comparisons act lane by lane.
#pragma once

#include "rlbm_device.cuh"

namespace rlbk {

struct pf2 {
    float2 v;
    __device__ __forceinline__ pf2() {}
    __device__ __forceinline__ pf2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ pf2(double a) : v(make_float2((float)a, (float)a)) {}
    __device__ __forceinline__ pf2(int a) : v(make_float2((float)a, (float)a)) {}
    __device__ __forceinline__ pf2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit pf2(float2 x) : v(x) {}
};

template <>
struct is_f32_lane<pf2> : std::true_type {};

__device__ __forceinline__ pf2 operator+(pf2 a, pf2 b) { return pf2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ pf2 operator-(pf2 a, pf2 b) {
    return pf2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
}
__device__ __forceinline__ pf2 operator*(pf2 a, pf2 b) { return pf2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ pf2 fmadd(pf2 a, pf2 b, pf2 c) { return pf2(__ffma2_rn(a.v, b.v, c.v)); }

// The rounded single operations of the double-float refinement
// (rlbm_device.cuh): the packed intrinsics are never contracted.
__device__ __forceinline__ pf2 xadd(pf2 a, pf2 b) { return a + b; }
__device__ __forceinline__ pf2 xsub(pf2 a, pf2 b) { return a - b; }
__device__ __forceinline__ pf2 xmul(pf2 a, pf2 b) { return a * b; }
__device__ __forceinline__ pf2 xfma(pf2 a, pf2 b, pf2 c) { return fmadd(a, b, c); }

__device__ __forceinline__ pf2 recip(pf2 x) { return pf2(__frcp_rn(x.v.x), __frcp_rn(x.v.y)); }
__device__ __forceinline__ pf2 fast_recip(pf2 x) { return pf2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }
__device__ __forceinline__ pf2 sqrt_(pf2 x) { return pf2(sqrtf(x.v.x), sqrtf(x.v.y)); }
__device__ __forceinline__ pf2 fast_rsqrt(pf2 x) { return pf2(rsqrt_approx(x.v.x), rsqrt_approx(x.v.y)); }
__device__ __forceinline__ pf2 absval(pf2 x) { return pf2(fabsf(x.v.x), fabsf(x.v.y)); }

// Lane-wise comparison; !mask is true only when the comparison fails in
// both lanes (a loop over the pair runs until both nodes are done).
struct pmask {
    bool a, b;
};
__device__ __forceinline__ pmask operator>(pf2 x, pf2 y) { return pmask{x.v.x > y.v.x, x.v.y > y.v.y}; }
__device__ __forceinline__ bool operator!(pmask m) { return !m.a && !m.b; }

}  // namespace rlbk
