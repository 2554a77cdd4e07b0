// Lane arithmetic of the step kernels (sm_103a).
//
// The per-node arithmetic of the method (steps 1-9 of Section III.B) is written once,
// over a "lane" type V: one node per value (float, double) or two nodes per value
// (float2, the paired step kernel, whose float work runs as packed f32x2 instructions:
// one issue slot for the same operation on two nodes).  Every operation below rounds
// exactly once and is never contracted or reassociated by the compiler (the _rn
// intrinsics), so a node gets the same bits whichever lane type carried it: the paired
// kernel, the one-node kernels, the bulk-copy kernels and the batch kernel agree bit for
// bit.  Where the arithmetic wants a fused multiply-add it says so (vfma).
//
// Reciprocal and logarithm work per lane: the exact library forms in double, the
// hardware approximations in float (below), well inside the FP32 error budget.
#pragma once

#include <cuda_runtime.h>

namespace fmlbm {

template <typename V> struct LaneTraits;
template <> struct LaneTraits<float> { using E = float; static constexpr int n = 1; };
template <> struct LaneTraits<double> { using E = double; static constexpr int n = 1; };
template <> struct LaneTraits<float2> { using E = float; static constexpr int n = 2; };

template <typename V> using LaneE = typename LaneTraits<V>::E;

// broadcast of a scalar to every lane
template <typename V> __device__ __forceinline__ V vbc(LaneE<V> c);
template <> __device__ __forceinline__ float vbc<float>(float c) { return c; }
template <> __device__ __forceinline__ double vbc<double>(double c) { return c; }
template <> __device__ __forceinline__ float2 vbc<float2>(float c) { return make_float2(c, c); }

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }

__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ double vneg(double a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

// a - b = a + (-b) exactly (negation is exact)
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }

__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// a * b + c, rounded once
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Per-lane reciprocal and natural logarithm.  In float: the hardware approximations of the
// PTX instructions rcp.approx and lg2.approx (documented maximum errors: 1 ulp for the
// reciprocal, 2^-22.6 absolute for the base-2 logarithm of the mantissa), then
// ln x = log2(x) ln 2 with one rounded product.  Written as instructions rather than
// through the fast-math library forms so that the compiler cannot fold them into a
// neighbouring operation differently in different kernels (a product with an approximate
// reciprocal becomes an approximate division, for example), which would break the
// bit-identity of the kernels.  Arguments are never denormal here (densities, 1 - beta and
// the like), so the flush-to-zero forms lose nothing.
__device__ __forceinline__ float srcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double srcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float sln(float x) {
    float l2;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(x));
    return __fmul_rn(l2, 0.693147180559945309f);  // ln 2
}
__device__ __forceinline__ double sln(double x) { return log(x); }
__device__ __forceinline__ float slog1p(float x) { return log1pf(x); }
__device__ __forceinline__ double slog1p(double x) { return log1p(x); }

__device__ __forceinline__ float vrcp(float x) { return srcp(x); }
__device__ __forceinline__ double vrcp(double x) { return srcp(x); }
__device__ __forceinline__ float2 vrcp(float2 x) { return make_float2(srcp(x.x), srcp(x.y)); }
__device__ __forceinline__ float vln(float x) { return sln(x); }
__device__ __forceinline__ double vln(double x) { return sln(x); }
__device__ __forceinline__ float2 vln(float2 x) { return make_float2(sln(x.x), sln(x.y)); }
__device__ __forceinline__ float vlog1p(float x) { return slog1p(x); }
__device__ __forceinline__ double vlog1p(double x) { return slog1p(x); }
__device__ __forceinline__ float2 vlog1p(float2 x) { return make_float2(slog1p(x.x), slog1p(x.y)); }

// lane k of a value (k < LaneTraits<V>::n) and its assignment
__device__ __forceinline__ float lane(float v, int) { return v; }
__device__ __forceinline__ double lane(double v, int) { return v; }
__device__ __forceinline__ float lane(float2 v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ void set_lane(float& v, int, float s) { v = s; }
__device__ __forceinline__ void set_lane(double& v, int, double s) { v = s; }
__device__ __forceinline__ void set_lane(float2& v, int k, float s) {
    if (k == 0) v.x = s;
    else v.y = s;
}

}  // namespace fmlbm
