// Element arithmetic of the generated cores and the adjustments, for one line (float) or
// two lines processed together (float2, with the packed FP32x2 instructions of sm_100+:
// one instruction does the operation for both lines).
#pragma once

#include <cuda_runtime.h>

__device__ __forceinline__ float vzero(float) { return 0.f; }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vmul(float c, float a) { return c * a; }
// c1 * a + c2 * b
__device__ __forceinline__ float vmac(float c1, float a, float c2, float b) { return fmaf(c1, a, c2 * b); }
// a * b + c with a, b, c of the element type (runtime coefficients)
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ float2 vzero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }
__device__ __forceinline__ float2 vneg(float2 a) { return __fmul2_rn(make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vmul(float c, float2 a) { return __fmul2_rn(make_float2(c, c), a); }
__device__ __forceinline__ float2 vmac(float c1, float2 a, float c2, float2 b) {
  return __ffma2_rn(make_float2(c1, c1), a, __fmul2_rn(make_float2(c2, c2), b));
}
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// (c.x a + d.x b, c.y a + d.y b) for scalars a, b broadcast to both halves: the first and last
// steps of the packed 64-point cores, one FP32x2 multiply and one FP32x2 FMA.
__device__ __forceinline__ float2 vpre2(float a, float b, float2 c, float2 d) {
  return __ffma2_rn(make_float2(b, b), d, __fmul2_rn(make_float2(a, a), c));
}
