// Two FP32 values in one register pair for the packed FP32 instructions of
// sm_100+ (fma/mul/add .f32x2): one instruction for both halves.  Used by the
// jet algebra of the tensor-core epilogues (two points per pair) and by the
// FP32 SIMT jet GEMMs (two channels per pair).
#pragma once

#include <cuda_runtime.h>

namespace jet {

struct f2 {
  float2 v;
  __device__ __forceinline__ f2() {}
  __device__ __forceinline__ f2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit f2(float2 x) : v(x) {}
};
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 jfma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }

}  // namespace jet
