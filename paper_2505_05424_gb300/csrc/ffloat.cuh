// ffloat.cuh -- two-float ("float-float") arithmetic: a value is hi + lo with
// |lo| <= ulp(hi)/2, about 48 significant bits, computed with FP32 instructions
// only.  Used for the ALM multipliers and the potential of the mixed path, whose
// per-element updates would otherwise need FP64 instructions (GB300 issues FP64
// FMA at about 1/70 of the FP32 rate).
//
// Error-free transformations: TwoSum (Knuth) and TwoProd via FMA.  No
// reassociation or contraction can change them: they contain no a*b+c patterns
// except the explicit fmaf.
#pragma once
#include <cuda_runtime.h>

namespace dot {

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return make_float2(s, e);
}

// (hi, lo) renormalised so that hi = fl(hi + lo).
__device__ __forceinline__ float2 quick_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return make_float2(s, e);
}

// ff + float
__device__ __forceinline__ float2 ff_add_f(float2 a, float b) {
  float2 s = two_sum(a.x, b);
  s.y += a.y;
  return quick_two_sum(s.x, s.y);
}

// ff + ff
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  s.y += a.y + b.y;
  return quick_two_sum(s.x, s.y);
}

__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

// ff * float
__device__ __forceinline__ float2 ff_mul_f(float2 a, float b) {
  const float p = a.x * b;
  float e = fmaf(a.x, b, -p);
  e = fmaf(a.y, b, e);
  return quick_two_sum(p, e);
}

// exact difference of two floats as an ff
__device__ __forceinline__ float2 ff_sub_exact(float a, float b) { return two_sum(a, -b); }

__device__ __forceinline__ double ff_to_double(float2 a) { return (double)a.x + (double)a.y; }

}  // namespace dot
