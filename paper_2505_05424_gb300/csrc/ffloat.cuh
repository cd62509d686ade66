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

// host or device: split a double into (hi, lo) floats
__host__ __device__ inline float2 ff_from_double(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// exact product of two floats as an ff (TwoProd via FMA)
__device__ __forceinline__ float2 two_prod(float a, float b) {
  const float p = a * b;
  return make_float2(p, fmaf(a, b, -p));
}

// ff * ff
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return quick_two_sum(p, e);
}

// ff^2
__device__ __forceinline__ float2 ff_sqr(float2 a) {
  const float p = a.x * a.x;
  float e = fmaf(a.x, a.x, -p);
  e = fmaf(2.f * a.x, a.y, e);
  return quick_two_sum(p, e);
}

// sqrt of a non-negative ff: FP32 root plus one Newton correction
__device__ __forceinline__ float2 ff_sqrt(float2 a) {
  if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
  const float s = sqrtf(a.x);
  const float2 s2 = two_prod(s, s);
  const float r = ((a.x - s2.x) - s2.y) + a.y;   // a - s^2, small
  return quick_two_sum(s, r / (2.f * s));
}

// ff / ff (b != 0): FP32 quotient plus one correction
__device__ __forceinline__ float2 ff_div(float2 a, float2 b) {
  const float q1 = a.x / b.x;
  const float2 p = ff_mul(make_float2(q1, 0.f), b);
  const float2 r = ff_add(a, ff_neg(p));
  const float q2 = r.x / b.x;
  return quick_two_sum(q1, q2);
}

// ff / float
__device__ __forceinline__ float2 ff_div_f(float2 a, float b) {
  const float q1 = a.x / b;
  const float2 p = two_prod(q1, b);
  const float r = ((a.x - p.x) - p.y) + a.y;
  return quick_two_sum(q1, r / b);
}

// a <= b for ff values
__device__ __forceinline__ bool ff_le(float2 a, float2 b) {
  return a.x < b.x || (a.x == b.x && a.y <= b.y);
}

__device__ __forceinline__ float ff_round(float2 a) { return a.x + a.y; }

// Projection onto the second-order cone {y_0 >= |ybar|} (eq. (app-proj)) of a
// two-float input.  The input of the ALM projection is dominated by -beta/sigma,
// often 10^2 - 10^3 times the O(1) point it projects to, so the tests and the
// boundary value (y_0 + |ybar|)/2 cancel: |ybar| and that sum are formed in
// two-float arithmetic (~2^-44 relative).  The boundary direction ybar/|ybar| only
// scales the O(1) result, so it is taken in FP32: every output component is then
// within a few FP32 ulps of its own (O(1)) value, the precision it is stored in.
// Case order: y if |ybar| <= y_0; 0 if |ybar| <= -y_0; else the boundary formula.
template <int K>
__device__ __forceinline__ void ff_proj_soc(float2* y) {
  // |ybar|^2: exact squares of the high parts summed with TwoSum, the rounding
  // errors and the cross terms 2 hi lo collected in one FP32 correction (all
  // terms are non-negative, so the compensated sum is accurate to ~2^-44)
  float sh = 0.f, sc = 0.f;
#pragma unroll
  for (int j = 1; j < K; ++j) {
    const float h = y[j].x;
    const float p = h * h;
    const float e = fmaf(2.f * h, y[j].y, fmaf(h, h, -p));
    const float2 t = two_sum(sh, p);
    sh = t.x;
    sc += t.y + e;
  }
  const float2 nb = ff_sqrt(quick_two_sum(sh, sc));
  if (ff_le(nb, y[0])) return;
  if (ff_le(nb, ff_neg(y[0]))) {
#pragma unroll
    for (int j = 0; j < K; ++j) y[j] = make_float2(0.f, 0.f);
    return;
  }
  const float2 sum = ff_add(y[0], nb);
  const float2 a = make_float2(0.5f * sum.x, 0.5f * sum.y);
  const float scale = (a.x + a.y) / nb.x;
  y[0] = a;
#pragma unroll
  for (int j = 1; j < K; ++j) y[j] = make_float2(scale * y[j].x, 0.f);
}

}  // namespace dot
