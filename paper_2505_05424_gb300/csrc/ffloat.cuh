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

// ---- packed pairs ---------------------------------------------------------
// sm_100-class GPUs execute add/sub/mul/fma on two FP32 lanes in one instruction
// (.f32x2), each lane an ordinary IEEE round-to-nearest operation.  A float2 here
// is such a lane pair; ff2 holds two two-float numbers, (h.x + l.x) and
// (h.y + l.y).  Every ff2 operation computes, lane by lane, exactly what the
// scalar operation of the same name above computes.

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0, %1}, rc;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0, %1}, rc;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0, %1}, rc;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

struct ff2 {
  float2 h, l;
};

__device__ __forceinline__ ff2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 bb = sub2(s, a);
  const float2 e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
  return ff2{s, e};
}
__device__ __forceinline__ ff2 quick_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return ff2{s, sub2(b, sub2(s, a))};
}
// lane-wise ff_add
__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) {
  ff2 s = two_sum2(a.h, b.h);
  s.l = add2(s.l, add2(a.l, b.l));
  return quick_two_sum2(s.h, s.l);
}
// lane-wise ff_add_f
__device__ __forceinline__ ff2 ff2_add_f(ff2 a, float2 b) {
  ff2 s = two_sum2(a.h, b);
  s.l = add2(s.l, a.l);
  return quick_two_sum2(s.h, s.l);
}
// lane-wise two_prod: the rounding error of each product by one FMA
__device__ __forceinline__ ff2 two_prod2(float2 a, float2 b) {
  const float2 p = mul2(a, b);
  return ff2{p, make_float2(fmaf(a.x, b.x, -p.x), fmaf(a.y, b.y, -p.y))};
}
__device__ __forceinline__ ff2 ff2_neg(ff2 a) {
  return ff2{make_float2(-a.h.x, -a.h.y), make_float2(-a.l.x, -a.l.y)};
}
// the two lanes of an ff2 as scalar two-floats, and back
__device__ __forceinline__ float2 ff2_lane0(ff2 a) { return make_float2(a.h.x, a.l.x); }
__device__ __forceinline__ float2 ff2_lane1(ff2 a) { return make_float2(a.h.y, a.l.y); }
__device__ __forceinline__ ff2 ff2_pack(float2 a, float2 b) {
  return ff2{make_float2(a.x, b.x), make_float2(a.y, b.y)};
}

// ---- cheaper forms used by the fused cone kernel ----------------------------

// ff / float given r ~ 1/b (a few ulps suffice): FP32 quotient a.x * r plus one
// correction from the exact remainder, as ff_div_f without its two divisions.
__device__ __forceinline__ float2 ff_div_f_r(float2 a, float b, float r) {
  const float q1 = a.x * r;
  const float2 p = two_prod(q1, b);
  const float rem = ((a.x - p.x) - p.y) + a.y;
  return quick_two_sum(q1, rem * r);
}

// sqrt of a non-negative ff from the FP32 reciprocal square root: s = a r with
// r ~ 1/sqrt(a), then one Newton correction (a - s^2) r / 2 from the exact square,
// accurate to ~2^-44 relative.  *rinv receives r (~1/sqrt(a) to a few ulps).
__device__ __forceinline__ float2 ff_sqrt_r(float2 a, float* rinv) {
  if (!(a.x > 0.f)) {
    *rinv = 0.f;
    return make_float2(0.f, 0.f);
  }
  const float r = rsqrtf(a.x);
  const float s = a.x * r;
  const float2 s2 = two_prod(s, s);
  const float rem = ((a.x - s2.x) - s2.y) + a.y;
  *rinv = r;
  return quick_two_sum(s, rem * (0.5f * r));
}

// Running sum of two-float terms with one normalisation at the end: the high parts
// are added by TwoSum (each rounding error kept exactly), the low parts and those
// errors in one FP32 correction.  Same accuracy class as a chain of ff_add.
struct ff_acc {
  float h, c;
};
__device__ __forceinline__ ff_acc acc_init(float2 a) { return ff_acc{a.x, a.y}; }
__device__ __forceinline__ void acc_add(ff_acc& s, float2 b) {
  const float2 t = two_sum(s.h, b.x);
  s.h = t.x;
  s.c += t.y + b.y;
}
__device__ __forceinline__ void acc_add_f(ff_acc& s, float b) {
  const float2 t = two_sum(s.h, b);
  s.h = t.x;
  s.c += t.y;
}
// + b * x for a two-float b and an FP32 x: the exact product of the high part by
// TwoProd, the low part's product into the correction
__device__ __forceinline__ void acc_add_mul(ff_acc& s, float2 b, float x) {
  const float p = b.x * x;
  const float e = fmaf(b.y, x, fmaf(b.x, x, -p));
  const float2 t = two_sum(s.h, p);
  s.h = t.x;
  s.c += t.y + e;
}
__device__ __forceinline__ float2 acc_get(const ff_acc& s) { return quick_two_sum(s.h, s.c); }

// Projection onto {y_0 >= |ybar|} (eq. (app-proj)) of a K = 10 cone held as five
// lane pairs: P[0] = (y_0, y_9), P[k] = (y_{2k-1}, y_{2k}) for k = 1..4.  The same
// method as ff_proj_soc (two-float |ybar|, FP32 boundary direction), with |ybar|^2
// summed in two lanes, the square root from rsqrt and the boundary scale from its
// reciprocal instead of divisions.
__device__ __forceinline__ void ff2_proj_soc10(ff2* P) {
  float2 sh = make_float2(0.f, 0.f), sc = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const float2 h = P[k].h;
    const float2 p = mul2(h, h);
    const float2 e0 = make_float2(fmaf(h.x, h.x, -p.x), fmaf(h.y, h.y, -p.y));
    const float2 e = fma2(add2(h, h), P[k].l, e0);
    const ff2 t = two_sum2(sh, p);
    sh = t.h;
    sc = add2(sc, add2(t.l, e));
  }
  // y_9 and the two lanes
  const float h9 = P[0].h.y;
  const float p9 = h9 * h9;
  const float e9 = fmaf(2.f * h9, P[0].l.y, fmaf(h9, h9, -p9));
  const float2 t1 = two_sum(sh.x, sh.y);
  const float2 t2 = two_sum(t1.x, p9);
  const float corr = ((sc.x + sc.y) + (t1.y + t2.y)) + e9;
  float r;
  const float2 nb = ff_sqrt_r(quick_two_sum(t2.x, corr), &r);
  const float2 y0 = ff2_lane0(P[0]);
  if (ff_le(nb, y0)) return;
  if (ff_le(nb, ff_neg(y0))) {
#pragma unroll
    for (int k = 0; k < 5; ++k) P[k] = ff2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    return;
  }
  const float2 sum = ff_add(y0, nb);
  const float2 a = make_float2(0.5f * sum.x, 0.5f * sum.y);
  const float scale = (a.x + a.y) * r;
  const float2 sc2 = make_float2(scale, scale), zero2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 1; k <= 4; ++k) P[k] = ff2{mul2(sc2, P[k].h), zero2};
  P[0] = ff2{make_float2(a.x, scale * P[0].h.y), make_float2(a.y, 0.f)};
}

}  // namespace dot
