// k_mixed.cu -- mixed-precision kernels of Algorithm 2 around the fused passes
// (k_fused2d.cu, k_fused3d.cu): line 1 (the b-assembly fused with the warm-start
// residual), the exact-residual step of the Poisson refinement, the multiplier
// rescale after a penalty change, and the stopping measures.
//
// Storage: q and z in FP32; the multipliers as alpha/sigma and beta/sigma and
// the potential phi as two-float pairs (hi, lo); the Poisson scratch in FP32.
// With the multipliers stored divided by sigma, every alpha/sigma and beta/sigma
// of Algorithm 2 is a load, the updates alpha += tau sigma (...) become
// alpha/sigma += tau (...), and a penalty change rescales the stored values once.  Arithmetic is FP32; updates of the
// two-float fields use error-free transformations (ffloat.cuh); the reduction
// tree of the stopping measures is FP64.  Kernels are templated on D so the cone
// (K = 4D + 2 components) lives in registers.
#include <cmath>

#include "dot_internal.cuh"
#include "dot_mixed.cuh"
#include "ffloat.cuh"

namespace dot {
namespace {

constexpr int kThreads = 256;

inline int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// A phi along an axis from the two-float potential, as an unevaluated pair
// (gh, gl): gh + gl = (phi_j - phi_i) / h to ~2^-44 relative.
__device__ __forceinline__ float2 grad_pair(const float2* phi, long long i, long long j, float invh) {
  const float2 a = phi[i], b = phi[j];
  const float2 dh = two_sum(b.x, -a.x);
  const float dl = (b.y - a.y) + dh.y;
  return make_float2(dh.x * invh, dl * invh);
}

// A phi - q with one rounding relative to the (small) difference itself.
__device__ __forceinline__ float grad_minus(float2 g, float q) { return (g.x - q) + g.y; }

constexpr int kMeanBlocks = kBsumParts;   // offset of mean(b) in a slot's bsum

// FP64 sum of a block's per-thread two-float partials into out[blockIdx.x].
__device__ __forceinline__ void block_sum_ff(float2 v, double* out) {
  double d = ff_to_double(v);
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  __shared__ double w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += w[k];
    out[blockIdx.x] = s;
  }
}

// Zero-mode partial sums per slot: one per block of k_sum_b.
inline int bsum_blocks(const Geo& g) {
  const long long nn = (long long)(g.T + 1) * g.P;
  long long b = (nn + kThreads - 1) / kThreads;
  return (int)(b < kBsumParts ? (b < 1 ? 1 : b) : kBsumParts);
}

// Sum of b (per-block partials, two-float per thread, FP64 per block): the exact
// zero mode of the right-hand side.  An FP32 DCT of a field with a large mean
// leaks O(u_32 * mean * sqrt(n)) into the other coefficients; removing the exact
// mean from the refinement residual lets the correction solve remove that leak.
// The refined Poisson operator (dot_poisson and the allocation-free entry point)
// uses it.
__global__ void k_sum_b(Geo g, MxFields fb) {
  const int slot = blockIdx.y;
  if (!fb.sp[slot].active) return;
  const MxFields f = slot_view(fb, g, slot);
  const long long n = (long long)(g.T + 1) * g.P;
  const float* b = f.b;
  const float* blo = f.blo;
  double* partials = f.bsum;
  float2 acc = make_float2(0.f, 0.f);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc = ff_add(acc, make_float2(b[i], blo[i]));
  block_sum_ff(acc, partials);
}

// Refinement residual r = b - mean(b) - A^*A phi1, with A^*A phi1 accumulated
// exactly in two-float arithmetic (each neighbour difference by TwoSum; 1/h^2 is
// an integer) and mean(b) from the FP64 partial sums.
// mean(b) from the per-block partial sums, once, as a two-float in bsum[kMeanBlocks]
__global__ void k_mean_b(Geo g, MxFields fb, int nparts) {
  const int slot = blockIdx.x;
  if (!fb.sp[slot].active) return;
  double* bsum = slot_view(fb, g, slot).bsum;
  const long long n = (long long)(g.T + 1) * g.P;
  __shared__ double sh[kThreads];
  double v = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) v += bsum[k];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = sh[0] / (double)n;
    const float hi = (float)m;
    reinterpret_cast<float2*>(bsum + kMeanBlocks)[0] = make_float2(hi, (float)(m - (double)hi));
  }
}

template <int D>
__global__ void k_residual(Geo g, MxFields fb) {
  const int slot = blockIdx.y;
  if (!fb.sp[slot].active) return;
  const MxFields f = slot_view(fb, g, slot);
  const float2 mean = reinterpret_cast<const float2*>(f.bsum + kMeanBlocks)[0];
  const long long n = (long long)(g.T + 1) * g.P;
  const float* x = f.phi1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = plane_of(g, i);
    const long long p = i - (long long)t * g.P;
    const float xi = x[i];
    float2 acc = make_float2(0.f, 0.f);
    {
      float2 s = make_float2(0.f, 0.f);
      if (t >= 1) s = ff_add(s, ff_sub_exact(xi, x[i - g.P]));
      if (t < g.T) s = ff_add(s, ff_sub_exact(xi, x[i + g.P]));
      const float ih = (float)g.invh[0];
      acc = ff_add(acc, ff_mul_f(s, ih * ih));
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int xd = coord(g, p, d);
      const long long st = g.sst[d];
      float2 s = make_float2(0.f, 0.f);
      if (xd >= 1) s = ff_add(s, ff_sub_exact(xi, x[i - st]));
      if (xd <= g.N[d] - 2) s = ff_add(s, ff_sub_exact(xi, x[i + st]));
      const float ih = (float)g.invh[1 + d];
      acc = ff_add(acc, ff_mul_f(s, ih * ih));
    }
    const float2 r = ff_add(make_float2(f.b[i], f.blo[i]), ff_neg(ff_add(acc, mean)));
    f.r[i] = r.x + r.y;
  }
}

// Line 2 warm-started from the previous iteration's potential:
//   r = b - A^*A phi^k,  delta = P(r),  phi^{k+1} = phi^k + delta.
// A^*A phi^k is accumulated from exact two-float neighbour differences of the
// two-float phi^k, so r is exact up to its final rounding to FP32 and the new
// potential carries the FP32 solve's relative error times |phi^{k+1} - phi^k|
// only (the inexact subproblem solves Algorithm 1 admits; phi^0 = 0 makes the
// first step a plain solve).  a - b of two two-float values, unnormalised:
__device__ __forceinline__ float2 ff_diff(float2 a, float2 b) {
  const float2 d = two_sum(a.x, -b.x);
  return make_float2(d.x, d.y + (a.y - b.y));
}

// Lines 1 and 2 fused: b = A^*(q - alpha/sigma) - c/sigma at a node, in
// two-float arithmetic (alpha/sigma and c/sigma are 10-10^3 times the O(1) part
// that survives their cancellation), and at once the warm-start residual
// r = b - A^*A phi^k, so b never reaches memory.  mean(b) is not subtracted: the
// equal masses make sum(b) vanish up to rounding (|sum b| ~ 1e-16 |c| / sigma),
// and the solve drops the zero mode.
template <int D>
__global__ void __launch_bounds__(kThreads, D == 2 ? 4 : 3) k_assemble_residual(Geo g, MxFields fb) {
  const int slot = blockIdx.y;
  // a slot without the assemble flag keeps the residual the fused kernel left in f.r
  if (!fb.sp[slot].active || !fb.sp[slot].assemble) return;
  const float2 isg = fb.sp[slot].isg;
  const MxFields f = slot_view(fb, g, slot);
  const long long n = (long long)(g.T + 1) * g.P;
  const float2* x = f.phi;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = plane_of(g, i);
    const long long p = i - (long long)t * g.P;
    const float ih0 = (float)g.invh[0];
    float2 acc = make_float2(0.f, 0.f);    // b
    float2 lap = make_float2(0.f, 0.f);    // A^*A phi
    const float2 xi = x[i];
    {
      float2 sd = make_float2(0.f, 0.f);
      if (t >= 1) {
        const float2 w = ff_add_f(ff_neg(f.al[0][i - g.P]), f.q[0][i - g.P]);
        acc = ff_add(acc, ff_mul_f(w, ih0));
        sd = ff_add(sd, ff_diff(xi, x[i - g.P]));
      }
      if (t < g.T) {
        const float2 w = ff_add_f(ff_neg(f.al[0][i]), f.q[0][i]);
        acc = ff_add(acc, ff_neg(ff_mul_f(w, ih0)));
        sd = ff_add(sd, ff_diff(xi, x[i + g.P]));
      }
      lap = ff_add(lap, ff_mul_f(sd, ih0 * ih0));
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int xd = coord(g, p, d);
      const float* qd = f.q[1 + d];
      const float2* ad = f.al[1 + d];
      const long long s = g.sst[d];
      const float ih = (float)g.invh[1 + d];
      float2 sd = make_float2(0.f, 0.f);
      if (xd >= 1) {
        const float2 w = ff_add_f(ff_neg(ad[i - s]), qd[i - s]);
        acc = ff_add(acc, ff_mul_f(w, ih));
        sd = ff_add(sd, ff_diff(xi, x[i - s]));
      }
      if (xd <= g.N[d] - 2) {
        const float2 w = ff_add_f(ff_neg(ad[i]), qd[i]);
        acc = ff_add(acc, ff_neg(ff_mul_f(w, ih)));
        sd = ff_add(sd, ff_diff(xi, x[i + s]));
      }
      lap = ff_add(lap, ff_mul_f(sd, ih * ih));
    }
    if (t == 0) acc = ff_add(acc, ff_neg(ff_mul(f.c0[p], isg)));
    if (t == g.T) acc = ff_add(acc, ff_mul(f.c1[p], isg));
    const float2 r = ff_add(acc, ff_neg(lap));
    f.r[i] = r.x + r.y;
  }
}

// After a penalty change sigma_old -> sigma_new: alpha/sigma and beta/sigma of the
// current set times sigma_old / sigma_new (two-float).
template <int D>
__global__ void k_rescale(Geo g, MxFields fb) {
  const int slot = blockIdx.y;
  const SlotParam sp = fb.sp[slot];
  if (!sp.active || (sp.rescale.x == 1.f && sp.rescale.y == 0.f)) return;
  const MxFields f = slot_view(fb, g, slot);
  const long long nn = (long long)(g.T + 1) * g.P, n0 = (long long)g.T * g.P;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long i = i0; i < n0; i += stride) f.al[0][i] = ff_mul(f.al[0][i], sp.rescale);
#pragma unroll
  for (int d = 0; d < D; ++d)
    for (long long i = i0; i < nn; i += stride) f.al[1 + d][i] = ff_mul(f.al[1 + d][i], sp.rescale);
  for (long long i = i0; i < (long long)g.K * n0; i += stride) f.beta[i] = ff_mul(f.beta[i], sp.rescale);
}

// phi^{k+1} = phi^k + delta (delta in phi1).
__global__ void k_phi_add(Geo g, MxFields fb) {
  const int slot = blockIdx.y;
  if (!fb.sp[slot].active) return;
  const long long n = (long long)(g.T + 1) * g.P;
  const MxFields f = slot_view(fb, g, slot);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    f.phi[i] = ff_add_f(f.phi[i], f.phi1[i]);
}

// phi = phi1 + delta as a two-float pair (out is slot-strided like phi).
__global__ void k_combine(Geo g, MxFields fb, float2* __restrict__ out) {
  const int slot = blockIdx.y;
  if (!fb.sp[slot].active) return;
  const long long n = (long long)(g.T + 1) * g.P;
  const MxFields f = slot_view(fb, g, slot);
  const float* __restrict__ phi1 = f.phi1;
  const float* __restrict__ delta = f.b;
  float2* __restrict__ phi = out + slot * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    phi[i] = two_sum(phi1[i], delta[i]);
}

template <int D>
__device__ __forceinline__ void gather_Fq(const Geo& g, float* const* q, long long i, long long p, float* x) {
  x[0] = q[0][i];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int xd = coord(g, p, d);
    const float* qd = q[1 + d];
    const long long s = g.sst[d];
    const bool lo = xd >= 1, hi = xd <= g.N[d] - 2;
    x[1 + 4 * d + 0] = lo ? qd[i - s] : 0.f;
    x[1 + 4 * d + 1] = hi ? qd[i] : 0.f;
    x[1 + 4 * d + 2] = lo ? qd[i + g.P - s] : 0.f;
    x[1 + 4 * d + 3] = hi ? qd[i + g.P] : 0.f;
  }
}

// ---- stopping measures: FP32 terms, per-thread FP32 sums, FP64 tree -----------

#ifndef KKT_MIN_BLOCKS
#define KKT_MIN_BLOCKS 3
#endif
// most blocks per slot of the stopping-measure kernel: one wave of KKT_MIN_BLOCKS
// CTAs on each of the GPU's 152 SMs
constexpr int kKktBlocks = 152 * KKT_MIN_BLOCKS;

__host__ __device__ inline long long kkt_partials_len_slot(const Geo& g) {
  return (long long)(g.D + 2) * kKktBlocks * R_NSLOTS;
}

// Blocks per slot of each stopping-measure kernel (at most kKktBlocks).
inline int kkt_blocks(const Geo& g) {
  const long long nn = (long long)(g.T + 1) * g.P;
  const long long b = (nn + 4 * kThreads - 1) / (4 * kThreads);
  return (int)(b < 1 ? 1 : (b > kKktBlocks ? kKktBlocks : b));
}

__device__ __forceinline__ void block_reduce_store(const float* accf, const double* accd, double* out_row) {
  __shared__ double sh[kThreads / 32][R_NSLOTS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < R_NSLOTS; ++k) {
    double v = (double)accf[k] + accd[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < R_NSLOTS) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += sh[w][threadIdx.x];
    out_row[threadIdx.x] = v;
  }
}

// One node's share of the stopping measures: its cone (t < T), its faces along
// every axis (the face after the node), and the node itself.
template <int D>
__device__ __forceinline__ void kkt_cone(const Geo& g, const MxFields& f, float sg, long long i, long long p,
                                         int use_z, float* acc) {
  constexpr int K = 4 * D + 2;
  const long long n0 = (long long)g.T * g.P;
  const float s_default = 0.70710678118654752f;
  const float ih0 = (float)g.invh[0];
  float x[K - 1];
  gather_Fq<D>(g, f.q, i, p, x);
  const float2 gp = grad_pair(f.phi, i, i + g.P, ih0);
  const float aphi = gp.x + gp.y;
  const float q0 = x[0];
  const float dq = grad_minus(gp, q0);
  acc[R_PRIM] += dq * dq;
  acc[R_APHI] += aphi * aphi;
  acc[R_Q] += q0 * q0;
  float ss = 0.f;
#pragma unroll
  for (int j = 1; j < K - 1; ++j) ss += x[j] * x[j];
  const float om = f.omega ? f.omega[p] : 1.f;
  const float fv = q0 + 0.125f * om * ss;
  const float a0 = sg * (f.al[0][i].x + f.al[0][i].y);
  const float m = fv + a0;
  const float rc = a0 - (m > 0.f ? m : 0.f);
  acc[R_COMP0] += rc * rc;
  acc[R_ALPHA0] += a0 * a0;
  acc[R_F] += fv * fv;
  const float s = f.somega ? f.somega[p] : s_default;
  if (use_z) {
    float r = (f.z[i] - 1.f) + q0;
    acc[R_SOCP] += r * r;
#pragma unroll
    for (int j = 1; j < K - 1; ++j) {
      r = fmaf(-s, x[j], f.z[(long long)j * n0 + i]);
      acc[R_SOCP] += r * r;
    }
    r = (f.z[(long long)(K - 1) * n0 + i] - 1.f) - q0;
    acc[R_SOCP] += r * r;
  }
  const float2 bK = f.beta[(long long)(K - 1) * n0 + i], b0 = f.beta[i];
  const float fbb = sg * ((bK.x - b0.x) + (bK.y - b0.y));
  acc[R_SOCD] += (fbb + a0) * (fbb + a0);
  acc[R_FBB] += fbb * fbb;
}

template <int D>
__device__ __forceinline__ void kkt_face(const Geo& g, const MxFields& f, float sg, int d, long long i, int t,
                                         long long p, float* acc, float2* dual) {
  const long long n0 = (long long)g.T * g.P;
  const float s_default = 0.70710678118654752f;
  const long long s = g.sst[d];
  const float* qd = f.q[1 + d];
  const float2* ad = f.al[1 + d];
  const float2* a0 = f.al[0];
  const int cbase = 1 + 4 * d;
  const float ih = (float)g.invh[1 + d];
  const float2 gp = grad_pair(f.phi, i, i + s, ih);
  const float aphi = gp.x + gp.y;
  const float q = qd[i];
  const float dq = grad_minus(gp, q);
  acc[R_PRIM] += dq * dq;
  acc[R_APHI] += aphi * aphi;
  acc[R_Q] += q * q;
  float den = 0.f, fbb = 0.f;
  const float om_l = f.omega ? f.omega[p] : 1.f, om_r = f.omega ? f.omega[p + s] : 1.f;
  const float s_l = f.somega ? f.somega[p] : s_default, s_r = f.somega ? f.somega[p + s] : s_default;
  if (t <= g.T - 1) {
    den += om_r * a0[i + s].x + om_l * a0[i].x;
    fbb += s_r * f.beta[(long long)(cbase + 0) * n0 + i + s].x + s_l * f.beta[(long long)(cbase + 1) * n0 + i].x;
  }
  if (t >= 1) {
    den += om_r * a0[i - g.P + s].x + om_l * a0[i - g.P].x;
    fbb += s_r * f.beta[(long long)(cbase + 2) * n0 + i - g.P + s].x +
           s_l * f.beta[(long long)(cbase + 3) * n0 + i - g.P].x;
  }
  den *= 0.25f * sg;
  fbb *= sg;
  const float gv = den * q;
  const float a = sg * (ad[i].x + ad[i].y);
  acc[R_COMPD] += (a - gv) * (a - gv);
  acc[R_ALPHAB] += a * a;
  acc[R_G] += gv * gv;
  // dual objective term: each ratio rounded once in FP32, the sum carried as a
  // two-float (no FP64 division on the per-element path)
  if (den > 0.f) *dual = ff_add_f(*dual, -(0.5f * a) * (a / den));
  acc[R_SOCD] += (fbb + a) * (fbb + a);
  acc[R_FBB] += fbb * fbb;
}

// A^*alpha + c at a node (in two-float arithmetic: the divergence of alpha cancels
// against c to the level of the dual residual) and <c, phi> in FP64.
template <int D>
__device__ __forceinline__ void kkt_node(const Geo& g, const MxFields& f, float2 sg2, long long i, int t,
                                         long long p, float* acc, double* dres, double* cphi) {
  float2 v = make_float2(0.f, 0.f);
  const float ih0 = (float)g.invh[0];
  if (t >= 1) v = ff_add(v, ff_mul_f(f.al[0][i - g.P], ih0));
  if (t < g.T) v = ff_add(v, ff_mul_f(ff_neg(f.al[0][i]), ih0));
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int x = coord(g, p, d);
    const float2* ad = f.al[1 + d];
    const long long s = g.sst[d];
    const float ih = (float)g.invh[1 + d];
    if (x >= 1) v = ff_add(v, ff_mul_f(ad[i - s], ih));
    if (x <= g.N[d] - 2) v = ff_add(v, ff_mul_f(ff_neg(ad[i]), ih));
  }
  v = ff_mul(v, sg2);   // A^* alpha = sigma A^*(alpha / sigma)
  double c = 0.0;
  if (t == 0) c += f.m0[p];
  if (t == g.T) c -= f.m1[p];
  if (c != 0.0) {
    const double res = ff_to_double(v) + c;
    *dres += res * res;
    *cphi += c * ff_to_double(f.phi[i]);
  } else {
    const float res = v.x + v.y;
    acc[R_DUALRES] += res * res;
  }
}

// All stopping-measure sums (one partial row per block), in D + 2 passes over the
// nodes: the cones, the faces of each axis, the nodes.  Separate loops keep each
// pass's loads in flight with few registers (one fused loop body needed ~220).
template <int D>
__global__ void __launch_bounds__(kThreads, KKT_MIN_BLOCKS) k_kkt(Geo g, MxFields fb, double* partials_all, int use_z) {
  const int slot = blockIdx.y;
  if (!fb.sp[slot].active) return;
  const MxFields f = slot_view(fb, g, slot);
  const float2 sg2 = fb.sp[slot].sg;
  const float sg = sg2.x + sg2.y;
  double* partials = partials_all + slot * kkt_partials_len_slot(g);
  float acc[R_NSLOTS];
#pragma unroll
  for (int k = 0; k < R_NSLOTS; ++k) acc[k] = 0.f;
  double dres = 0.0, cphi = 0.0;
  float2 dual = make_float2(0.f, 0.f);
  const long long n = (long long)(g.T + 1) * g.P, n0 = (long long)g.T * g.P;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
#pragma unroll 1
  for (long long i = i0; i < n0; i += stride) {
    const int t = plane_of(g, i);
    kkt_cone<D>(g, f, sg, i, i - (long long)t * g.P, use_z, acc);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
#pragma unroll 1
    for (long long i = i0; i < n; i += stride) {
      const int t = plane_of(g, i);
      const long long p = i - (long long)t * g.P;
      if (coord(g, p, d) <= g.N[d] - 2) kkt_face<D>(g, f, sg, d, i, t, p, acc, &dual);
    }
  }
#pragma unroll 1
  for (long long i = i0; i < n; i += stride) {
    const int t = plane_of(g, i);
    kkt_node<D>(g, f, sg2, i, t, i - (long long)t * g.P, acc, &dres, &cphi);
  }
  double accd[R_NSLOTS];
#pragma unroll
  for (int k = 0; k < R_NSLOTS; ++k) accd[k] = 0.0;
  accd[R_DUALRES] = dres;
  accd[R_CPHI] = cphi;
  accd[R_DUALOBJ] = ff_to_double(dual);
  block_reduce_store(acc, accd, partials + (long long)blockIdx.x * R_NSLOTS);
}

// rows: kernel groups (D + 2) x kb blocks; group j's partials start at row j * kKktBlocks.
__global__ void k_kkt_final(Geo g, const SlotParam* sp, const double* partials_all, int groups, int kb,
                            double* out_all, const double* socp_all, int nsocp) {
  const int slot = blockIdx.x;
  if (!sp[slot].active) return;
  const double* partials = partials_all + slot * kkt_partials_len_slot(g);
  double* out = out_all + slot * R_NSLOTS;
  const double* socp_part = socp_all ? socp_all + (long long)slot * nsocp : nullptr;
  const int rows = groups * kb;
  __shared__ double sh[kThreads];
  for (int k = 0; k < R_NSLOTS; ++k) {
    double v = 0.0;
    for (int e = threadIdx.x; e < rows; e += blockDim.x) {
      const int j = e / kb, r = e - j * kb;
      v += partials[((long long)j * kKktBlocks + r) * R_NSLOTS + k];
    }
    if (k == R_SOCP && socp_part)
      for (int r = threadIdx.x; r < nsocp; r += blockDim.x) v += socp_part[r];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    __syncthreads();
  }
}

// Line 2 with one refinement step: phi1 = P(b); r = b - A^*A phi1 (exact);
// delta = P(r); out = phi1 + delta as a two-float pair.  Overwrites f.b with delta.
template <int D>
void poisson_refined_tmpl(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, float2* out,
                          bool have_bsum, cudaStream_t s, LaunchCounter lc) {
  const long long nn = (long long)(g.T + 1) * g.P;
  const int nb = bsum_blocks(g);
  if (!have_bsum) {
    k_sum_b<<<dim3(nb, G), kThreads, 0, s>>>(g, f);
    lc.launched(KID_RESIDUAL);
  }
  k_mean_b<<<G, kThreads, 0, s>>>(g, f, nb);
  launch_poisson_mx(g, G, ps, f.b, f.phi1, s, lc, nullptr);
  k_residual<D><<<dim3(grid_for(nn), G), kThreads, 0, s>>>(g, f);
  lc.launched(KID_RESIDUAL, 2);
  launch_poisson_mx(g, G, ps, f.r, f.b, s, lc, nullptr);
  k_combine<<<dim3(grid_for(nn), G), kThreads, 0, s>>>(g, f, out);
  lc.launched(KID_COMBINE);
}

// delta = P(f.r), phi += delta: the last DCT pass adds into phi when it runs on
// the tensor cores; otherwise delta goes through phi1 and one more kernel.
void poisson_add_tmpl(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, cudaStream_t s,
                      LaunchCounter lc) {
  const long long nn = (long long)(g.T + 1) * g.P;
  if (launch_poisson_mx(g, G, ps, f.r, f.phi1, s, lc, f.phi)) return;
  k_phi_add<<<dim3(grid_for(nn), G), kThreads, 0, s>>>(g, f);
  lc.launched(KID_COMBINE);
}

// Lines 1 and 2 of an iteration (fused b-assembly and residual, one solve).
template <int D>
void assemble_solve_tmpl(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, cudaStream_t s,
                         LaunchCounter lc) {
  const long long nn = (long long)(g.T + 1) * g.P;
  k_assemble_residual<D><<<dim3(grid_for(nn), G), kThreads, 0, s>>>(g, f);
  lc.launched(KID_ASSEMBLE_B);
  poisson_add_tmpl(g, G, f, ps, s, lc);
}

template <int D>
void launch_kkt_tmpl(const Geo& g, int G, const MxFields& f, double* partials, double* out,
                     const double* socp_part, int nsocp, cudaStream_t s, LaunchCounter lc) {
  const int kb = kkt_blocks(g);
  k_kkt<D><<<dim3(kb, G), kThreads, 0, s>>>(g, f, partials, socp_part ? 0 : 1);
  k_kkt_final<<<G, kThreads, 0, s>>>(g, f.sp, partials, 1, kb, out, socp_part, nsocp);
  lc.launched(KID_KKT, 2);
}

}  // namespace

void launch_poisson_refined_mx(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, float2* out,
                               bool have_bsum, cudaStream_t s, LaunchCounter lc) {
  if (g.D == 2) poisson_refined_tmpl<2>(g, G, f, ps, out, have_bsum, s, lc);
  else poisson_refined_tmpl<3>(g, G, f, ps, out, have_bsum, s, lc);
}

void launch_rescale_mx(const Geo& g, int G, const MxFields& f, cudaStream_t s, LaunchCounter lc) {
  const long long nb = (long long)g.K * g.T * g.P;
  if (g.D == 2) k_rescale<2><<<dim3(grid_for(nb), G), kThreads, 0, s>>>(g, f);
  else k_rescale<3><<<dim3(grid_for(nb), G), kThreads, 0, s>>>(g, f);
  lc.launched(KID_UPDATE_BETA);
}

void launch_solve_residual_mx(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, cudaStream_t s,
                              LaunchCounter lc) {
  poisson_add_tmpl(g, G, f, ps, s, lc);
}

void launch_assemble_solve_mx(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, cudaStream_t s,
                              LaunchCounter lc) {
  if (g.D == 2) assemble_solve_tmpl<2>(g, G, f, ps, s, lc);
  else assemble_solve_tmpl<3>(g, G, f, ps, s, lc);
}

void launch_kkt_mx(const Geo& g, int G, const MxFields& f, double* partials, double* out,
                   const double* socp_part, int nsocp, cudaStream_t s, LaunchCounter lc) {
  if (g.D == 2) launch_kkt_tmpl<2>(g, G, f, partials, out, socp_part, nsocp, s, lc);
  else launch_kkt_tmpl<3>(g, G, f, partials, out, socp_part, nsocp, s, lc);
}

long long kkt_partials_len_mx(const Geo& g) { return kkt_partials_len_slot(g); }

}  // namespace dot
