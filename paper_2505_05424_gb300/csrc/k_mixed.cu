// k_mixed.cu -- mixed-precision kernels of Algorithm 2 (lines 1, 3, 4, 5, 6),
// the exact-residual step of the Poisson refinement, and the stopping measures.
//
// Storage: q and z in FP32; alpha, beta and phi as two-float pairs (hi, lo);
// b and the Poisson scratch in FP32.  Arithmetic is FP32; updates of the
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

// A phi along an axis from the two-float potential: the difference of the hi
// parts is exact or rounded relative to the difference itself.
__device__ __forceinline__ float grad_ff(const float2* phi, long long i, long long j, float invh) {
  const float2 a = phi[i], b = phi[j];
  return ((b.x - a.x) + (b.y - a.y)) * invh;
}

// Line 1: b = A^*(q - alpha/sigma) - c/sigma.
template <int D>
__global__ void k_assemble_b(Geo g, MxFields f, float isg) {
  const long long n = (long long)(g.T + 1) * g.P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / g.P);
    const long long p = i - (long long)t * g.P;
    const float ih0 = (float)g.invh[0];
    float acc = 0.f;
    if (t >= 1) acc += (f.q[0][i - g.P] - f.al[0][i - g.P].x * isg) * ih0;
    if (t < g.T) acc -= (f.q[0][i] - f.al[0][i].x * isg) * ih0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int x = coord(g, p, d);
      const float* qd = f.q[1 + d];
      const float2* ad = f.al[1 + d];
      const long long s = g.sst[d];
      const float ih = (float)g.invh[1 + d];
      if (x >= 1) acc += (qd[i - s] - ad[i - s].x * isg) * ih;
      if (x <= g.N[d] - 2) acc -= (qd[i] - ad[i].x * isg) * ih;
    }
    float c = 0.f;
    if (t == 0) c += f.m0f[p];
    if (t == g.T) c -= f.m1f[p];
    f.b[i] = acc - c * isg;
  }
}

// Refinement residual r = b - A^*A phi1, with A^*A phi1 accumulated exactly in
// two-float arithmetic (each neighbour difference by TwoSum; 1/h^2 is an integer).
template <int D>
__global__ void k_residual(Geo g, MxFields f) {
  const long long n = (long long)(g.T + 1) * g.P;
  const float* x = f.phi1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / g.P);
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
    const float2 r = ff_add_f(ff_neg(acc), f.b[i]);
    f.r[i] = r.x + r.y;
  }
}

// phi = phi1 + delta as a two-float pair.
__global__ void k_combine(long long n, const float* __restrict__ phi1, const float* __restrict__ delta,
                          float2* __restrict__ phi) {
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

template <int K>
__device__ __forceinline__ void proj_soc(float* y) {
  float nb2 = 0.f;
#pragma unroll
  for (int j = 1; j < K; ++j) nb2 = fmaf(y[j], y[j], nb2);
  const float nb = sqrtf(nb2);
  if (nb <= y[0]) return;
  if (nb <= -y[0]) {
#pragma unroll
    for (int j = 0; j < K; ++j) y[j] = 0.f;
    return;
  }
  const float a = 0.5f * (y[0] + nb);
  const float sc = a / nb;
  y[0] = a;
#pragma unroll
  for (int j = 1; j < K; ++j) y[j] *= sc;
}

// Line 3: z = Pi_Q(B F q + d - beta/sigma).
template <int D>
__global__ void k_project(Geo g, MxFields f, float isg) {
  constexpr int K = 4 * D + 2;
  const long long n0 = (long long)g.T * g.P;
  const float s_default = 0.70710678118654752f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i % g.P;
    float x[K - 1];
    gather_Fq<D>(g, f.q, i, p, x);
    const float s = f.somega ? f.somega[p] : s_default;
    float y[K];
    y[0] = -x[0] + 1.f - f.beta[i].x * isg;
#pragma unroll
    for (int j = 1; j < K - 1; ++j) y[j] = s * x[j] - f.beta[(long long)j * n0 + i].x * isg;
    y[K - 1] = x[0] + 1.f - f.beta[(long long)(K - 1) * n0 + i].x * isg;
    proj_soc<K>(y);
#pragma unroll
    for (int j = 0; j < K; ++j) f.z[(long long)j * n0 + i] = y[j];
  }
}

// Lines 4-5 on the time faces (diagonal 3, F^*B^*u = u_{K-1} - u_0).
template <int D>
__global__ void k_update_q0(Geo g, MxFields f, float sigma, float tau) {
  constexpr int K = 4 * D + 2;
  const long long n0 = (long long)g.T * g.P;
  const float isg = 1.f / sigma, ts = tau * sigma;
  const float ih0 = (float)g.invh[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0;
       i += (long long)gridDim.x * blockDim.x) {
    const float aphi = grad_ff(f.phi, i, i + g.P, ih0);
    const float uK = f.z[(long long)(K - 1) * n0 + i] + f.beta[(long long)(K - 1) * n0 + i].x * isg;
    const float u0 = f.z[i] + f.beta[i].x * isg;
    const float2 a = f.al[0][i];
    const float qn = (aphi + a.x * isg + (uK - u0)) * (1.f / 3.f);
    f.q[0][i] = qn;
    f.al[0][i] = ff_add_f(a, ts * (aphi - qn));
  }
}

// Lines 4-5 on the faces of axis d (see the FP64 kernel for the cone bookkeeping).
template <int D>
__global__ void k_update_qd(Geo g, MxFields f, int d, float sigma, float tau) {
  const long long n = (long long)(g.T + 1) * g.P;
  const long long n0 = (long long)g.T * g.P;
  const float isg = 1.f / sigma, ts = tau * sigma;
  const float s_default = 0.70710678118654752f;
  const long long s = g.sst[d];
  float* qd = f.q[1 + d];
  float2* ad = f.al[1 + d];
  const float ih = (float)g.invh[1 + d];
  const int cbase = 1 + 4 * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / g.P);
    const long long p = i - (long long)t * g.P;
    const int j = coord(g, p, d);
    if (j > g.N[d] - 2) continue;
    const float aphi = grad_ff(f.phi, i, i + s, ih);
    const float s_r = f.somega ? f.somega[p + s] : s_default;
    const float s_l = f.somega ? f.somega[p] : s_default;
    float acc = 0.f, dg = 0.f;
    if (t <= g.T - 1) {
      const long long o1 = (long long)(cbase + 0) * n0 + i + s;
      const long long o2 = (long long)(cbase + 1) * n0 + i;
      acc += s_r * (f.z[o1] + f.beta[o1].x * isg) + s_l * (f.z[o2] + f.beta[o2].x * isg);
      dg += s_r * s_r + s_l * s_l;
    }
    if (t >= 1) {
      const long long o3 = (long long)(cbase + 2) * n0 + i - g.P + s;
      const long long o4 = (long long)(cbase + 3) * n0 + i - g.P;
      acc += s_r * (f.z[o3] + f.beta[o3].x * isg) + s_l * (f.z[o4] + f.beta[o4].x * isg);
      dg += s_r * s_r + s_l * s_l;
    }
    const float2 a = ad[i];
    const float qn = (aphi + a.x * isg + acc) / (1.f + dg);
    qd[i] = qn;
    ad[i] = ff_add_f(a, ts * (aphi - qn));
  }
}

// Line 6: beta += tau sigma (z - B F q - d).
template <int D>
__global__ void k_update_beta(Geo g, MxFields f, float ts) {
  constexpr int K = 4 * D + 2;
  const long long n0 = (long long)g.T * g.P;
  const float s_default = 0.70710678118654752f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i % g.P;
    float x[K - 1];
    gather_Fq<D>(g, f.q, i, p, x);
    const float s = f.somega ? f.somega[p] : s_default;
    f.beta[i] = ff_add_f(f.beta[i], ts * (f.z[i] + x[0] - 1.f));
#pragma unroll
    for (int j = 1; j < K - 1; ++j) {
      const long long o = (long long)j * n0 + i;
      f.beta[o] = ff_add_f(f.beta[o], ts * (f.z[o] - s * x[j]));
    }
    const long long o = (long long)(K - 1) * n0 + i;
    f.beta[o] = ff_add_f(f.beta[o], ts * (f.z[o] - x[0] - 1.f));
  }
}

// ---- stopping measures: FP32 terms, per-thread FP32 sums, FP64 tree -----------

constexpr int kKktBlocks = 608;

__device__ __forceinline__ void block_reduce_store(const float* accf, const double* accd, double* out_row) {
  __shared__ double sh[kThreads / 32][R_NSLOTS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

template <int D>
__global__ void k_kkt_cones(Geo g, MxFields f, double* partials) {
  constexpr int K = 4 * D + 2;
  float acc[R_NSLOTS];
  double accd[R_NSLOTS];
  for (int k = 0; k < R_NSLOTS; ++k) { acc[k] = 0.f; accd[k] = 0.0; }
  const long long n0 = (long long)g.T * g.P;
  const float s_default = 0.70710678118654752f;
  const float ih0 = (float)g.invh[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i % g.P;
    float x[K - 1];
    gather_Fq<D>(g, f.q, i, p, x);
    const float aphi = grad_ff(f.phi, i, i + g.P, ih0);
    const float q0 = x[0];
    acc[R_PRIM] += (aphi - q0) * (aphi - q0);
    acc[R_APHI] += aphi * aphi;
    acc[R_Q] += q0 * q0;
    float ss = 0.f;
#pragma unroll
    for (int j = 1; j < K - 1; ++j) ss += x[j] * x[j];
    const float om = f.omega ? f.omega[p] : 1.f;
    const float fv = q0 + 0.125f * om * ss;
    const float a0 = f.al[0][i].x + f.al[0][i].y;
    const float m = fv + a0;
    const float rc = a0 - (m > 0.f ? m : 0.f);
    acc[R_COMP0] += rc * rc;
    acc[R_ALPHA0] += a0 * a0;
    acc[R_F] += fv * fv;
    const float s = f.somega ? f.somega[p] : s_default;
    float r = f.z[i] + q0 - 1.f;
    acc[R_SOCP] += r * r;
#pragma unroll
    for (int j = 1; j < K - 1; ++j) {
      r = f.z[(long long)j * n0 + i] - s * x[j];
      acc[R_SOCP] += r * r;
    }
    r = f.z[(long long)(K - 1) * n0 + i] - q0 - 1.f;
    acc[R_SOCP] += r * r;
    const float2 bK = f.beta[(long long)(K - 1) * n0 + i], b0 = f.beta[i];
    const float fbb = (bK.x - b0.x) + (bK.y - b0.y);
    acc[R_SOCD] += (fbb + a0) * (fbb + a0);
    acc[R_FBB] += fbb * fbb;
  }
  block_reduce_store(acc, accd, partials + (long long)blockIdx.x * R_NSLOTS);
}

template <int D>
__global__ void k_kkt_faces(Geo g, MxFields f, int d, double* partials) {
  float acc[R_NSLOTS];
  double accd[R_NSLOTS];
  for (int k = 0; k < R_NSLOTS; ++k) { acc[k] = 0.f; accd[k] = 0.0; }
  const long long n = (long long)(g.T + 1) * g.P;
  const long long n0 = (long long)g.T * g.P;
  const float s_default = 0.70710678118654752f;
  const long long s = g.sst[d];
  const float* qd = f.q[1 + d];
  const float2* ad = f.al[1 + d];
  const float2* a0 = f.al[0];
  const int cbase = 1 + 4 * d;
  const float ih = (float)g.invh[1 + d];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / g.P);
    const long long p = i - (long long)t * g.P;
    const int j = coord(g, p, d);
    if (j > g.N[d] - 2) continue;
    const float aphi = grad_ff(f.phi, i, i + s, ih);
    const float q = qd[i];
    acc[R_PRIM] += (aphi - q) * (aphi - q);
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
    den *= 0.25f;
    const float gv = den * q;
    const float a = ad[i].x + ad[i].y;
    acc[R_COMPD] += (a - gv) * (a - gv);
    acc[R_ALPHAB] += a * a;
    acc[R_G] += gv * gv;
    if (den > 0.f) accd[R_DUALOBJ] -= 0.5 * (double)a * (double)a / (double)den;
    acc[R_SOCD] += (fbb + a) * (fbb + a);
    acc[R_FBB] += fbb * fbb;
  }
  block_reduce_store(acc, accd, partials + (long long)blockIdx.x * R_NSLOTS);
}

// Nodes: A^*alpha + c (in two-float arithmetic: the divergence of alpha cancels
// against c to the level of the dual residual) and <c, phi> in FP64.
template <int D>
__global__ void k_kkt_nodes(Geo g, MxFields f, double* partials) {
  float acc[R_NSLOTS];
  double accd[R_NSLOTS];
  for (int k = 0; k < R_NSLOTS; ++k) { acc[k] = 0.f; accd[k] = 0.0; }
  const long long n = (long long)(g.T + 1) * g.P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / g.P);
    const long long p = i - (long long)t * g.P;
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
    double c = 0.0;
    if (t == 0) c += f.m0[p];
    if (t == g.T) c -= f.m1[p];
    if (c != 0.0) {
      const double res = ff_to_double(v) + c;
      accd[R_DUALRES] += res * res;
      accd[R_CPHI] += c * ff_to_double(f.phi[i]);
    } else {
      const float res = v.x + v.y;
      acc[R_DUALRES] += res * res;
    }
  }
  block_reduce_store(acc, accd, partials + (long long)blockIdx.x * R_NSLOTS);
}

__global__ void k_kkt_final(const double* partials, int rows, double* out) {
  __shared__ double sh[kThreads];
  for (int k = 0; k < R_NSLOTS; ++k) {
    double v = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) v += partials[(long long)r * R_NSLOTS + k];
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
void poisson_refined_tmpl(const Geo& g, const MxFields& f, const MxPoisson& ps, float2* out, cudaStream_t s,
                          LaunchCounter lc) {
  const long long nn = (long long)(g.T + 1) * g.P;
  launch_poisson_mx(g, ps, f.b, f.phi1, s, lc);
  k_residual<D><<<grid_for(nn), kThreads, 0, s>>>(g, f);
  lc.launched(KID_RESIDUAL);
  launch_poisson_mx(g, ps, f.r, f.b, s, lc);
  k_combine<<<grid_for(nn), kThreads, 0, s>>>(nn, f.phi1, f.b, out);
  lc.launched(KID_COMBINE);
}

template <int D>
void launch_iter_tmpl(const Geo& g, const MxFields& f, const MxPoisson& ps, double sigma, double tau,
                      cudaStream_t s, LaunchCounter lc) {
  const long long nn = (long long)(g.T + 1) * g.P, n0 = (long long)g.T * g.P;
  const float isg = (float)(1.0 / sigma);
  k_assemble_b<D><<<grid_for(nn), kThreads, 0, s>>>(g, f, isg);                 // line 1
  lc.launched(KID_ASSEMBLE_B);
  poisson_refined_tmpl<D>(g, f, ps, f.phi, s, lc);                                // line 2
  k_project<D><<<grid_for(n0), kThreads, 0, s>>>(g, f, isg);                      // line 3
  lc.launched(KID_PROJECT);
  k_update_q0<D><<<grid_for(n0), kThreads, 0, s>>>(g, f, (float)sigma, (float)tau);  // lines 4-5
  lc.launched(KID_UPDATE_Q0);
  for (int d = 0; d < D; ++d) {
    k_update_qd<D><<<grid_for(nn), kThreads, 0, s>>>(g, f, d, (float)sigma, (float)tau);
    lc.launched(KID_UPDATE_QD);
  }
  k_update_beta<D><<<grid_for(n0), kThreads, 0, s>>>(g, f, (float)(tau * sigma));  // line 6
  lc.launched(KID_UPDATE_BETA);
}

template <int D>
void launch_kkt_tmpl(const Geo& g, const MxFields& f, double* partials, double* out, cudaStream_t s,
                     LaunchCounter lc) {
  k_kkt_cones<D><<<kKktBlocks, kThreads, 0, s>>>(g, f, partials);
  for (int d = 0; d < D; ++d)
    k_kkt_faces<D><<<kKktBlocks, kThreads, 0, s>>>(g, f, d, partials + (long long)(1 + d) * kKktBlocks * R_NSLOTS);
  k_kkt_nodes<D><<<kKktBlocks, kThreads, 0, s>>>(g, f, partials + (long long)(1 + D) * kKktBlocks * R_NSLOTS);
  k_kkt_final<<<1, kThreads, 0, s>>>(partials, (D + 2) * kKktBlocks, out);
  lc.launched(KID_KKT, D + 3);
}

}  // namespace

void launch_iterate_mx(const Geo& g, const MxFields& f, const MxPoisson& ps, double sigma, double tau,
                       cudaStream_t s, LaunchCounter lc) {
  if (g.D == 2) launch_iter_tmpl<2>(g, f, ps, sigma, tau, s, lc);
  else launch_iter_tmpl<3>(g, f, ps, sigma, tau, s, lc);
}

void launch_poisson_refined_mx(const Geo& g, const MxFields& f, const MxPoisson& ps, float2* out,
                               cudaStream_t s, LaunchCounter lc) {
  if (g.D == 2) poisson_refined_tmpl<2>(g, f, ps, out, s, lc);
  else poisson_refined_tmpl<3>(g, f, ps, out, s, lc);
}

void launch_kkt_mx(const Geo& g, const MxFields& f, double* partials, double* out, cudaStream_t s,
                   LaunchCounter lc) {
  if (g.D == 2) launch_kkt_tmpl<2>(g, f, partials, out, s, lc);
  else launch_kkt_tmpl<3>(g, f, partials, out, s, lc);
}

long long kkt_partials_len_mx(const Geo& g) { return (long long)(g.D + 2) * kKktBlocks * R_NSLOTS; }

}  // namespace dot
