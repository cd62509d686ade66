// k_fp64.cu -- FP64 reference path: the element-wise and stencil steps of
// Algorithm 2 (lines 1, 3, 4, 5, 6) and the stopping-measure reductions of Sec. 5.3.
//
// One thread per grid point (grid-stride loops).  Every neighbour is addressed
// through the padded plane layout described in dot_internal.cuh.
#include <cmath>

#include "dot_internal.cuh"

namespace dot {
namespace {

constexpr int kThreads = 256;

inline int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// Line 1 of Algorithm 2: b = A^*(q - alpha/sigma) - c/sigma on every node.
// A^* scatters +w/h to the node above a face and -w/h to the node below it, so a
// node gathers +w(face below) - w(face above) along each axis.  c is rho0's
// masses on plane 0 and -rho1's masses on plane T (eq. (defc)).
__global__ void k_assemble_b(Geo g, F64Fields f, double sigma) {
  const long long n = (long long)(g.T + 1) * g.P;
  const double isg = 1.0 / sigma;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = plane_of(g, i);
    const long long p = i - (long long)t * g.P;
    double acc = 0.0;
    if (t >= 1) acc += (f.q[0][i - g.P] - f.al[0][i - g.P] * isg) * g.invh[0];
    if (t < g.T) acc -= (f.q[0][i] - f.al[0][i] * isg) * g.invh[0];
    for (int d = 0; d < g.D; ++d) {
      const int x = coord(g, p, d);
      const double* qd = f.q[1 + d];
      const double* ad = f.al[1 + d];
      const long long s = g.sst[d];
      if (x >= 1) acc += (qd[i - s] - ad[i - s] * isg) * g.invh[1 + d];
      if (x <= g.N[d] - 2) acc -= (qd[i] - ad[i] * isg) * g.invh[1 + d];
    }
    double c = 0.0;
    if (t == 0) c += f.m0[p];
    if (t == g.T) c -= f.m1[p];
    f.b[i] = acc - c * isg;
  }
}

// Gather x = F q for cone (t, p): x[0] = q_0, x[1 + 4d + (v-1)] = F^d_v q_d (eq. (fdetails)).
__device__ __forceinline__ void gather_Fq(const Geo& g, double* const* q, long long i, long long p,
                                          double* x) {
  x[0] = q[0][i];
  for (int d = 0; d < g.D; ++d) {
    const int xd = coord(g, p, d);
    const double* qd = q[1 + d];
    const long long s = g.sst[d];
    const bool lo = xd >= 1, hi = xd <= g.N[d] - 2;
    x[1 + 4 * d + 0] = lo ? qd[i - s] : 0.0;            // (t,   x_d - 1/2)
    x[1 + 4 * d + 1] = hi ? qd[i] : 0.0;                // (t,   x_d + 1/2)
    x[1 + 4 * d + 2] = lo ? qd[i + g.P - s] : 0.0;      // (t+1, x_d - 1/2)
    x[1 + 4 * d + 3] = hi ? qd[i + g.P] : 0.0;          // (t+1, x_d + 1/2)
  }
}

// Projection onto the second-order cone {y0 >= |ybar|}, eq. (app-proj), in place.
__device__ __forceinline__ void proj_soc(int K, double* y) {
  double nb = 0.0;
  for (int j = 1; j < K; ++j) nb += y[j] * y[j];
  nb = sqrt(nb);
  if (nb <= y[0]) return;
  if (nb <= -y[0]) {
    for (int j = 0; j < K; ++j) y[j] = 0.0;
    return;
  }
  const double a = 0.5 * (y[0] + nb);
  const double scale = a / nb;   // one division (FP64 divisions are costly on this GPU)
  y[0] = a;
  for (int j = 1; j < K; ++j) y[j] = scale * y[j];
}

// Line 3: z = Pi_Q(B F q + d - beta/sigma), one cone per thread.
__global__ void k_project(Geo g, F64Fields f, double sigma) {
  const long long n0 = (long long)g.T * g.P;
  const double s_default = sqrt(0.5);
  const double isg = 1.0 / sigma;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i - (long long)plane_of(g, i) * g.P;
    double x[kMaxK];
    gather_Fq(g, f.q, i, p, x);
    const double s = f.somega ? f.somega[p] : s_default;
    const int K = g.K;
    double y[kMaxK];
    y[0] = -x[0] + 1.0 - f.beta[i] * isg;
    for (int j = 1; j < K - 1; ++j) y[j] = s * x[j] - f.beta[(long long)j * n0 + i] * isg;
    y[K - 1] = x[0] + 1.0 - f.beta[(long long)(K - 1) * n0 + i] * isg;
    proj_soc(K, y);
    for (int j = 0; j < K; ++j) f.z[(long long)j * n0 + i] = y[j];
  }
}

// Lines 4-5 on the time faces: the diagonal of I + F^*B^*BF is 3 on q_0
// (Proposition 3.2), F^*B^*u on q_0 is u_{K-1} - u_0.
__global__ void k_update_q0(Geo g, F64Fields f, double sigma, double tau) {
  const long long n0 = (long long)g.T * g.P;
  const int K = g.K;
  const double isg = 1.0 / sigma;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0;
       i += (long long)gridDim.x * blockDim.x) {
    const double aphi = (f.phi[i + g.P] - f.phi[i]) * g.invh[0];
    const double uK = f.z[(long long)(K - 1) * n0 + i] - 1.0 + f.beta[(long long)(K - 1) * n0 + i] * isg;
    const double u0 = f.z[i] - 1.0 + f.beta[i] * isg;
    const double a = f.al[0][i];
    const double qn = (aphi + a * isg + (uK - u0)) / 3.0;
    f.q[0][i] = qn;
    f.al[0][i] = a + tau * sigma * (aphi - qn);
  }
}

// Lines 4-5 on the faces of axis d: q_d at face (t, j) collects s_c (z + beta/sigma)
// of component 1 + 4d + (v-1) from the (up to) four cones that F^d_v maps it to:
// v=1: cone (t, j+1); v=2: cone (t, j); v=3: cone (t-1, j+1); v=4: cone (t-1, j).
// Its diagonal entry is 1 + sum of s_c^2 over those cones (Proposition 3.2 with
// the weighted B).  Pads (j = N_d - 1) are left at 0.
__global__ void k_update_qd(Geo g, F64Fields f, int d, double sigma, double tau) {
  const long long n = (long long)(g.T + 1) * g.P;
  const long long n0 = (long long)g.T * g.P;
  const double isg = 1.0 / sigma;
  const double s_default = sqrt(0.5);
  const long long s = g.sst[d];
  double* qd = f.q[1 + d];
  double* ad = f.al[1 + d];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = plane_of(g, i);
    const long long p = i - (long long)t * g.P;
    const int j = coord(g, p, d);
    if (j > g.N[d] - 2) continue;
    const double aphi = (f.phi[i + s] - f.phi[i]) * g.invh[1 + d];
    double acc = 0.0, dg = 0.0;
    const int cbase = 1 + 4 * d;
    if (t <= g.T - 1) {
      {  // v = 1: cone (t, j+1)
        const long long c = i + s;
        const double sc = f.somega ? f.somega[p + s] : s_default;
        const long long o = (long long)(cbase + 0) * n0 + c;
        acc += sc * (f.z[o] + f.beta[o] * isg);
        dg += sc * sc;
      }
      {  // v = 2: cone (t, j)
        const long long c = i;
        const double sc = f.somega ? f.somega[p] : s_default;
        const long long o = (long long)(cbase + 1) * n0 + c;
        acc += sc * (f.z[o] + f.beta[o] * isg);
        dg += sc * sc;
      }
    }
    if (t >= 1) {
      {  // v = 3: cone (t-1, j+1)
        const long long c = i - g.P + s;
        const double sc = f.somega ? f.somega[p + s] : s_default;
        const long long o = (long long)(cbase + 2) * n0 + c;
        acc += sc * (f.z[o] + f.beta[o] * isg);
        dg += sc * sc;
      }
      {  // v = 4: cone (t-1, j)
        const long long c = i - g.P;
        const double sc = f.somega ? f.somega[p] : s_default;
        const long long o = (long long)(cbase + 3) * n0 + c;
        acc += sc * (f.z[o] + f.beta[o] * isg);
        dg += sc * sc;
      }
    }
    const double a = ad[i];
    const double qn = (aphi + a * isg + acc) / (1.0 + dg);
    qd[i] = qn;
    ad[i] = a + tau * sigma * (aphi - qn);
  }
}

// Line 6: beta += tau sigma (z - B F q - d) with the new q.
__global__ void k_update_beta(Geo g, F64Fields f, double sigma, double tau) {
  const long long n0 = (long long)g.T * g.P;
  const double s_default = sqrt(0.5);
  const int K = g.K;
  const double ts = tau * sigma;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i - (long long)plane_of(g, i) * g.P;
    double x[kMaxK];
    gather_Fq(g, f.q, i, p, x);
    const double s = f.somega ? f.somega[p] : s_default;
    {
      const long long o = i;
      f.beta[o] += ts * (f.z[o] - (-x[0]) - 1.0);
    }
    for (int j = 1; j < K - 1; ++j) {
      const long long o = (long long)j * n0 + i;
      f.beta[o] += ts * (f.z[o] - s * x[j] - 0.0);
    }
    {
      const long long o = (long long)(K - 1) * n0 + i;
      f.beta[o] += ts * (f.z[o] - x[0] - 1.0);
    }
  }
}

// ---- stopping measures ------------------------------------------------------

constexpr int kKktBlocks = 608;

__device__ __forceinline__ void block_reduce_store(double* acc, double* out_row) {
  __shared__ double sh[kThreads / 32][R_NSLOTS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < R_NSLOTS; ++k) {
    double v = acc[k];
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

// Cones (time faces): eta_P terms of q_0, f(q), complementarity of alpha_0,
// z - BFq - d, and F^*B^*beta + alpha on q_0.
__global__ void k_kkt_cones(Geo g, F64Fields f, double* partials) {
  double acc[R_NSLOTS];
  for (int k = 0; k < R_NSLOTS; ++k) acc[k] = 0.0;
  const long long n0 = (long long)g.T * g.P;
  const double s_default = sqrt(0.5);
  const int K = g.K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i - (long long)plane_of(g, i) * g.P;
    double x[kMaxK];
    gather_Fq(g, f.q, i, p, x);
    const double aphi = (f.phi[i + g.P] - f.phi[i]) * g.invh[0];
    const double q0 = x[0];
    acc[R_PRIM] += (aphi - q0) * (aphi - q0);
    acc[R_APHI] += aphi * aphi;
    acc[R_Q] += q0 * q0;
    // f = q_0 + 1/2 omega L_T L_X^*(|q_bar|^2) = q_0 + (omega/8) sum_v x_v^2 (eq. (f1vf2v))
    double ss = 0.0;
    for (int j = 1; j < K - 1; ++j) ss += x[j] * x[j];
    const double om = f.omega ? f.omega[p] : 1.0;
    const double fv = q0 + 0.5 * om * (0.25 * ss);
    const double a0 = f.al[0][i];
    const double m = fv + a0;
    const double rc = a0 - (m > 0.0 ? m : 0.0);
    acc[R_COMP0] += rc * rc;
    acc[R_ALPHA0] += a0 * a0;
    acc[R_F] += fv * fv;
    const double s = f.somega ? f.somega[p] : s_default;
    double r = f.z[i] - (-q0) - 1.0;
    acc[R_SOCP] += r * r;
    for (int j = 1; j < K - 1; ++j) {
      r = f.z[(long long)j * n0 + i] - s * x[j];
      acc[R_SOCP] += r * r;
    }
    r = f.z[(long long)(K - 1) * n0 + i] - q0 - 1.0;
    acc[R_SOCP] += r * r;
    const double fbb = f.beta[(long long)(K - 1) * n0 + i] - f.beta[i];
    acc[R_SOCD] += (fbb + a0) * (fbb + a0);
    acc[R_FBB] += fbb * fbb;
  }
  block_reduce_store(acc, partials + (long long)blockIdx.x * R_NSLOTS);
}

// Faces of axis d: eta_P terms, g_d = (L_X^d L_T^*(omega alpha_0)) o q_d (the mean of
// omega alpha_0 over the up-to-four cones touching the face, each weighted 1/4),
// the dual objective term, and F^*B^*beta + alpha on q_d.
__global__ void k_kkt_faces(Geo g, F64Fields f, int d, double* partials) {
  double acc[R_NSLOTS];
  for (int k = 0; k < R_NSLOTS; ++k) acc[k] = 0.0;
  const long long n = (long long)(g.T + 1) * g.P;
  const long long n0 = (long long)g.T * g.P;
  const double s_default = sqrt(0.5);
  const long long s = g.sst[d];
  const double* qd = f.q[1 + d];
  const double* ad = f.al[1 + d];
  const double* a0 = f.al[0];
  const int cbase = 1 + 4 * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = plane_of(g, i);
    const long long p = i - (long long)t * g.P;
    const int j = coord(g, p, d);
    if (j > g.N[d] - 2) continue;
    const double aphi = (f.phi[i + s] - f.phi[i]) * g.invh[1 + d];
    const double q = qd[i];
    acc[R_PRIM] += (aphi - q) * (aphi - q);
    acc[R_APHI] += aphi * aphi;
    acc[R_Q] += q * q;
    double den = 0.0, fbb = 0.0;
    const double om_l = f.omega ? f.omega[p] : 1.0, om_r = f.omega ? f.omega[p + s] : 1.0;
    const double s_l = f.somega ? f.somega[p] : s_default, s_r = f.somega ? f.somega[p + s] : s_default;
    if (t <= g.T - 1) {
      den += om_r * a0[i + s] + om_l * a0[i];
      fbb += s_r * f.beta[(long long)(cbase + 0) * n0 + i + s] + s_l * f.beta[(long long)(cbase + 1) * n0 + i];
    }
    if (t >= 1) {
      den += om_r * a0[i - g.P + s] + om_l * a0[i - g.P];
      fbb += s_r * f.beta[(long long)(cbase + 2) * n0 + i - g.P + s] +
             s_l * f.beta[(long long)(cbase + 3) * n0 + i - g.P];
    }
    den *= 0.25;
    const double gv = den * q;
    const double a = ad[i];
    acc[R_COMPD] += (a - gv) * (a - gv);
    acc[R_ALPHAB] += a * a;
    acc[R_G] += gv * gv;
    if (den > 0.0) acc[R_DUALOBJ] -= 0.5 * a * a / den;
    acc[R_SOCD] += (fbb + a) * (fbb + a);
    acc[R_FBB] += fbb * fbb;
  }
  block_reduce_store(acc, partials + (long long)blockIdx.x * R_NSLOTS);
}

// Nodes: A^* alpha + c and <c, phi>.
__global__ void k_kkt_nodes(Geo g, F64Fields f, double* partials) {
  double acc[R_NSLOTS];
  for (int k = 0; k < R_NSLOTS; ++k) acc[k] = 0.0;
  const long long n = (long long)(g.T + 1) * g.P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = plane_of(g, i);
    const long long p = i - (long long)t * g.P;
    double v = 0.0;
    if (t >= 1) v += f.al[0][i - g.P] * g.invh[0];
    if (t < g.T) v -= f.al[0][i] * g.invh[0];
    for (int d = 0; d < g.D; ++d) {
      const int x = coord(g, p, d);
      const double* ad = f.al[1 + d];
      const long long s = g.sst[d];
      if (x >= 1) v += ad[i - s] * g.invh[1 + d];
      if (x <= g.N[d] - 2) v -= ad[i] * g.invh[1 + d];
    }
    double c = 0.0;
    if (t == 0) c += f.m0[p];
    if (t == g.T) c -= f.m1[p];
    v += c;
    acc[R_DUALRES] += v * v;
    acc[R_CPHI] += c * f.phi[i];
  }
  block_reduce_store(acc, partials + (long long)blockIdx.x * R_NSLOTS);
}

// Fixed-order sum of the partial rows: deterministic run to run.
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

}  // namespace

void launch_assemble_b_f64(const Geo& g, const F64Fields& f, double sigma, cudaStream_t s, LaunchCounter lc) {
  k_assemble_b<<<grid_for((long long)(g.T + 1) * g.P), kThreads, 0, s>>>(g, f, sigma);
  lc.launched(KID_ASSEMBLE_B);
}

void launch_project_f64(const Geo& g, const F64Fields& f, double sigma, cudaStream_t s, LaunchCounter lc) {
  k_project<<<grid_for((long long)g.T * g.P), kThreads, 0, s>>>(g, f, sigma);
  lc.launched(KID_PROJECT);
}

void launch_update_q_alpha_f64(const Geo& g, const F64Fields& f, double sigma, double tau, cudaStream_t s,
                               LaunchCounter lc) {
  k_update_q0<<<grid_for((long long)g.T * g.P), kThreads, 0, s>>>(g, f, sigma, tau);
  lc.launched(KID_UPDATE_Q0);
  for (int d = 0; d < g.D; ++d) {
    k_update_qd<<<grid_for((long long)(g.T + 1) * g.P), kThreads, 0, s>>>(g, f, d, sigma, tau);
    lc.launched(KID_UPDATE_QD);
  }
}

void launch_update_beta_f64(const Geo& g, const F64Fields& f, double sigma, double tau, cudaStream_t s,
                            LaunchCounter lc) {
  k_update_beta<<<grid_for((long long)g.T * g.P), kThreads, 0, s>>>(g, f, sigma, tau);
  lc.launched(KID_UPDATE_BETA);
}

long long kkt_partials_len(const Geo& g) { return (long long)(g.D + 2) * kKktBlocks * R_NSLOTS; }

void launch_kkt_f64(const Geo& g, const F64Fields& f, double* partials, double* out, cudaStream_t s,
                    LaunchCounter lc) {
  k_kkt_cones<<<kKktBlocks, kThreads, 0, s>>>(g, f, partials);
  for (int d = 0; d < g.D; ++d)
    k_kkt_faces<<<kKktBlocks, kThreads, 0, s>>>(g, f, d, partials + (long long)(1 + d) * kKktBlocks * R_NSLOTS);
  k_kkt_nodes<<<kKktBlocks, kThreads, 0, s>>>(g, f, partials + (long long)(1 + g.D) * kKktBlocks * R_NSLOTS);
  k_kkt_final<<<1, kThreads, 0, s>>>(partials, (g.D + 2) * kKktBlocks, out);
  lc.launched(KID_KKT, g.D + 3);
}

}  // namespace dot
