// k_fused2d.cu -- lines 3-6 of Algorithm 2 (cone projection, q and alpha updates,
// beta update) fused into one pass over the mixed-path state, for D = 2.
//
// A CTA owns a 16 x 32 (x, y) tile of the spatial grid and a chunk [ta, tb) of
// cone times, and marches along time.  At cone time t it
//   A. projects z(t) = Pi_K(B F q^k + d - beta^k/sigma) for the tile's cones and a
//      one-cone halo ring, keeps u_v = z_v + beta_v/sigma (v = 1..8, the parts
//      F^*B^* sends to space faces) in shared memory for two time levels, keeps the
//      owned cones' z in registers, and updates q_0, alpha_0 of the owned cones
//      (diagonal 3, Proposition 3.2);
//   B. updates q_d, alpha_d at the faces of time node t that touch the tile
//      (including the one halo face per axis that the tile's cones read);
//   C. updates beta of the owned cones at time t-1, which needs q^{k+1} on the
//      faces of time nodes t-1 and t (kept in shared memory).
// beta is read once (plus an L2 re-read in C) and written once; z never reaches
// HBM.  q, alpha and beta are double-buffered: every read is of iteration k and
// every write of k+1, so neighbouring CTAs may run at any relative time.
// Per element: y and the projection tests in two-float arithmetic, FP32 z and q, two-float
// face right-hand sides and multiplier updates (ffloat.cuh), as in k_fused3d.cu.
#include <cmath>

#include "dot_internal.cuh"
#include "dot_mixed.cuh"
#include "dot_tc.cuh"
#include "ffloat.cuh"

#ifndef FUSED_V2_MIN_BLOCKS
#define FUSED_V2_MIN_BLOCKS 2
#endif

namespace dot {
namespace {

constexpr int TX = 16, TY = 32;          // owned tile (x rows, y columns)
constexpr int HX = TX + 2, HY = TY + 2;  // cone halo rectangle
constexpr int NH = HX * HY;              // 612 cones
constexpr int NRING = NH - TX * TY;      // 100 halo-ring cones
constexpr int K2 = 10;                   // 4D + 2 for D = 2
constexpr int kThreads = 256;
constexpr int NQ1 = (TX + 1) * TY;       // x-faces per time node: j in [x0-1, x0+15], y owned
constexpr int NQ2 = TX * (TY + 1);       // y-faces per time node: x owned, j in [y0-1, y0+31]

// The multipliers are stored as alpha/sigma and beta/sigma (k_mixed.cu), so the
// projection input is BFq + d - (stored beta) and the updates add tau (...).
struct FusedArgs {
  // iteration k (read)
  const float* q[3];
  const float2* al[3];
  const float2* beta;
  // iteration k+1 (write)
  float* qn[3];
  float2* aln[3];
  float2* betan;
  const float2* phi;   // phi^{k+1}
  const float* somega;
  float ts;            // tau (set per slot from sp)
  int tchunk;          // cone times per CTA
  int nchunk;          // time chunks per slot (grid z = slots x chunks)
  const SlotParam* sp;
  double* socp_part;   // per-block sum of |z - B F q^{k+1} - d|^2, or nullptr
  long long socp_per_slot;
  int* err;            // set when a pipeline wait gave up
  // TMA kernel only (nullable r): the next iteration's lines 1-2 residual
  // r = A^*(q^{k+1} - alpha^{k+1}/sigma) - c/sigma - A^*A phi^{k+1} at every node
  float* r;
  const float2* c0;
  const float2* c1;
  float2 isg;          // 1/sigma (set per slot from sp)
};

// The arguments of slot b of a batch.
__device__ __forceinline__ FusedArgs fused_slot(FusedArgs a, const Geo& g, int b) {
  const long long nn = (long long)(g.T + 1) * g.P, n0 = (long long)g.T * g.P;
  a.ts = a.sp[b].tau;
  a.isg = a.sp[b].isg;
  if (b == 0) return a;
  a.q[0] += b * n0;
  a.al[0] += b * n0;
  a.qn[0] += b * n0;
  a.aln[0] += b * n0;
  for (int d = 1; d < 3; ++d) {
    a.q[d] += b * nn;
    a.al[d] += b * nn;
    a.qn[d] += b * nn;
    a.aln[d] += b * nn;
  }
  a.beta += b * K2 * n0;
  a.betan += b * K2 * n0;
  a.phi += b * nn;
  if (a.somega) a.somega += b * g.P;
  if (a.socp_part) a.socp_part += b * a.socp_per_slot;
  if (a.r) {
    a.r += b * nn;
    a.c0 += b * g.P;
    a.c1 += b * g.P;
  }
  return a;
}

// halo-ring cone number r (0..99) -> (xh, yh) on the border of the HX x HY rectangle
__device__ __forceinline__ void ring_pos(int r, int* xh, int* yh) {
  if (r < HY) { *xh = 0; *yh = r; return; }
  r -= HY;
  if (r < HY) { *xh = HX - 1; *yh = r; return; }
  r -= HY;
  if (r < HX - 2) { *xh = 1 + r; *yh = 0; return; }
  r -= HX - 2;
  *xh = 1 + r;
  *yh = HY - 1;
}

__device__ __forceinline__ float2 grad_pair(const float2* phi, long long i, long long j, float invh) {
  const float2 a = phi[i], b = phi[j];
  const float2 dh = two_sum(b.x, -a.x);
  const float dl = (b.y - a.y) + dh.y;
  return make_float2(dh.x * invh, dl * invh);
}

__device__ __forceinline__ float grad_minus(float2 g, float q) { return (g.x - q) + g.y; }

// z of cone (t, x, y) from iteration-k data, formed and projected in two-float
// arithmetic (y = BFq + d - beta/sigma is dominated by beta/sigma); returns false
// for a cone outside the grid.
__device__ __forceinline__ bool cone_z(const Geo& g, const FusedArgs& a, int t, int x, int y, float2* z) {
  if (x < 0 || y < 0 || x >= g.N[0] || y >= g.N[1]) return false;
  const long long P = g.P, n0 = (long long)g.T * P;
  const long long N1 = g.N[1];
  const long long i = (long long)t * P + (long long)x * N1 + y;
  const float* q1 = a.q[1];
  const float* q2 = a.q[2];
  const bool xl = x >= 1, xr = x <= g.N[0] - 2, yl = y >= 1, yr = y <= g.N[1] - 2;
  float xv[K2 - 1];
  xv[0] = a.q[0][i];
  xv[1] = xl ? q1[i - N1] : 0.f;
  xv[2] = xr ? q1[i] : 0.f;
  xv[3] = xl ? q1[i + P - N1] : 0.f;
  xv[4] = xr ? q1[i + P] : 0.f;
  xv[5] = yl ? q2[i - 1] : 0.f;
  xv[6] = yr ? q2[i] : 0.f;
  xv[7] = yl ? q2[i + P - 1] : 0.f;
  xv[8] = yr ? q2[i + P] : 0.f;
  const float s = a.somega ? a.somega[(long long)x * N1 + y] : 0.70710678118654752f;
  z[0] = ff_add(two_sum(-xv[0], 1.f), ff_neg(a.beta[i]));
#pragma unroll
  for (int j = 1; j < K2 - 1; ++j)
    z[j] = ff_add(two_prod(s, xv[j]), ff_neg(a.beta[(long long)j * n0 + i]));
  z[K2 - 1] = ff_add(two_sum(xv[0], 1.f), ff_neg(a.beta[(long long)(K2 - 1) * n0 + i]));
  ff_proj_soc<K2>(z);
  return true;
}

constexpr int kSmemFused = (2 * 8 * NH) * 8 + (2 * NQ1 + 2 * NQ2) * 4;

__global__ void __launch_bounds__(kThreads, 2) k_fused2d(Geo g, FusedArgs a_in) {
  const int slot = blockIdx.z / a_in.nchunk, chunk = blockIdx.z - slot * a_in.nchunk;
  if (!a_in.sp[slot].active) return;
  const FusedArgs a = fused_slot(a_in, g, slot);
  // u_1..u_8 (two-float) of every halo cone at two time levels, then q^{k+1} on
  // the tile's x-faces and y-faces at two node levels
  extern __shared__ __align__(16) unsigned char fsm[];
  float2 (*su)[8][NH] = reinterpret_cast<float2 (*)[8][NH]>(fsm);
  float (*sq1)[NQ1] = reinterpret_cast<float (*)[NQ1]>(fsm + (2 * 8 * NH) * 8);
  float (*sq2)[NQ2] = reinterpret_cast<float (*)[NQ2]>(fsm + (2 * 8 * NH) * 8 + 2 * NQ1 * 4);

  const int tid = threadIdx.x;
  const int ly = tid & 31, lx = tid >> 5;   // owned nodes (x0 + lx + 8r, y0 + ly)
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int ta = chunk * a.tchunk;
  const int tb = min(g.T, ta + a.tchunk);
  const bool last_chunk = (tb == g.T);
  const long long P = g.P, n0 = (long long)g.T * P;
  const long long N1 = g.N[1];
  const float ts = a.ts;
  const float ih0 = (float)g.invh[0], ih1 = (float)g.invh[1], ih2 = (float)g.invh[2];
  const float s_def = 0.70710678118654752f;

  // registers of the two owned cones: z at the current and previous cone time,
  // q_0^{k+1} at the previous cone time
  float zc[2][K2], zp[2][K2];
  float q0c[2] = {0.f, 0.f}, q0p[2] = {0.f, 0.f};
  float socp = 0.f;
  bool own_ok[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) own_ok[r] = (x0 + lx + 8 * r) < g.N[0] && (y0 + ly) < g.N[1];

  const int tstart = ta > 0 ? ta - 1 : 0;
  for (int t = tstart; t <= tb; ++t) {
    const int lev = t & 1;
    // ---------------- A: cones at time t ----------------
    if (t <= g.T - 1) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int x = x0 + lx + 8 * r, y = y0 + ly;
        const int hc = (lx + 8 * r + 1) * HY + (ly + 1);
        float2 z[K2];
        const bool ok = own_ok[r] && cone_z(g, a, t, x, y, z);
        if (ok) {
          const long long i = (long long)t * P + (long long)x * N1 + y;
#pragma unroll
          for (int v = 0; v < 8; ++v) su[lev][v][hc] = ff_add(z[1 + v], a.beta[(long long)(1 + v) * n0 + i]);
          if (t >= ta && t < tb) {
            // lines 4-5 on q_0: rhs = A_0 phi + (alpha_0 + beta_{K-1} - beta_0)/sigma + (z_{K-1} - z_0),
            // diagonal 3, in two-float arithmetic
            const float2 gp = grad_pair(a.phi, i, i + P, ih0);
            const float2 al = a.al[0][i];
            const float2 db = ff_add(a.beta[(long long)(K2 - 1) * n0 + i], ff_neg(a.beta[i]));
            float2 rhs = ff_add(gp, ff_add(al, db));
            rhs = ff_add(rhs, ff_add(z[K2 - 1], ff_neg(z[0])));
            const float qn = ff_round(ff_div_f(rhs, 3.f));
            a.qn[0][i] = qn;
            a.aln[0][i] = ff_add_f(al, ts * grad_minus(gp, qn));
            q0c[r] = qn;   // becomes q0p at the end of this step
          }
#pragma unroll
          for (int j = 0; j < K2; ++j) zc[r][j] = ff_round(z[j]);
        } else {
#pragma unroll
          for (int v = 0; v < 8; ++v) su[lev][v][hc] = make_float2(0.f, 0.f);
        }
      }
      for (int rr = tid; rr < NRING; rr += kThreads) {
        int xh, yh;
        ring_pos(rr, &xh, &yh);
        const int x = x0 - 1 + xh, y = y0 - 1 + yh;
        const int hc = xh * HY + yh;
        float2 z[K2];
        if (cone_z(g, a, t, x, y, z)) {
          const long long i = (long long)t * P + (long long)x * N1 + y;
#pragma unroll
          for (int v = 0; v < 8; ++v) su[lev][v][hc] = ff_add(z[1 + v], a.beta[(long long)(1 + v) * n0 + i]);
        } else {
#pragma unroll
          for (int v = 0; v < 8; ++v) su[lev][v][hc] = make_float2(0.f, 0.f);
        }
      }
    }
    __syncthreads();
    // ---------------- B: faces at time node t ----------------
    const bool write_node = t >= ta && ((t < tb) || (last_chunk && t == g.T));
    if (t >= ta) {
      const bool has_now = t <= g.T - 1, has_prev = t >= 1;
      const int lp = lev ^ 1;
      for (int e = tid; e < NQ1 + NQ2; e += kThreads) {
        if (e < NQ1) {
          // x-face (t, j, y): j = x0 - 1 + e / TY, y = y0 + e % TY
          const int jx = e / TY, yy = e % TY;
          const int j = x0 - 1 + jx, y = y0 + yy;
          float qv = 0.f;
          if (j >= 0 && j <= g.N[0] - 2 && y < g.N[1]) {
            const long long i = (long long)t * P + (long long)j * N1 + y;
            const float2 gp = grad_pair(a.phi, i, i + N1, ih1);
            // cones (j+1, y) and (j, y) at halo rows jx+1 and jx, column yy+1
            const int hr = (jx + 1) * HY + (yy + 1), hl = jx * HY + (yy + 1);
            const float sr = a.somega ? a.somega[(long long)(j + 1) * N1 + y] : s_def;
            const float sl = a.somega ? a.somega[(long long)j * N1 + y] : s_def;
            float2 acc = make_float2(0.f, 0.f);
            float dg = 0.f;
            if (has_now) {
              acc = ff_add(acc, ff_add(ff_mul_f(su[lev][0][hr], sr), ff_mul_f(su[lev][1][hl], sl)));
              dg += sr * sr + sl * sl;
            }
            if (has_prev) {
              acc = ff_add(acc, ff_add(ff_mul_f(su[lp][2][hr], sr), ff_mul_f(su[lp][3][hl], sl)));
              dg += sr * sr + sl * sl;
            }
            const float2 al = a.al[1][i];
            const float2 rhs = ff_add(ff_add(gp, al), acc);
            qv = ff_round(ff_div_f(rhs, 1.f + dg));
            if (write_node && jx >= 1) {
              a.qn[1][i] = qv;
              a.aln[1][i] = ff_add_f(al, ts * grad_minus(gp, qv));
            }
          }
          sq1[lev][e] = qv;
        } else {
          // y-face (t, x, j): x = x0 + f / (TY+1), j = y0 - 1 + f % (TY+1)
          const int f = e - NQ1;
          const int xx = f / (TY + 1), jy = f % (TY + 1);
          const int x = x0 + xx, j = y0 - 1 + jy;
          float qv = 0.f;
          if (x < g.N[0] && j >= 0 && j <= g.N[1] - 2) {
            const long long i = (long long)t * P + (long long)x * N1 + j;
            const float2 gp = grad_pair(a.phi, i, i + 1, ih2);
            // cones (x, j+1) and (x, j) at halo row xx+1, columns jy+1 and jy
            const int hr = (xx + 1) * HY + (jy + 1), hl = (xx + 1) * HY + jy;
            const float sr = a.somega ? a.somega[(long long)x * N1 + j + 1] : s_def;
            const float sl = a.somega ? a.somega[(long long)x * N1 + j] : s_def;
            float2 acc = make_float2(0.f, 0.f);
            float dg = 0.f;
            if (has_now) {
              acc = ff_add(acc, ff_add(ff_mul_f(su[lev][4][hr], sr), ff_mul_f(su[lev][5][hl], sl)));
              dg += sr * sr + sl * sl;
            }
            if (has_prev) {
              acc = ff_add(acc, ff_add(ff_mul_f(su[lp][6][hr], sr), ff_mul_f(su[lp][7][hl], sl)));
              dg += sr * sr + sl * sl;
            }
            const float2 al = a.al[2][i];
            const float2 rhs = ff_add(ff_add(gp, al), acc);
            qv = ff_round(ff_div_f(rhs, 1.f + dg));
            if (write_node && jy >= 1) {
              a.qn[2][i] = qv;
              a.aln[2][i] = ff_add_f(al, ts * grad_minus(gp, qv));
            }
          }
          sq2[lev][f] = qv;
        }
      }
    }
    __syncthreads();
    // ---------------- C: beta of the owned cones at time t-1 ----------------
    if (t - 1 >= ta && t - 1 < tb) {
      const int lp = lev ^ 1;   // node t-1 faces; node t faces at lev
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!own_ok[r]) continue;
        const int xo = lx + 8 * r;   // 0..15
        const int x = x0 + xo, y = y0 + ly;
        const long long i = (long long)(t - 1) * P + (long long)x * N1 + y;
        const bool xl = x >= 1, xr = x <= g.N[0] - 2, yl = y >= 1, yr = y <= g.N[1] - 2;
        float xv[K2 - 1];
        xv[0] = q0p[r];
        // x-faces j = x-1 (row xo) and j = x (row xo+1) of the tile's face list
        xv[1] = xl ? sq1[lp][xo * TY + ly] : 0.f;
        xv[2] = xr ? sq1[lp][(xo + 1) * TY + ly] : 0.f;
        xv[3] = xl ? sq1[lev][xo * TY + ly] : 0.f;
        xv[4] = xr ? sq1[lev][(xo + 1) * TY + ly] : 0.f;
        // y-faces j = y-1 (column ly) and j = y (column ly+1)
        xv[5] = yl ? sq2[lp][xo * (TY + 1) + ly] : 0.f;
        xv[6] = yr ? sq2[lp][xo * (TY + 1) + ly + 1] : 0.f;
        xv[7] = yl ? sq2[lev][xo * (TY + 1) + ly] : 0.f;
        xv[8] = yr ? sq2[lev][xo * (TY + 1) + ly + 1] : 0.f;
        const float s = a.somega ? a.somega[(long long)x * N1 + y] : s_def;
        const float* z = zp[r];
        float inc = (z[0] - 1.f) + xv[0];
        socp = fmaf(inc, inc, socp);
        a.betan[i] = ff_add_f(a.beta[i], ts * inc);
#pragma unroll
        for (int j = 1; j < K2 - 1; ++j) {
          const long long o = (long long)j * n0 + i;
          inc = fmaf(-s, xv[j], z[j]);
          socp = fmaf(inc, inc, socp);
          a.betan[o] = ff_add_f(a.beta[o], ts * inc);
        }
        const long long o = (long long)(K2 - 1) * n0 + i;
        inc = (z[K2 - 1] - 1.f) - xv[0];
        socp = fmaf(inc, inc, socp);
        a.betan[o] = ff_add_f(a.beta[o], ts * inc);
      }
    }
    // the current cone time becomes the previous one
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      q0p[r] = q0c[r];
#pragma unroll
      for (int j = 0; j < K2; ++j) zp[r][j] = zc[r][j];
    }
    __syncthreads();
  }
  if (a.socp_part) {
    // block sum of the beta increments' squares (the eta_P^soc term), FP64 tree
    double v = (double)socp;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double wsum[kThreads / 32];
    if ((tid & 31) == 0) wsum[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double b = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) b += wsum[w];
      a.socp_part[(chunk * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = b;
    }
  }
}

}  // namespace

bool fused2d_supported(const Geo& g) { return g.D == 2; }

long long fused2d_blocks(const Geo& g) {
  const int tchunk = g.T <= 16 ? g.T : 16;
  return (long long)((g.N[0] + TX - 1) / TX) * ((g.N[1] + TY - 1) / TY) * ((g.T + tchunk - 1) / tchunk);
}

void launch_fused2d(const Geo& g, int G, const MxFields& f, const MxFields& fn, double* socp_part,
                    cudaStream_t s, LaunchCounter lc) {
  FusedArgs a;
  for (int d = 0; d < 3; ++d) {
    a.q[d] = f.q[d];
    a.al[d] = f.al[d];
    a.qn[d] = fn.q[d];
    a.aln[d] = fn.al[d];
  }
  a.beta = f.beta;
  a.betan = fn.beta;
  a.phi = f.phi;
  a.somega = f.somega;
  a.ts = 0.f;
  a.tchunk = g.T <= 16 ? g.T : 16;
  a.nchunk = (g.T + a.tchunk - 1) / a.tchunk;
  a.sp = f.sp;
  a.socp_part = socp_part;
  a.socp_per_slot = fused2d_blocks(g);
  a.err = nullptr;
  a.r = nullptr;
  a.c0 = a.c1 = nullptr;
  dim3 grid((unsigned)((g.N[0] + TX - 1) / TX), (unsigned)((g.N[1] + TY - 1) / TY), (unsigned)(a.nchunk * G));
  static std::atomic<unsigned long long> smem_done{0};
  smem_optin((const void*)k_fused2d, kSmemFused, &smem_done);
  k_fused2d<<<grid, kThreads, kSmemFused, s>>>(g, a);
  lc.launched(KID_FUSED);
}

}  // namespace dot

// ---------------------------------------------------------------------------
// v2: the same pass with beta staged through shared memory by TMA.
//
// beta is three quarters of the pass's traffic.  One elected thread loads each
// time step's beta tile -- all 10 components of a 10 x 36 (x, y) window around
// the CTA's 8 x 32 tile -- with one 4-D TMA box into a ring of three buffers, so
// the load for cone time t+1 runs while the CTA computes time t (buffer t-1 is
// still needed by the faces and the beta update).  q, alpha and phi are small and
// read directly.  Requires N_y even (TMA: 16-byte row strides and an even start
// column for 8-byte elements).
namespace dot {
namespace {

#ifndef FUSED_V2_VX
#define FUSED_V2_VX 8
#endif
#ifndef FUSED_V2_THREADS
#define FUSED_V2_THREADS 352
#endif
#ifndef FUSED_V2_TCHUNK
#define FUSED_V2_TCHUNK 16
#endif
constexpr int VX = FUSED_V2_VX, VY = 32;     // owned tile: one cone per thread
constexpr int VHX = VX + 2, VHY = VY + 2;    // cone halo 10 x 34
constexpr int VNH = VHX * VHY;               // 340 cones
constexpr int VBW = VY + 4;                  // beta tile columns: y in [y0-2, y0+34)
constexpr int VNQ1 = (VX + 1) * VY;          // 288 x-faces: j in [x0-1, x0+7], y owned
constexpr int VNQ2 = VX * (VY + 1);          // 264 y-faces: x owned, j in [y0-1, y0+31]
constexpr int kBetaTile = K2 * VHX * VBW;    // 3600 two-floats = 28800 bytes
constexpr int kBetaTileBytes = kBetaTile * 8;
// z of the halo cones: components 1, 2, 5, 6 of cone time t (read by the faces of
// node t) once, components 3, 4, 7, 8 (read by the faces of node t+1) for two
// cone times
constexpr int kOffZ = 3 * kBetaTileBytes;                 // ztn [4][VNH] floats
constexpr int kOffZP = kOffZ + 4 * VNH * 4;               // ztp [2][4][VNH] floats
constexpr int kOffQ1 = kOffZP + 2 * 4 * VNH * 4;          // [2][VNQ1] floats
constexpr int kOffQ2 = kOffQ1 + 2 * VNQ1 * 4;             // [2][VNQ2] floats
constexpr int kOffW1 = kOffQ2 + 2 * VNQ2 * 4;             // [VNQ1] two-float q - alpha/sigma - A phi
constexpr int kOffW2 = kOffW1 + VNQ1 * 8;                 // [VNQ2] two-float
constexpr int kOffBar = (kOffW2 + VNQ2 * 8 + 15) / 16 * 16;
constexpr int kSmemV2 = kOffBar + 64;
static_assert(kOffW1 % 16 == 0, "two-float face arrays are 16-byte aligned");
// 11 warps: one thread per cone of the 10 x 34 halo rectangle (256 owned + 84
// ring cones), so phase A takes one round; 552 faces take two
constexpr int kThreadsV2 = FUSED_V2_THREADS;
static_assert(kThreadsV2 >= VX * VY + 2 * (VX + VY + 2) && kThreadsV2 % 32 == 0, "a thread per halo cone");
constexpr int kMinBlocksV2 = FUSED_V2_MIN_BLOCKS;
// most cone times per CTA (fused2d_tma_tchunk)
constexpr int kTchunkV2 = FUSED_V2_TCHUNK;

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity) { return mbar_wait_bounded(sa(bar), parity); }

__device__ __forceinline__ void issue_beta(const CUtensorMap* tm, float2* dst, uint64_t* bar, int y, int x, int t,
                                           int slot) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(kBetaTileBytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, %7}], [%2];"
      ::"r"(sa(dst)), "l"(tm), "r"(sa(bar)), "r"(y), "r"(x), "r"(t), "r"(0), "r"(slot)
      : "memory");
}

// beta of halo cone (xh, yh) component c in a tile (column yw = yh + 1)
__device__ __forceinline__ float2 bt(const float2* tile, int c, int xh, int yh) {
  return tile[(c * VHX + xh) * VBW + yh + 1];
}

// z components 1..8 of a halo cone into the tiles, from the lane pairs of
// ff2_proj_soc10: (1, 2), (5, 6) -> ztn; (3, 4), (7, 8) -> ztp
__device__ __forceinline__ void put_z(float (*ztn)[VNH], float (*ztp)[VNH], int hc, const ff2* P) {
  const float2 r1 = add2(P[1].h, P[1].l), r2 = add2(P[2].h, P[2].l);
  const float2 r3 = add2(P[3].h, P[3].l), r4 = add2(P[4].h, P[4].l);
  ztn[0][hc] = r1.x;
  ztn[1][hc] = r1.y;
  ztn[2][hc] = r3.x;
  ztn[3][hc] = r3.y;
  ztp[0][hc] = r2.x;
  ztp[1][hc] = r2.y;
  ztp[2][hc] = r4.x;
  ztp[3][hc] = r4.y;
}
__device__ __forceinline__ void put_z0(float (*ztn)[VNH], float (*ztp)[VNH], int hc) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    ztn[v][hc] = 0.f;
    ztp[v][hc] = 0.f;
  }
}
// The q^k values a cone (t, x, y) reads: q_0 at the cone, and the q_1, q_2 faces on
// either side of it on time nodes t (v = 1, 2) and t+1 (v = 3, 4), zero where F
// has no source face.  A thread keeps its cone column for all cone times, and the
// node-(t+1) values of cone t are the node-t values of cone t+1, so per cone time
// it loads q_0 and the node-(t+1) pairs only.
struct ConeQ {
  float x0;
  float2 xb, xd;   // (q_1 left, right), (q_2 left, right) on node t+1
};
__device__ __forceinline__ void load_cone_q(const Geo& g, const FusedArgs& a, int t, int x, int y, ConeQ* c) {
  const int P_ = (int)g.P, N1 = g.N[1];
  const int i = t * P_ + x * N1 + y;
  const bool xl = x >= 1, xr = x <= g.N[0] - 2, yl = y >= 1, yr = y <= g.N[1] - 2;
  c->x0 = a.q[0][i];
  c->xb = make_float2(xl ? a.q[1][i + P_ - N1] : 0.f, xr ? a.q[1][i + P_] : 0.f);
  c->xd = make_float2(yl ? a.q[2][i + P_ - 1] : 0.f, yr ? a.q[2][i + P_] : 0.f);
}
// the node-t pairs (at the first cone time of a chunk)
__device__ __forceinline__ void load_cone_q_node(const Geo& g, const FusedArgs& a, int t, int x, int y, float2* xa,
                                                 float2* xc) {
  const int P_ = (int)g.P, N1 = g.N[1];
  const int i = t * P_ + x * N1 + y;
  const bool xl = x >= 1, xr = x <= g.N[0] - 2, yl = y >= 1, yr = y <= g.N[1] - 2;
  *xa = make_float2(xl ? a.q[1][i - N1] : 0.f, xr ? a.q[1][i] : 0.f);
  *xc = make_float2(yl ? a.q[2][i - 1] : 0.f, yr ? a.q[2][i] : 0.f);
}
// z of a cone from its q^k values and its beta tile entries, in two-float
// arithmetic, as five lane pairs P[0] = (z_0, z_9), P[k] = (z_{2k-1}, z_{2k}).
__device__ __forceinline__ void cone_z(float x0, float2 xa, float2 xb, float2 xc, float2 xd, float s,
                                       const float2* tile, int xh, int yh, ff2* P) {
  const float2 s2 = make_float2(s, s);
  // y = B F q + d - beta/sigma: (1 - x_0, s x_1, ..., s x_8, 1 + x_0) - beta/sigma
  P[0] = ff2_add(two_sum2(make_float2(-x0, x0), make_float2(1.f, 1.f)),
                 ff2_neg(ff2_pack(bt(tile, 0, xh, yh), bt(tile, K2 - 1, xh, yh))));
  P[1] = ff2_add(two_prod2(s2, xa), ff2_neg(ff2_pack(bt(tile, 1, xh, yh), bt(tile, 2, xh, yh))));
  P[2] = ff2_add(two_prod2(s2, xb), ff2_neg(ff2_pack(bt(tile, 3, xh, yh), bt(tile, 4, xh, yh))));
  P[3] = ff2_add(two_prod2(s2, xc), ff2_neg(ff2_pack(bt(tile, 5, xh, yh), bt(tile, 6, xh, yh))));
  P[4] = ff2_add(two_prod2(s2, xd), ff2_neg(ff2_pack(bt(tile, 7, xh, yh), bt(tile, 8, xh, yh))));
  ff2_proj_soc10(P);
}

__device__ __forceinline__ float2 grad_of(float2 a, float2 b, float invh) {
  const float2 dh = two_sum(b.x, -a.x);
  const float dl = (b.y - a.y) + dh.y;
  return make_float2(dh.x * invh, dl * invh);
}

// One space face's update (line 4-5 of Algorithm 2 for q_d, alpha_d at one face):
// rhs = A_d phi + alpha/sigma + sum over the cones reading the face of
// s (z + beta/sigma), q = rhs / (1 + sum s^2), alpha/sigma += tau (A_d phi - q).
// Returns q; *w = q - alpha/sigma - A_d phi (the next residual's face term).
__device__ __forceinline__ float face_update(float2 gp, float2 al, bool has_now, bool has_prev, float2 bnr,
                                             float2 bnl, float2 bpr, float2 bpl, float znr, float znl, float zpr,
                                             float zpl, float sr, float sl, float ts, float2* alnew, float2* w) {
  ff_acc acc = acc_init(gp);
  acc_add(acc, al);
  float zs = 0.f, dg = 0.f;
  if (has_now) {
    acc_add_mul(acc, bnr, sr);
    acc_add_mul(acc, bnl, sl);
    zs += sr * znr + sl * znl;
    dg += sr * sr + sl * sl;
  }
  if (has_prev) {
    acc_add_mul(acc, bpr, sr);
    acc_add_mul(acc, bpl, sl);
    zs += sr * zpr + sl * zpl;
    dg += sr * sr + sl * sl;
  }
  acc_add_f(acc, zs);
  const float den = 1.f + dg;
  const float qv = ff_round(ff_div_f_r(acc_get(acc), den, __frcp_rn(den)));
  const float gm = grad_minus(gp, qv);
  *alnew = ff_add_f(al, ts * gm);
  *w = ff_add_f(ff_neg(*alnew), -gm);
  return qv;
}

__global__ void __launch_bounds__(kThreadsV2, kMinBlocksV2) k_fused2d_tma(const __grid_constant__ CUtensorMap tmb, Geo g,
                                                        FusedArgs a_in) {
  const int slot = blockIdx.z / a_in.nchunk, chunk = blockIdx.z - slot * a_in.nchunk;
  if (!a_in.sp[slot].active) return;
  const FusedArgs a = fused_slot(a_in, g, slot);
  extern __shared__ __align__(128) unsigned char sm[];
  float2* btiles = reinterpret_cast<float2*>(sm);
  float (*ztn)[VNH] = reinterpret_cast<float (*)[VNH]>(sm + kOffZ);
  float (*ztp)[4][VNH] = reinterpret_cast<float (*)[4][VNH]>(sm + kOffZP);
  float (*sq1)[VNQ1] = reinterpret_cast<float (*)[VNQ1]>(sm + kOffQ1);
  float (*sq2)[VNQ2] = reinterpret_cast<float (*)[VNQ2]>(sm + kOffQ2);
  float2* sw1 = reinterpret_cast<float2*>(sm + kOffW1);
  float2* sw2 = reinterpret_cast<float2*>(sm + kOffW2);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kOffBar);

  const int tid = threadIdx.x;
  const bool owner = tid < VX * VY;             // threads 0..255 own a cone column
  const int ly = tid & 31, lx = tid >> 5;       // owned node (x0 + lx, y0 + ly)
  const int x0 = blockIdx.x * VX, y0 = blockIdx.y * VY;
  const int ta = chunk * a.tchunk;
  const int tb = min(g.T, ta + a.tchunk);
  const bool last_chunk = (tb == g.T);
  const int P = (int)g.P, n0 = g.T * P, N1 = g.N[1];
  const float ts = a.ts;
  const float ih0 = (float)g.invh[0], ih1 = (float)g.invh[1], ih2 = (float)g.invh[2];
  const float s_def = 0.70710678118654752f;
  const int xo = x0 + lx, yo = y0 + ly;
  const bool own_ok = owner && xo < g.N[0] && yo < g.N[1];
  const int tstart = ta > 0 ? ta - 1 : 0;
  const int tlast_cone = min(tb, g.T - 1);      // last cone time whose beta tile is loaded

  // this thread's cone column: its owned cone, or one of the 84 halo-ring cones
  // (threads 256..339); the same for every cone time
  int cxh = -1, cyh = -1;
  if (owner) {
    cxh = lx + 1;
    cyh = ly + 1;
  } else if (tid < VNH) {
    int r = tid - VX * VY;
    if (r < VHY) { cxh = 0; cyh = r; }
    else if ((r -= VHY) < VHY) { cxh = VHX - 1; cyh = r; }
    else if ((r -= VHY) < VHX - 2) { cxh = 1 + r; cyh = 0; }
    else { r -= VHX - 2; cxh = 1 + r; cyh = VHY - 1; }
  }
  const int cx = x0 - 1 + cxh, cy = y0 - 1 + cyh, chc = cxh * VHY + cyh;
  const bool cone_ok = cxh >= 0 && cx >= 0 && cy >= 0 && cx < g.N[0] && cy < g.N[1];
  const float cs = (cone_ok && a.somega) ? a.somega[cx * N1 + cy] : s_def;
  // q^k of the cone column (node-t pairs and the next cone time's values), and the
  // owner's potential on node t and alpha_0 / sigma of its cone, loaded a step ahead
  float2 xa = make_float2(0.f, 0.f), xc = make_float2(0.f, 0.f);
  ConeQ cq;
  cq.x0 = 0.f;
  cq.xb = cq.xd = make_float2(0.f, 0.f);
  float2 ph_t = make_float2(0.f, 0.f), ph_n = make_float2(0.f, 0.f), al0 = make_float2(0.f, 0.f);
  if (cone_ok && tstart <= g.T - 1) {
    load_cone_q_node(g, a, tstart, cx, cy, &xa, &xc);
    load_cone_q(g, a, tstart, cx, cy, &cq);
    if (owner && tstart < tb) {
      const int i = tstart * P + xo * N1 + yo;
      ph_t = a.phi[i];
      ph_n = a.phi[i + P];
      al0 = a.al[0][i];
    }
  }

  if (tid == 0) {
    for (int b = 0; b < 3; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bars[b])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned phase[3] = {0u, 0u, 0u};
  bool inflight[3] = {false, false, false};   // meaningful on the issuing thread
  if (tid == 0 && tstart <= tlast_cone) {
    issue_beta(&tmb, btiles + (tstart % 3) * kBetaTile, &bars[tstart % 3], y0 - 2, x0 - 1, tstart, slot);
    inflight[tstart % 3] = true;
  }

  // FP32 z of the owned cone at times t (zc) and t-1 (zp), lane pairs as ff2_proj_soc10
  float2 zc[5], zp[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) zc[k] = zp[k] = make_float2(0.f, 0.f);
  float q0c = 0.f, q0p = 0.f;
  float2 socp = make_float2(0.f, 0.f);
  float2 w0c = make_float2(0.f, 0.f), w0p = make_float2(0.f, 0.f);   // q_0 - alpha_0/sigma - A_0 phi, cones t, t-1
  bool failed = false;

  for (int t = tstart; t <= tb; ++t) {
    const int lev = t & 1, lp = lev ^ 1;
    const int bcur = t % 3, bprev = (t + 2) % 3;
    const float2* tcur = btiles + bcur * kBetaTile;
    const float2* tprev = btiles + bprev * kBetaTile;
    // every thread waits for the tile of cone time t itself; a wait that gives up
    // is made uniform at the barrier after step A
    bool ok = true;
    if (t <= g.T - 1) {
      ok = bar_wait(&bars[bcur], phase[bcur]);
      if (ok) {
        phase[bcur] ^= 1u;
        inflight[bcur] = false;
      }
    }
    // ---------------- A: cones at time t ----------------
    if (t <= g.T - 1 && cxh >= 0) {
      if (cone_ok) {
        ff2 z[5];
        cone_z(cq.x0, xa, cq.xb, xc, cq.xd, cs, tcur, cxh, cyh, z);
        put_z(ztn, ztp[lev], chc, z);
        // the cone before the chunk (t = ta - 1) is updated for the residual only
        if (owner && t < tb) {
          const int i = t * P + xo * N1 + yo;
          const float2 gp = grad_of(ph_t, ph_n, ih0);
          const float2 al = al0;
          // q_0 (diagonal 3): rhs = A_0 phi + alpha_0/sigma + u_9 - u_0 with
          // u = z + beta/sigma (F^*B^* of components 0 and K-1)
          const ff2 u = ff2_add(z[0], ff2_pack(bt(tcur, 0, cxh, cyh), bt(tcur, K2 - 1, cxh, cyh)));
          ff_acc acc = acc_init(gp);
          acc_add(acc, al);
          acc_add(acc, ff2_lane1(u));
          acc_add(acc, ff_neg(ff2_lane0(u)));
          const float qn = ff_round(ff_div_f_r(acc_get(acc), 3.f, 1.f / 3.f));
          const float gm = grad_minus(gp, qn);
          const float2 aln = ff_add_f(al, ts * gm);
          if (t >= ta) {
            a.qn[0][i] = qn;
            a.aln[0][i] = aln;
          }
          q0c = qn;
          w0c = ff_add_f(ff_neg(aln), -gm);   // q - alpha/sigma - A phi
          // the next cone time's potential and alpha_0 / sigma
          ph_t = ph_n;
          if (t + 1 < tb) {
            ph_n = a.phi[i + 2 * P];
            al0 = a.al[0][i + P];
          }
        }
        if (owner) {
#pragma unroll
          for (int k = 0; k < 5; ++k) zc[k] = add2(z[k].h, z[k].l);
        }
        // the next cone time's q^k: node t+1 pairs move down, the rest is loaded now
        xa = cq.xb;
        xc = cq.xd;
        if (t + 1 <= tlast_cone) load_cone_q(g, a, t + 1, cx, cy, &cq);
      } else {
        put_z0(ztn, ztp[lev], chc);
      }
    }
    if (__syncthreads_or(!ok)) { failed = true; break; }
    // prefetch the next cone time's beta into buffer (t+1) % 3 = (t-2) % 3, whose
    // last reader (step C of t-1) every thread has left at the barrier above
    if (tid == 0 && t + 1 <= tlast_cone) {
      const int nb = (t + 1) % 3;
      issue_beta(&tmb, btiles + nb * kBetaTile, &bars[nb], y0 - 2, x0 - 1, t + 1, slot);
      inflight[nb] = true;
    }
    // ---------------- B: faces at time node t ----------------
    const bool write_node = t >= ta && ((t < tb) || (last_chunk && t == g.T));
    if (t >= ta) {
      const bool has_now = t <= g.T - 1, has_prev = t >= 1;
      const float2 z2 = make_float2(0.f, 0.f);
      for (int e = tid; e < VNQ1 + VNQ2; e += kThreadsV2) {
        if (e < VNQ1) {
          const int jx = e / VY, yy = e % VY;
          const int j = x0 - 1 + jx, y = y0 + yy;
          float qv = 0.f;
          float2 wv = z2;
          if (j >= 0 && j <= g.N[0] - 2 && y < g.N[1]) {
            const int i = t * P + j * N1 + y;
            const int xr = jx + 1, xl = jx, yh = yy + 1;
            const float sr = a.somega ? a.somega[(j + 1) * N1 + y] : s_def;
            const float sl = a.somega ? a.somega[j * N1 + y] : s_def;
            float2 aln;
            qv = face_update(grad_pair(a.phi, i, i + N1, ih1), a.al[1][i], has_now, has_prev,
                             has_now ? bt(tcur, 1, xr, yh) : z2, has_now ? bt(tcur, 2, xl, yh) : z2,
                             has_prev ? bt(tprev, 3, xr, yh) : z2, has_prev ? bt(tprev, 4, xl, yh) : z2,
                             ztn[0][xr * VHY + yh], ztn[1][xl * VHY + yh], ztp[lp][0][xr * VHY + yh],
                             ztp[lp][1][xl * VHY + yh], sr, sl, ts, &aln, &wv);
            if (write_node && jx >= 1) {
              a.qn[1][i] = qv;
              a.aln[1][i] = aln;
            }
          }
          sq1[lev][e] = qv;
          sw1[e] = wv;
        } else {
          const int f = e - VNQ1;
          const int xx = f / (VY + 1), jy = f % (VY + 1);
          const int x = x0 + xx, j = y0 - 1 + jy;
          float qv = 0.f;
          float2 wv = z2;
          if (x < g.N[0] && j >= 0 && j <= g.N[1] - 2) {
            const int i = t * P + x * N1 + j;
            const int xh = xx + 1, yr = jy + 1, yl = jy;
            const float sr = a.somega ? a.somega[x * N1 + j + 1] : s_def;
            const float sl = a.somega ? a.somega[x * N1 + j] : s_def;
            float2 aln;
            qv = face_update(grad_pair(a.phi, i, i + 1, ih2), a.al[2][i], has_now, has_prev,
                             has_now ? bt(tcur, 5, xh, yr) : z2, has_now ? bt(tcur, 6, xh, yl) : z2,
                             has_prev ? bt(tprev, 7, xh, yr) : z2, has_prev ? bt(tprev, 8, xh, yl) : z2,
                             ztn[2][xh * VHY + yr], ztn[3][xh * VHY + yl], ztp[lp][2][xh * VHY + yr],
                             ztp[lp][3][xh * VHY + yl], sr, sl, ts, &aln, &wv);
            if (write_node && jy >= 1) {
              a.qn[2][i] = qv;
              a.aln[2][i] = aln;
            }
          }
          sq2[lev][f] = qv;
          sw2[f] = wv;
        }
      }
    }
    __syncthreads();
    // ---------------- C: beta of the owned cone at time t-1 ----------------
    if (own_ok && t - 1 >= ta && t - 1 < tb) {
      const int i = (t - 1) * P + xo * N1 + yo;
      const bool xl = xo >= 1, xr = xo <= g.N[0] - 2, yl = yo >= 1, yr = yo <= g.N[1] - 2;
      const float2 xa = make_float2(xl ? sq1[lp][lx * VY + ly] : 0.f, xr ? sq1[lp][(lx + 1) * VY + ly] : 0.f);
      const float2 xb = make_float2(xl ? sq1[lev][lx * VY + ly] : 0.f, xr ? sq1[lev][(lx + 1) * VY + ly] : 0.f);
      const float2 xc = make_float2(yl ? sq2[lp][lx * (VY + 1) + ly] : 0.f, yr ? sq2[lp][lx * (VY + 1) + ly + 1] : 0.f);
      const float2 xd = make_float2(yl ? sq2[lev][lx * (VY + 1) + ly] : 0.f, yr ? sq2[lev][lx * (VY + 1) + ly + 1] : 0.f);
      const float s = a.somega ? a.somega[xo * N1 + yo] : s_def;
      const int xh = lx + 1, yh = ly + 1;
      const float2 ns2 = make_float2(-s, -s), ts2 = make_float2(ts, ts);
      // increments z - B F q^{k+1} - d, lane pairs as zp
      float2 inc[5];
      inc[0] = add2(sub2(zp[0], make_float2(1.f, 1.f)), make_float2(q0p, -q0p));
      inc[1] = fma2(ns2, xa, zp[1]);
      inc[2] = fma2(ns2, xb, zp[2]);
      inc[3] = fma2(ns2, xc, zp[3]);
      inc[4] = fma2(ns2, xd, zp[4]);
#pragma unroll
      for (int k = 0; k < 5; ++k) socp = fma2(inc[k], inc[k], socp);
      const int c0 = 0, c1 = K2 - 1;
      ff2 B = ff2_add_f(ff2_pack(bt(tprev, c0, xh, yh), bt(tprev, c1, xh, yh)), mul2(ts2, inc[0]));
      a.betan[c0 * n0 + i] = ff2_lane0(B);
      a.betan[c1 * n0 + i] = ff2_lane1(B);
#pragma unroll
      for (int k = 1; k <= 4; ++k) {
        const int j = 2 * k - 1;
        B = ff2_add_f(ff2_pack(bt(tprev, j, xh, yh), bt(tprev, j + 1, xh, yh)), mul2(ts2, inc[k]));
        a.betan[j * n0 + i] = ff2_lane0(B);
        a.betan[(j + 1) * n0 + i] = ff2_lane1(B);
      }
    }
    // the next iteration's residual at the owned node of time t:
    // r = A^*(q - alpha/sigma) - c/sigma - A^*A phi = A^*(q - alpha/sigma - A phi) - c/sigma,
    // with q - alpha/sigma - A phi of the node's faces from steps A and B
    if (a.r && own_ok && write_node) {
      const int i = t * P + xo * N1 + yo;
      const int p = xo * N1 + yo;
      ff_acc acc{0.f, 0.f};
      if (t >= 1) acc_add_mul(acc, w0p, ih0);
      if (t < g.T) acc_add_mul(acc, w0c, -ih0);
      // faces j = x - 1 / x (and y - 1 / y); the slots beyond the walls hold zero
      acc_add_mul(acc, sw1[lx * VY + ly], ih1);
      acc_add_mul(acc, sw1[(lx + 1) * VY + ly], -ih1);
      acc_add_mul(acc, sw2[lx * (VY + 1) + ly], ih2);
      acc_add_mul(acc, sw2[lx * (VY + 1) + ly + 1], -ih2);
      if (t == 0) acc_add(acc, ff_neg(ff_mul(a.c0[p], a.isg)));
      if (t == g.T) acc_add(acc, ff_mul(a.c1[p], a.isg));
      a.r[i] = acc.h + acc.c;
    }
    q0p = q0c;
    w0p = w0c;
#pragma unroll
    for (int k = 0; k < 5; ++k) zp[k] = zc[k];
    // no barrier here: step A of t+1 writes only ztn and ztp[lev of t+1] (read by
    // step B of t, which every thread finished before step C) and registers; step B
    // of t+1, which overwrites the faces step C reads, follows the barrier after A
  }
  if (failed) {
    // a tile load did not complete in time: wait (bounded) for the loads this
    // CTA still has in flight, then report through the error flag
    if (tid == 0) {
      for (int b = 0; b < 3; ++b)
        if (inflight[b]) bar_wait(&bars[b], phase[b]);
      atomicExch(a.err, 1);
    }
    return;
  }
  if (a.socp_part) {
    double v = (double)socp.x + (double)socp.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double wsum[kThreadsV2 / 32];
    if ((tid & 31) == 0) wsum[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double b = 0.0;
      for (int w = 0; w < kThreadsV2 / 32; ++w) b += wsum[w];
      a.socp_part[(chunk * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = b;
    }
  }
}

}  // namespace
}  // namespace dot

namespace dot {

bool fused2d_tma_supported(const Geo& g) { return g.D == 2 && g.N[1] % 2 == 0; }

// Cone times per CTA for a batch of G solves of grid g: kTchunkV2, halved (down to 2)
// while the launch would have fewer than 256 CTAs, so that small grids still occupy
// the GPU (measured: 128^2 x 32 80 -> 60 us per launch with 8, 32^2 x 16 66 -> 19 us
// with 2); each chunk recomputes one cone time before it (1/tchunk extra work).
int fused2d_tma_tchunk(const Geo& g, int G) {
  const long long tiles = (long long)((g.N[0] + VX - 1) / VX) * ((g.N[1] + VY - 1) / VY) * G;
  int tc = g.T <= kTchunkV2 ? g.T : kTchunkV2;
  while (tc > 2 && tiles * ((g.T + tc - 1) / tc) < 256) tc = (tc + 1) / 2;
  return tc;
}

long long fused2d_tma_blocks(const Geo& g, int G) {
  const int tchunk = fused2d_tma_tchunk(g, G);
  return (long long)((g.N[0] + VX - 1) / VX) * ((g.N[1] + VY - 1) / VY) * ((g.T + tchunk - 1) / tchunk);
}

bool launch_fused2d_tma(const Geo& g, int G, const MxFields& f, const MxFields& fn, double* socp_part, int* err,
                        bool residual, cudaStream_t s, LaunchCounter lc) {
  FusedArgs a;
  for (int d = 0; d < 3; ++d) {
    a.q[d] = f.q[d];
    a.al[d] = f.al[d];
    a.qn[d] = fn.q[d];
    a.aln[d] = fn.al[d];
  }
  a.beta = f.beta;
  a.betan = fn.beta;
  a.phi = f.phi;
  a.somega = f.somega;
  a.ts = 0.f;
  a.tchunk = fused2d_tma_tchunk(g, G);
  a.nchunk = (g.T + a.tchunk - 1) / a.tchunk;
  a.sp = f.sp;
  a.socp_part = socp_part;
  a.socp_per_slot = fused2d_tma_blocks(g, G);
  a.err = err;
  a.r = residual ? f.r : nullptr;
  a.c0 = f.c0;
  a.c1 = f.c1;
  a.isg = make_float2(0.f, 0.f);
  // beta as a 5-D tensor of 8-byte elements: (y, x, t, component, slot)
  CUtensorMap tm;
  const cuuint64_t dims[5] = {(cuuint64_t)g.N[1], (cuuint64_t)g.N[0], (cuuint64_t)g.T, (cuuint64_t)K2,
                              (cuuint64_t)G};
  const cuuint64_t str[4] = {(cuuint64_t)g.N[1] * 8, (cuuint64_t)g.P * 8, (cuuint64_t)g.T * g.P * 8,
                             (cuuint64_t)K2 * g.T * g.P * 8};
  const cuuint32_t box[5] = {VBW, VHX, 1, K2, 1};
  if (!encode_tensor_map(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, f.beta, dims, str, box)) return false;
  static std::atomic<unsigned long long> smem_done{0};
  smem_optin((const void*)k_fused2d_tma, kSmemV2, &smem_done);
  dim3 grid((unsigned)((g.N[0] + VX - 1) / VX), (unsigned)((g.N[1] + VY - 1) / VY), (unsigned)(a.nchunk * G));
  k_fused2d_tma<<<grid, kThreadsV2, kSmemV2, s>>>(tm, g, a);
  lc.launched(KID_FUSED);
  return true;
}

}  // namespace dot
