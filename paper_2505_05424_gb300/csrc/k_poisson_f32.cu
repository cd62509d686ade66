// k_poisson_f32.cu -- FP32 Poisson solve of the mixed path: the orthonormal
// DCT-II along every axis as a dense per-axis GEMM, division by the Neumann
// eigenvalues (zero mode set to 0), DCT-III back (Sec. 4, phi-subproblem).
#include "dot_mixed.cuh"

namespace dot {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kPad = 68;

// Y[o][k][i] = sum_m C[k][m] X[o][m][i] (or C^T); 256 threads, 4x4 outputs each.
__global__ void __launch_bounds__(256) k_axis_f32(const float* __restrict__ C, const float* __restrict__ X,
                                                  float* __restrict__ Y, int M, long long inner, long long ncol,
                                                  int transpose) {
  __shared__ __align__(16) float As[kBK][kPad];  // As[m][k]
  __shared__ __align__(16) float Bs[kBK][kPad];  // Bs[m][col]
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const long long col0 = (long long)blockIdx.x * kBN;
  const int k0 = blockIdx.y * kBM;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int m0 = 0; m0 < M; m0 += kBK) {
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int e = tid + 256 * jj;
      const int r = e / kBK, c = e % kBK;
      const int k = k0 + r, m = m0 + c;
      float v = 0.f;
      if (k < M && m < M) v = transpose ? C[(long long)m * M + k] : C[(long long)k * M + m];
      As[c][r] = v;
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int e = tid + 256 * jj;
      int r, c;
      if (inner == 1) { c = e / kBK; r = e % kBK; } else { r = e / kBN; c = e % kBN; }
      const int m = m0 + r;
      const long long col = col0 + c;
      float v = 0.f;
      if (m < M && col < ncol) {
        const long long o = col / inner, i = col - o * inner;
        v = X[(o * M + m) * inner + i];
      }
      Bs[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int k = k0 + ty * 4 + a;
    if (k >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const long long col = col0 + tx * 4 + b;
      if (col >= ncol) continue;
      const long long o = col / inner, i = col - o * inner;
      Y[(o * M + k) * inner + i] = acc[a][b];
    }
  }
}

__global__ void k_scale_lambda_f32(Geo g, MxPoisson ps, float* v) {
  const long long n = (long long)(g.T + 1) * g.P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (i == 0) { v[0] = 0.f; continue; }
    const int kt = (int)(i / g.P);
    const long long p = i - (long long)kt * g.P;
    float lam = ps.lam[0][kt];
    for (int d = 0; d < g.D; ++d) lam += ps.lam[1 + d][coord(g, p, d)];
    v[i] = v[i] / lam;
  }
}

void axis(const Geo& g, int a, const float* C, int transpose, const float* X, float* Y, cudaStream_t s,
          LaunchCounter lc) {
  const long long nn = (long long)(g.T + 1) * g.P;
  const int M = a == 0 ? g.T + 1 : g.N[a - 1];
  const long long inner = a == 0 ? g.P : g.sst[a - 1];
  const long long ncol = nn / M;
  dim3 grid((unsigned)((ncol + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM));
  k_axis_f32<<<grid, 256, 0, s>>>(C, X, Y, M, inner, ncol, transpose);
  lc.launched(KID_DCT_AXIS);
}

}  // namespace

void launch_poisson_mx(const Geo& g, const MxPoisson& ps, const float* src, float* dst, cudaStream_t s,
                       LaunchCounter lc) {
  float* w[2] = {ps.w1, ps.w2};
  int ci = 0;
  axis(g, 0, ps.C[0], 0, src, w[0], s, lc);
  for (int a = 1; a <= g.D; ++a) {
    axis(g, a, ps.C[a], 0, w[ci], w[1 - ci], s, lc);
    ci = 1 - ci;
  }
  const long long nn = (long long)(g.T + 1) * g.P;
  long long blocks = (nn + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scale_lambda_f32<<<(int)blocks, 256, 0, s>>>(g, ps, w[ci]);
  lc.launched(KID_SCALE);
  for (int a = 0; a <= g.D; ++a) {
    float* out = (a == g.D) ? dst : w[1 - ci];
    axis(g, a, ps.C[a], 1, w[ci], out, s, lc);
    ci = 1 - ci;
  }
}

}  // namespace dot
