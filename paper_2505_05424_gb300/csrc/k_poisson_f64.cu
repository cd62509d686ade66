// k_poisson_f64.cu -- FP64 Poisson solve A^*A phi = b on rge(A^*) (Sec. 4: the
// phi-subproblem of Algorithm 2).  A^*A is the Neumann Laplacian of the node
// grid; the orthonormal DCT-II along every axis diagonalises it with eigenvalues
// sum_a (4/h_a^2) sin^2(pi k_a / (2 M_a)).  Each per-axis transform is a dense
// GEMM  Y[o][k][i] = sum_m C[k][m] X[o][m][i]  run on the FP64 tensor path
// (mma.sync m8n8k4 .f64, which GB300 executes about 4x faster than FP64 FMA).
#include "dot_internal.cuh"

namespace dot {
namespace {

constexpr int kBM = 64;   // rows of C (output frequencies) per CTA
constexpr int kBN = 64;   // columns (o, i) per CTA
constexpr int kBK = 16;   // reduction chunk
constexpr int kAPad = 20; // padded row length of the C tile (2-way bank pattern)
constexpr int kBPad = 72; // padded row length of the X tile

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// Y = C (or C^T) applied along an axis of length M with `inner` contiguous
// elements after it; ncol = outer * inner columns.  128 threads: warp w owns the
// 32x32 sub-tile (rows 32*(w>>1), cols 32*(w&1)) as 4x4 fragments of 8x8.
__global__ void __launch_bounds__(128) k_axis_dmma(const double* __restrict__ C, const double* __restrict__ X,
                                                   double* __restrict__ Y, int M, long long inner,
                                                   long long ncol, int transpose, FastDiv finner) {
  __shared__ double As[kBM][kAPad];
  __shared__ double Bs[kBK][kBPad];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long col0 = (long long)blockIdx.x * kBN;
  const int k0 = blockIdx.y * kBM;
  const int rbase = 32 * (warp >> 1), cbase = 32 * (warp & 1);
  double acc[4][4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;

  for (int m0 = 0; m0 < M; m0 += kBK) {
    // C tile: 64 x 16
#pragma unroll
    for (int jj = 0; jj < (kBM * kBK) / 128; ++jj) {
      const int e = tid + 128 * jj;
      const int r = e / kBK, c = e % kBK;
      const int k = k0 + r, m = m0 + c;
      double v = 0.0;
      if (k < M && m < M) v = transpose ? C[(long long)m * M + k] : C[(long long)k * M + m];
      As[r][c] = v;
    }
    // X tile: 16 x 64
#pragma unroll
    for (int jj = 0; jj < (kBK * kBN) / 128; ++jj) {
      const int e = tid + 128 * jj;
      int r, c;
      if (inner == 1) { c = e / kBK; r = e % kBK; } else { r = e / kBN; c = e % kBN; }
      const int m = m0 + r;
      const long long col = col0 + c;
      double v = 0.0;
      if (m < M && col < ncol) {
        const long long o = fdiv((unsigned)col, finner), i = col - o * inner;
        v = X[(o * M + m) * inner + i];
      }
      Bs[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) af[a] = As[rbase + 8 * a + (lane >> 2)][kk + (lane & 3)];
#pragma unroll
      for (int b = 0; b < 4; ++b) bf[b] = Bs[kk + (lane & 3)][cbase + 8 * b + (lane >> 2)];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dmma(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
    }
    __syncthreads();
  }
  // D fragment: row = lane >> 2, cols 2*(lane & 3) + {0, 1}
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int k = k0 + rbase + 8 * a + (lane >> 2);
    if (k >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long col = col0 + cbase + 8 * b + 2 * (lane & 3) + h;
        if (col >= ncol) continue;
        const long long o = fdiv((unsigned)col, finner), i = col - o * inner;
        Y[(o * M + k) * inner + i] = acc[a][b][h];
      }
    }
  }
}

// phi_hat /= lambda(k); the zero mode (k = 0 on every axis) is set to 0 exactly.
__global__ void k_scale_lambda(Geo g, DctTables64 t, double* v) {
  const long long n = (long long)(g.T + 1) * g.P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (i == 0) { v[0] = 0.0; continue; }
    const int kt = plane_of(g, i);
    const long long p = i - (long long)kt * g.P;
    double lam = t.lam[0][kt];
    for (int d = 0; d < g.D; ++d) lam += t.lam[1 + d][coord(g, p, d)];
    v[i] = v[i] / lam;
  }
}

void axis_transform(const Geo& g, int axis, const double* C, int transpose, const double* X, double* Y,
                    cudaStream_t s, LaunchCounter lc) {
  long long n_nodes = (long long)(g.T + 1) * g.P;
  int M = axis == 0 ? g.T + 1 : g.N[axis - 1];
  long long inner = axis == 0 ? g.P : g.sst[axis - 1];
  long long ncol = n_nodes / M;
  dim3 grid((unsigned)((ncol + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM));
  k_axis_dmma<<<grid, 128, 0, s>>>(C, X, Y, M, inner, ncol, transpose, make_fastdiv((unsigned)inner));
  lc.launched(KID_DCT_AXIS);
}

}  // namespace

void launch_poisson_f64(const Geo& g, const DctTables64& t, double* b, double* w1, double* phi, cudaStream_t s,
                        LaunchCounter lc) {
  double* bufs[2] = {b, w1};
  int ci = 0;
  for (int a = 0; a <= g.D; ++a) {
    axis_transform(g, a, t.C[a], 0, bufs[ci], bufs[1 - ci], s, lc);
    ci = 1 - ci;
  }
  long long n = (long long)(g.T + 1) * g.P;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scale_lambda<<<(int)blocks, 256, 0, s>>>(g, t, bufs[ci]);
  lc.launched(KID_SCALE);
  for (int a = 0; a <= g.D; ++a) {
    double* dst = (a == g.D) ? phi : bufs[1 - ci];
    axis_transform(g, a, t.C[a], 1, bufs[ci], dst, s, lc);
    ci = 1 - ci;
  }
}

}  // namespace dot
