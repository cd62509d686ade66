// k_poisson_f32.cu -- the mixed-path Poisson solve A^*A phi = b on rge(A^*)
// (Sec. 4, phi-subproblem of Algorithm 2): orthonormal DCT-II along every axis,
// division by the Neumann eigenvalues with the zero mode set to 0, DCT-III back.
//
// Data flow ("rotated" passes): every spatial pass transforms the innermost axis
// of its input and writes that axis outermost, so every pass is a K-major GEMM:
//   2D  [t][x][y] -y-> [ky][t][x] -x-> [kx][ky][t] -t-> [t][kx][ky]
//       -ky^T-> [y][t][kx] -kx^T (rows along y)-> [t][x][y]
//   3D  [t][x][y][z] -z-> -y-> -x-> [kx][ky][kz][t] -t-> [t][kx][ky][kz]
//       -kz^T-> -ky^T-> [y][z][t][kx] -kx^T (rows along (y,z))-> [t][x][y][z]
// Tensor-core flow (every axis on tcgen05, k_dct_tc.cu, 3xTF32): the last forward
// spatial pass writes the time rows padded to ldt = 4*ceil((T+1)/4) floats, the
// time axis runs as two passes (DCT-II with the eigenvalue scaling in its
// epilogue, then DCT-III), and a batch of G solves of one grid is transformed in
// the same passes (the group index is carried outermost through every layout).
// SIMT flow (one solve; axes the tensor-core pass cannot take): the spatial passes
// run on the kernel below, in FP32 with the same output layouts, and the time axis
// is one fused pass per column of spatial frequencies: DCT-II, scale, DCT-III.
#include <cstring>

#include "dot_mixed.cuh"
#include "dot_tc.cuh"

namespace dot {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kPad = 68;

// SIMT rotated pass.  Rows r of the input are contiguous K-vectors.
// mode 0: row r -> Out[k*R + r];  mode 1: row (a, b) -> Out[b*K*A + k*A + a].
__global__ void __launch_bounds__(256) k_rot_pass_f32(const float* __restrict__ Bm, const float* __restrict__ X,
                                                      float* __restrict__ Y, int K, long long R, int mode, int A,
                                                      int Bd, FastDiv fA) {
  __shared__ __align__(16) float Ws[kBK][kPad];   // Ws[j][k] = Bm[k][j]
  __shared__ __align__(16) float Xs[kBK][kPad];   // Xs[j][row]
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const long long row0 = (long long)blockIdx.x * kBN;
  const int k0 = blockIdx.y * kBM;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int j0 = 0; j0 < K; j0 += kBK) {
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int e = tid + 256 * jj;
      const int r = e / kBK, c = e % kBK;
      const int k = k0 + r, j = j0 + c;
      Ws[c][r] = (k < K && j < K) ? Bm[(long long)k * K + j] : 0.f;
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int e = tid + 256 * jj;
      const int c = e / kBK, r = e % kBK;     // consecutive threads read consecutive j
      const long long row = row0 + c;
      const int j = j0 + r;
      long long src = -1;
      if (row < R && j < K) {
        if (mode == 0) {
          src = row * K + j;
        } else {
          // row enumerates (b, a) with a fastest: a = row % A, b = row / A
          const long long b = fdiv((unsigned)row, fA), a = row - b * A;
          src = (a * Bd + b) * K + j;
        }
      }
      Xs[r][c] = src >= 0 ? X[src] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 w = *reinterpret_cast<const float4*>(&Ws[kk][ty * 4]);
      const float4 x = *reinterpret_cast<const float4*>(&Xs[kk][tx * 4]);
      const float wv[4] = {w.x, w.y, w.z, w.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wv[a], xv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int k = k0 + ty * 4 + a;
    if (k >= K) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const long long row = row0 + tx * 4 + b;
      if (row >= R) continue;
      long long dst;
      if (mode == 0) {
        dst = (long long)k * R + row;
      } else {
        const long long bb = fdiv((unsigned)row, fA), aa = row - bb * A;
        dst = bb * (long long)K * A + (long long)k * A + aa;
      }
      Y[dst] = acc[a][b];
    }
  }
}

// Time axis: X = [S][M] (M = T+1 innermost) -> Y = [M][S]:
//   Y[:, s] = C_t^T diag(1/lambda(., s)) C_t X[s, :]   (lambda(0, 0) -> zero mode).
// 64 columns s per block.  C_t (zero-padded to Mp = 16*ceil(M/16)), the tile and
// its transform live in shared memory; thread (tk, ts) owns rows tk + 16i and the
// four columns 4ts..4ts+3, so each shared load feeds several FMAs.
template <int R>
__global__ void __launch_bounds__(256) k_tsolve_f32(Geo g, const float* __restrict__ Ct,
                                                    const float* __restrict__ lam_t, MxPoisson ps,
                                                    const float* __restrict__ X, float* __restrict__ Y) {
  extern __shared__ __align__(16) float sm[];
  const int M = g.T + 1;
  constexpr int Mp = 16 * R;
  constexpr int XS = 65;          // odd row stride of the input tile: conflict-free transposed fill
  const long long S = g.P;
  float* C = sm;                  // Mp*Mp, C[k*Mp + t]
  float* xt = C + Mp * Mp;        // Mp*XS: xt[t*XS + s]
  float* yt = xt + Mp * XS;       // Mp*64: yt[k*64 + s]
  const long long s0 = (long long)blockIdx.x * 64;
  for (int e = threadIdx.x; e < Mp * Mp; e += blockDim.x) {
    const int k = e / Mp, t = e % Mp;
    C[e] = (k < M && t < M) ? Ct[k * M + t] : 0.f;
  }
  // the tile's 64 columns are 64*M contiguous floats: read them linearly
  const long long ncol = (S - s0) < 64 ? (S - s0) : 64;
  for (int e = threadIdx.x; e < 64 * M; e += blockDim.x) {
    const int s = e / M, t = e - s * M;
    xt[t * XS + s] = s < ncol ? X[s0 * M + e] : 0.f;
  }
  for (int e = threadIdx.x; e < (Mp - M) * 64; e += blockDim.x) xt[(M + e / 64) * XS + e % 64] = 0.f;
  __syncthreads();
  const int tk = threadIdx.x >> 4, ts = threadIdx.x & 15;
  float acc[R][4];
  // forward DCT-II along t
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
  for (int t = 0; t < Mp; ++t) {
    const float* xr = &xt[t * XS + 4 * ts];
    const float b0 = xr[0], b1 = xr[1], b2 = xr[2], b3 = xr[3];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float a = C[(tk + 16 * i) * Mp + t];
      acc[i][0] = fmaf(a, b0, acc[i][0]);
      acc[i][1] = fmaf(a, b1, acc[i][1]);
      acc[i][2] = fmaf(a, b2, acc[i][2]);
      acc[i][3] = fmaf(a, b3, acc[i][3]);
    }
  }
  // scale by 1/lambda(k, s); the zero mode (k = 0, s = 0) is set to 0
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const long long col = s0 + 4 * ts + j;
    float lsp = 0.f;
    for (int d = 0; d < g.D; ++d) lsp += ps.lam[1 + d][coord(g, col < S ? col : 0, d)];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int k = tk + 16 * i;
      const float lam = (k < M ? lam_t[k] : 1.f) + lsp;
      yt[k * 64 + 4 * ts + j] = (k == 0 && col == 0) ? 0.f : acc[i][j] / lam;
    }
  }
  __syncthreads();
  // inverse DCT-III along t: out[t][s] = sum_k C[k][t] yt[k][s]
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
  for (int k = 0; k < Mp; ++k) {
    const float4 b = *reinterpret_cast<const float4*>(&yt[k * 64 + 4 * ts]);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float a = C[k * Mp + tk + 16 * i];
      acc[i][0] = fmaf(a, b.x, acc[i][0]);
      acc[i][1] = fmaf(a, b.y, acc[i][1]);
      acc[i][2] = fmaf(a, b.z, acc[i][2]);
      acc[i][3] = fmaf(a, b.w, acc[i][3]);
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int t = tk + 16 * i;
    if (t >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long col = s0 + 4 * ts + j;
      if (col < S) Y[(long long)t * S + col] = acc[i][j];
    }
  }
}

// One spatial pass of length K over total elements n (one solve): tensor cores
// when possible, else the SIMT kernel.
void spatial_pass(const MxPoisson& ps, int axis, bool inverse, const float* X, float* Y, int K, long long n,
                  int mode, int A, int Bd, cudaStream_t s, LaunchCounter lc) {
  const long long R = n / K;
  if (ps.use_tc && K % 4 == 0 && tc_pass_supported(K)) {
    TcPass p;
    std::memset(&p, 0, sizeof(p));
    p.X = X;
    p.ldx = K;
    p.Bhi = inverse ? ps.CThi[axis] : ps.Chi[axis];
    p.Blo = inverse ? ps.CTlo[axis] : ps.Clo[axis];
    p.ldb = K;
    p.out = Y;
    p.K = K;
    p.err = ps.err;
    if (mode == 0) {
      p.mode = TC_ROWS_FLAT;
      p.R = R;
      p.A = (int)R;
      p.M = 1;
      p.ldo = 1;
    } else {
      p.mode = TC_ROWS_A;
      p.A = A;
      p.Bd = Bd;
      p.G = 1;
    }
    if (launch_tc_pass(p, s)) {
      lc.launched(KID_DCT_TC);
      return;
    }
  }
  const float* Bm = inverse ? ps.CT[axis] : ps.C[axis];
  dim3 grid((unsigned)((R + kBN - 1) / kBN), (unsigned)((K + kBM - 1) / kBM));
  k_rot_pass_f32<<<grid, 256, 0, s>>>(Bm, X, Y, K, R, mode, A, Bd, make_fastdiv((unsigned)(A > 0 ? A : 1)));
  lc.launched(KID_DCT_AXIS);
}

}  // namespace

size_t tsolve_smem_bytes(const Geo& g) {
  const size_t Mp = ((size_t)g.T + 1 + 15) / 16 * 16;
  return (Mp * Mp + Mp * 65 + Mp * 64) * sizeof(float);
}

template <int R>
void launch_tsolve_r(const Geo& g, const MxPoisson& ps, const float* X, float* Y, cudaStream_t s) {
  const size_t sm = tsolve_smem_bytes(g);
  static std::atomic<unsigned long long> smem_done{0};
  smem_optin((const void*)k_tsolve_f32<R>, 220 * 1024, &smem_done);
  k_tsolve_f32<R><<<(unsigned)((g.P + 63) / 64), 256, sm, s>>>(g, ps.C[0], ps.lam[0], ps, X, Y);
}

// the time-axis pass, specialised on the number of 16-row groups of the padded axis
void launch_tsolve(const Geo& g, const MxPoisson& ps, const float* X, float* Y, cudaStream_t s) {
  switch ((g.T + 1 + 15) / 16) {
    case 1: launch_tsolve_r<1>(g, ps, X, Y, s); break;
    case 2: launch_tsolve_r<2>(g, ps, X, Y, s); break;
    case 3: launch_tsolve_r<3>(g, ps, X, Y, s); break;
    case 4: launch_tsolve_r<4>(g, ps, X, Y, s); break;
    case 5: launch_tsolve_r<5>(g, ps, X, Y, s); break;
    case 6: launch_tsolve_r<6>(g, ps, X, Y, s); break;
    case 7: launch_tsolve_r<7>(g, ps, X, Y, s); break;
    case 8: launch_tsolve_r<8>(g, ps, X, Y, s); break;
    case 9: launch_tsolve_r<9>(g, ps, X, Y, s); break;
    default: launch_tsolve_r<10>(g, ps, X, Y, s); break;
  }
}

// The tensor-core flow applies when every axis is within the tcgen05 pass's
// range and the spatial rows have 16-byte strides.
bool poisson_tc_flow(const Geo& g, const MxPoisson& ps) {
  if (!ps.use_tc || !ps.tpad[0] || !tc_pass_supported(g.T + 1)) return false;
  for (int d = 0; d < g.D; ++d)
    if (!tc_pass_supported(g.N[d]) || g.N[d] % 4 != 0) return false;
  return true;
}

size_t poisson_scratch_elems(const Geo& g) {
  const size_t nn = (size_t)(g.T + 1) * g.P;
  const size_t padded = (size_t)g.P * time_ld(g);
  return nn > padded ? nn : padded;
}

namespace {

bool tc_pass(const MxPoisson& ps, TcPass p, int axis, bool inverse, cudaStream_t s, LaunchCounter lc) {
  p.Bhi = inverse ? ps.CThi[axis] : ps.Chi[axis];
  p.Blo = inverse ? ps.CTlo[axis] : ps.Clo[axis];
  p.ldb = p.K;
  p.err = ps.err;
  if (!launch_tc_pass(p, s)) return false;
  lc.launched(KID_DCT_TC);
  return true;
}

// The tensor-core flow for G solves stored one after the other.
bool poisson_tc(const Geo& g, int G, const MxPoisson& ps, const float* src, float* dst, cudaStream_t s,
                LaunchCounter lc, float2* accum) {
  const long long nn = (long long)(g.T + 1) * g.P;
  const int M = g.T + 1, ldt = time_ld(g);
  float* w[2] = {ps.w1, ps.w2};
  const float* cur = src;
  int nx = 0;
  // forward spatial passes, innermost axis first; the last one (axis 1) pads the time rows
  for (int a = g.D; a >= 1; --a) {
    TcPass p;
    std::memset(&p, 0, sizeof(p));
    const int K = g.N[a - 1];
    p.X = cur;
    p.ldx = K;
    p.out = w[nx];
    p.K = K;
    p.mode = TC_ROWS_FLAT;
    p.R = (long long)G * nn / K;
    p.A = (int)(nn / K);
    p.M = a == 1 ? M : 1;
    p.ldo = a == 1 ? ldt : 1;
    if (!tc_pass(ps, p, a, false, s, lc)) return false;
    cur = w[nx];
    nx ^= 1;
  }
  // time axis: DCT-II + eigenvalue scale (rows keep their place), then DCT-III
  {
    TcPass p;
    std::memset(&p, 0, sizeof(p));
    p.X = cur;
    p.ldx = ldt;
    p.Bhi = ps.tpad[0];
    p.Blo = ps.tpad[1];
    p.ldb = ldt;
    p.out = w[nx];
    p.K = M;
    p.mode = TC_KEEP;
    p.R = (long long)G * g.P;
    p.ldo = ldt;
    p.geo = &g;
    for (int a = 0; a <= g.D; ++a) p.lam[a] = ps.lam[a];
    p.err = ps.err;
    if (!launch_tc_pass(p, s)) return false;
    lc.launched(KID_SCALE);
    cur = w[nx];
    nx ^= 1;
    p.X = cur;
    p.Bhi = ps.tpad[2];
    p.Blo = ps.tpad[3];
    p.out = w[nx];
    p.mode = TC_ROWS_FLAT;
    p.A = (int)g.P;
    p.M = 1;
    p.ldo = 1;
    p.geo = nullptr;
    if (!launch_tc_pass(p, s)) return false;
    lc.launched(KID_SCALE);
    cur = w[nx];
    nx ^= 1;
  }
  // inverse spatial passes, innermost axis first; the last one (axis 1) runs with
  // rows along the flattened trailing spatial axes so it lands in [t][x][...]
  for (int a = g.D; a >= 1; --a) {
    const bool last = (a == 1);
    const int K = g.N[a - 1];
    TcPass p;
    std::memset(&p, 0, sizeof(p));
    p.X = cur;
    p.ldx = K;
    p.out = last ? dst : w[nx];
    p.K = K;
    if (!last) {
      p.mode = TC_ROWS_FLAT;
      p.R = (long long)G * nn / K;
      p.A = (int)(nn / K);
      p.M = 1;
      p.ldo = 1;
    } else {
      p.mode = TC_ROWS_A;
      p.A = (int)(g.P / K);
      p.Bd = M;
      p.G = G;
      p.accum = accum;
    }
    if (!tc_pass(ps, p, a, true, s, lc)) return false;
    cur = p.out;
    nx ^= 1;
  }
  return true;
}

}  // namespace

bool launch_poisson_mx(const Geo& g, int G, const MxPoisson& ps, const float* src, float* dst, cudaStream_t s,
                       LaunchCounter lc, float2* accum) {
  if (poisson_tc_flow(g, ps) && poisson_tc(g, G, ps, src, dst, s, lc, accum)) return accum != nullptr;
  // SIMT flow (one solve)
  const long long n = (long long)(g.T + 1) * g.P;
  float* w[2] = {ps.w1, ps.w2};
  int ci = -1;   // index of the buffer holding the current field, -1 = src
  auto cur = [&]() -> const float* { return ci < 0 ? src : w[ci]; };
  auto next = [&]() { return ci < 0 ? 0 : 1 - ci; };
  for (int a = g.D; a >= 1; --a) {
    const int nx = next();
    spatial_pass(ps, a, false, cur(), w[nx], g.N[a - 1], n, 0, 0, 0, s, lc);
    ci = nx;
  }
  {
    const int nx = next();
    launch_tsolve(g, ps, cur(), w[nx], s);
    lc.launched(KID_SCALE);
    ci = nx;
  }
  for (int a = g.D; a >= 1; --a) {
    const bool last = (a == 1);
    float* out = last ? dst : w[next()];
    const int K = g.N[a - 1];
    const int mode = last ? 1 : 0;
    const int A = last ? (int)(g.P / K) : 0;
    const int Bd = last ? g.T + 1 : 0;
    spatial_pass(ps, a, true, cur(), out, K, n, mode, A, Bd, s, lc);
    if (!last) ci = next();
  }
  return false;
}

}  // namespace dot
