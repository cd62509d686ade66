// k_fused3d.cu -- lines 3-6 of Algorithm 2 for D = 3 in two passes over the
// mixed-path state, and the next iteration's lines 1-2 residual.
//
// The D = 2 pass (k_fused2d.cu) recomputes a one-cone halo around each tile so
// that z never reaches memory.  In three dimensions that halo would cost ~1.8
// projections per cone and a beta tile of ~200 KB per time step, so z (FP32, K
// components) is stored once and read back from L2:
//   k_cone3 : per cone, z = Pi_K(B F q^k + d - beta^k/sigma) and the q_0, alpha_0
//             update (diagonal 3, Proposition 3.2) into the k+1 set;
//   k_face3 : a CTA owns a 4 x 4 x 32 tile of cells and a chunk of time nodes and
//             marches along time.  At node t it updates q_d, alpha_d of every space
//             face the tile's cones read (lines 4-5), keeping q^{k+1} and
//             w = q - alpha/sigma - A phi of those faces in shared memory; then beta of
//             the tile's cones at time t-1 (line 6) from the faces of nodes t-1 and
//             t; then the residual r = A^*(q - alpha/sigma - A phi) - c/sigma at the
//             tile's nodes of time t, which the next iteration's Poisson solve reads
//             (the warm start of lines 1-2).
// q, alpha and beta are double-buffered (iteration k read, k+1 written), so the
// faces on a tile's lower boundary, which both neighbouring tiles compute, are
// written by one of them only.  Per element: two-float y, projection, face
// right-hand sides and multiplier updates (ffloat.cuh), FP32 q and z, as in the D = 2
// pass.
#include <cmath>

#include "dot_internal.cuh"
#include "dot_mixed.cuh"
#include "ffloat.cuh"

namespace dot {
namespace {

constexpr int K3 = 14;                     // 4D + 2 for D = 3
constexpr int FX = 4, FY = 4, FZ = 32;     // owned tile: cells along axes 1, 2, 3 (axis 3 contiguous)
constexpr int NFX = (FX + 1) * FY * FZ;    // 640 faces of axis 1 per time node: j in [x0-1, x0+3]
constexpr int NFY = FX * (FY + 1) * FZ;    // 640 faces of axis 2: j in [y0-1, y0+3]
constexpr int NFZ = FX * FY * (FZ + 1);    // 528 faces of axis 3: j in [z0-1, z0+31]
constexpr int NF3 = NFX + NFY + NFZ;       // 1808
constexpr int kCells3 = FX * FY * FZ;      // 512
constexpr int kThreads3 = 256;             // two cells per thread
static_assert(kCells3 == 2 * kThreads3 && FZ == 32 && FY == 4, "cell and face numbering below");
constexpr int kTchunk3 = 8;                // time nodes written per CTA (more CTAs than SMs x 5 on 64^3 x 32)
constexpr int kConeThreads = 256;
constexpr float kSdef = 0.70710678118654752f;   // sqrt(omega/2) for omega = 1

struct Fused3Args {
  // iteration k (read)
  const float* q[4];
  const float2* al[4];
  const float2* beta;
  // iteration k+1 (written)
  float* qn[4];
  float2* aln[4];
  float2* betan;
  float* z;              // K * T * P, written by k_cone3, read by k_face3
  const float2* phi;     // phi^{k+1}
  const float* somega;   // sqrt(omega/2) per cell, or nullptr
  const SlotParam* sp;
  float* r;              // residual of the next iteration's lines 1-2, or nullptr
  const float2* c0;
  const float2* c1;
  float ih[4];           // 1/h per axis (0 = time)
  int tchunk, nchunk;
};

// The arguments of slot b of a batch.
__device__ __forceinline__ Fused3Args slot3(Fused3Args a, const Geo& g, int b) {
  if (b == 0) return a;
  const long long nn = (long long)(g.T + 1) * g.P, n0 = (long long)g.T * g.P;
  a.q[0] += b * n0;
  a.al[0] += b * n0;
  a.qn[0] += b * n0;
  a.aln[0] += b * n0;
  for (int d = 1; d < 4; ++d) {
    a.q[d] += b * nn;
    a.al[d] += b * nn;
    a.qn[d] += b * nn;
    a.aln[d] += b * nn;
  }
  a.beta += b * K3 * n0;
  a.betan += b * K3 * n0;
  a.z += b * K3 * n0;
  a.phi += b * nn;
  if (a.somega) a.somega += b * g.P;
  if (a.r) {
    a.r += b * nn;
    a.c0 += b * g.P;
    a.c1 += b * g.P;
  }
  return a;
}

// A phi along an axis from the two-float potential as an unevaluated pair.
__device__ __forceinline__ float2 grad3(const float2* phi, int i, int j, float invh) {
  const float2 a = phi[i], b = phi[j];
  const float2 dh = two_sum(b.x, -a.x);
  const float dl = (b.y - a.y) + dh.y;
  return make_float2(dh.x * invh, dl * invh);
}

__device__ __forceinline__ float grad_minus3(float2 g, float q) { return (g.x - q) + g.y; }

// Line 3 and lines 4-5 on the time faces.  One thread per cone (t, x): the
// projection input y = B F q^k + d - beta^k/sigma in two-float arithmetic, z stored
// rounded to FP32, then q_0, alpha_0 of the cone from rhs = A_0 phi + alpha_0/sigma +
// u_{K-1} - u_0 with u = z + beta/sigma (F^*B^* of components 0 and K-1), diagonal 3.
__global__ void __launch_bounds__(kConeThreads) k_cone3(Geo g, Fused3Args a_in) {
  const int slot = blockIdx.y;
  if (!a_in.sp[slot].active) return;
  const Fused3Args a = slot3(a_in, g, slot);
  const float ts = a_in.sp[slot].tau;
  const int P = (int)g.P, n0 = g.T * P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x) {
    const int t = (int)fdiv((unsigned)i, g.fP);
    const int p = i - t * P;
    // F q^k: q_0 at the cone, then per axis the faces left / right of the cell on
    // time nodes t and t+1 (zero where F has no source face)
    float x[K3 - 1];
    x[0] = a.q[0][i];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int xd = coord(g, p, d);
      const int st = (int)g.sst[d];
      const float* qd = a.q[1 + d];
      const bool lo = xd >= 1, hi = xd <= g.N[d] - 2;
      x[1 + 4 * d] = lo ? qd[i - st] : 0.f;
      x[2 + 4 * d] = hi ? qd[i] : 0.f;
      x[3 + 4 * d] = lo ? qd[i + P - st] : 0.f;
      x[4 + 4 * d] = hi ? qd[i + P] : 0.f;
    }
    const float s = a.somega ? a.somega[p] : kSdef;
    float2 y[K3];
    y[0] = ff_add(two_sum(-x[0], 1.f), ff_neg(a.beta[i]));
#pragma unroll
    for (int j = 1; j < K3 - 1; ++j) y[j] = ff_add(two_prod(s, x[j]), ff_neg(a.beta[j * n0 + i]));
    y[K3 - 1] = ff_add(two_sum(x[0], 1.f), ff_neg(a.beta[(K3 - 1) * n0 + i]));
    ff_proj_soc<K3>(y);
    float zr[K3];
#pragma unroll
    for (int j = 0; j < K3; ++j) {
      zr[j] = ff_round(y[j]);
      a.z[j * n0 + i] = zr[j];
    }
    const float2 gp = grad3(a.phi, i, i + P, a.ih[0]);
    const float2 db = ff_add(a.beta[(K3 - 1) * n0 + i], ff_neg(a.beta[i]));
    const float2 al = a.al[0][i];
    float2 rhs = ff_add(gp, ff_add(al, db));
    rhs = ff_add_f(rhs, zr[K3 - 1] - zr[0]);
    const float qn = ff_round(ff_div_f(rhs, 3.f));
    a.qn[0][i] = qn;
    a.aln[0][i] = ff_add_f(al, ts * grad_minus3(gp, qn));
  }
}


// Face e of a tile's face set at one time node.  Faces are numbered axis by axis:
// axis 1 as [j 0..4][y 0..3][z 0..31], axis 2 as [x 0..3][j 0..4][z 0..31], axis 3 as
// [x 0..3][y 0..3][j 0..32], where local face j lies between cells j-1 and j of the
// tile (j = 0 is the face below the tile's first cell, which the neighbouring tile
// owns).  Gives the axis, the cell (X, Y, Z) whose upper face it is along that axis
// (X, Y or Z may be -1) and the local j.
struct FaceLoc {
  int d, X, Y, Z, jl;
};
__device__ __forceinline__ FaceLoc face_loc(int e, int x0, int y0, int z0) {
  FaceLoc f;
  if (e < NFX) {
    const int jx = e >> 7, rem = e & 127;
    f.d = 0; f.jl = jx;
    f.X = x0 - 1 + jx; f.Y = y0 + (rem >> 5); f.Z = z0 + (rem & 31);
  } else if (e < NFX + NFY) {
    const int k = e - NFX, cx = k / ((FY + 1) * FZ), rem = k - cx * ((FY + 1) * FZ), jy = rem >> 5;
    f.d = 1; f.jl = jy;
    f.X = x0 + cx; f.Y = y0 - 1 + jy; f.Z = z0 + (rem & 31);
  } else {
    const int k = e - NFX - NFY, cxy = k / (FZ + 1), jz = k - cxy * (FZ + 1);
    f.d = 2; f.jl = jz;
    f.X = x0 + (cxy >> 2); f.Y = y0 + (cxy & 3); f.Z = z0 - 1 + jz;
  }
  return f;
}
// Slots of the faces below (lo) and above (hi) cell (cx, cy, cz) of the tile along each axis.
__device__ __forceinline__ int slot_lo(int d, int cx, int cy, int cz) {
  return d == 0 ? (cx * FY + cy) * FZ + cz
       : d == 1 ? NFX + (cx * (FY + 1) + cy) * FZ + cz
                : NFX + NFY + (cx * FY + cy) * (FZ + 1) + cz;
}
__device__ __forceinline__ int slot_hi(int d, int cx, int cy, int cz) {
  return d == 0 ? slot_lo(0, cx, cy, cz) + FY * FZ : d == 1 ? slot_lo(1, cx, cy, cz) + FZ : slot_lo(2, cx, cy, cz) + 1;
}

// w = q - alpha/sigma - A_0 phi of the time face of cone (c, p) from the k+1 values
// k_cone3 wrote (the same operations as its update, so the same value).
__device__ __forceinline__ float2 w_time(const Fused3Args& a, int ic, int P) {
  const float2 gp = grad3(a.phi, ic, ic + P, a.ih[0]);
  const float gm = grad_minus3(gp, a.qn[0][ic]);
  return ff_add_f(ff_neg(a.aln[0][ic]), -gm);
}

__global__ void __launch_bounds__(kThreads3, 5) k_face3(Geo g, Fused3Args a_in) {
  const int slot = blockIdx.z / a_in.nchunk, chunk = blockIdx.z - slot * a_in.nchunk;
  if (!a_in.sp[slot].active) return;
  const Fused3Args a = slot3(a_in, g, slot);
  const float ts = a_in.sp[slot].tau;
  const float2 isg = a_in.sp[slot].isg;
  __shared__ float sq[2][NF3];    // q^{k+1} of the tile's faces on time nodes of parity 0 / 1
  __shared__ float2 sw[NF3];      // w = q - alpha/sigma - A phi of the faces of the current node

  const int tid = threadIdx.x;
  const int nty = (g.N[1] + FY - 1) / FY;
  const int x0 = blockIdx.y * FX, y0 = (blockIdx.x % nty) * FY, z0 = (blockIdx.x / nty) * FZ;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const int P = (int)g.P, n0 = g.T * P;
  const int ta = chunk * a.tchunk, tb = min(g.T, ta + a.tchunk);
  const bool last_chunk = tb == g.T;

  // this thread's two cells
  int cp[2];
  bool cok[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int c = tid + k * kThreads3, cz = c & 31, cxy = c >> 5;
    const int X = x0 + (cxy >> 2), Y = y0 + (cxy & 3), Z = z0 + cz;
    cok[k] = X < N0 && Y < N1 && Z < N2;
    cp[k] = (X * N1 + Y) * N2 + Z;
  }
  // w of the time face below the first node (cone ta - 1)
  float2 w0p[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  if (a.r && ta >= 1) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (cok[k]) w0p[k] = w_time(a, (ta - 1) * P + cp[k], P);
  }

  for (int t = ta; t <= tb; ++t) {
    const bool write_node = t < tb || (last_chunk && t == g.T);
    float* sqc = sq[t & 1];
    // ---------------- lines 4-5 at the space faces of node t ----------------
    for (int e = tid; e < NF3; e += kThreads3) {
      const FaceLoc f = face_loc(e, x0, y0, z0);
      const int jd = f.d == 0 ? f.X : f.d == 1 ? f.Y : f.Z;       // the face's coordinate along its axis
      const int Nd = f.d == 0 ? N0 : f.d == 1 ? N1 : N2;
      const bool valid = f.X >= 0 && f.Y >= 0 && f.Z >= 0 && f.X < N0 && f.Y < N1 && f.Z < N2 && jd <= Nd - 2;
      float qv = 0.f;
      float2 wv = make_float2(0.f, 0.f);
      if (valid) {
        const int p = (f.X * N1 + f.Y) * N2 + f.Z;
        const int s = f.d == 0 ? N1 * N2 : f.d == 1 ? N2 : 1;   // stride of the face's axis
        const int i = t * P + p;
        // this axis's fields, selected without indexing the argument arrays at run time
        const float2* ald = f.d == 0 ? a.al[1] : f.d == 1 ? a.al[2] : a.al[3];
        const float ihd = f.d == 0 ? a.ih[1] : f.d == 1 ? a.ih[2] : a.ih[3];
        const float2 gp = grad3(a.phi, i, i + s, ihd);
        const float s_r = a.somega ? a.somega[p + s] : kSdef;
        const float s_l = a.somega ? a.somega[p] : kSdef;
        const float2 al = ald[i];
        float2 mb = al;               // alpha/sigma + sum_c s_c beta_c/sigma
        float zs = 0.f, dg = 0.f;     // sum_c s_c z_c, sum_c s_c^2
        const int cb = 1 + 4 * f.d;
        if (t <= g.T - 1) {
          const int o1 = cb * n0 + i + s, o2 = (cb + 1) * n0 + i;
          mb = ff_add(mb, ff_add(ff_mul_f(a.beta[o1], s_r), ff_mul_f(a.beta[o2], s_l)));
          zs += s_r * a.z[o1] + s_l * a.z[o2];
          dg += s_r * s_r + s_l * s_l;
        }
        if (t >= 1) {
          const int o3 = (cb + 2) * n0 + i - P + s, o4 = (cb + 3) * n0 + i - P;
          mb = ff_add(mb, ff_add(ff_mul_f(a.beta[o3], s_r), ff_mul_f(a.beta[o4], s_l)));
          zs += s_r * a.z[o3] + s_l * a.z[o4];
          dg += s_r * s_r + s_l * s_l;
        }
        const float2 rhs = ff_add_f(ff_add(gp, mb), zs);
        qv = ff_round(ff_div_f(rhs, 1.f + dg));
        const float gm = grad_minus3(gp, qv);
        const float2 aln = ff_add_f(al, ts * gm);
        wv = ff_add_f(ff_neg(aln), -gm);
        if (write_node && f.jl >= 1) {
          float* qnd = f.d == 0 ? a.qn[1] : f.d == 1 ? a.qn[2] : a.qn[3];
          float2* alnd = f.d == 0 ? a.aln[1] : f.d == 1 ? a.aln[2] : a.aln[3];
          qnd[i] = qv;
          alnd[i] = aln;
        }
      }
      sqc[e] = qv;
      sw[e] = wv;
    }
    __syncthreads();
    const float* sqp = sq[(t & 1) ^ 1];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!cok[k]) continue;
      const int c = tid + k * kThreads3, cz = c & 31, cxy = c >> 5, cx = cxy >> 2, cy = cxy & 3;
      const int p = cp[k];
      // ---------------- line 6: beta of cone t-1 ----------------
      if (t - 1 >= ta) {
        const int ic = (t - 1) * P + p;
        float x[K3 - 1];
        x[0] = a.qn[0][ic];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int lo = slot_lo(d, cx, cy, cz), hi = slot_hi(d, cx, cy, cz);
          x[1 + 4 * d] = sqp[lo];   // faces of node t-1 (zero beyond a wall)
          x[2 + 4 * d] = sqp[hi];
          x[3 + 4 * d] = sqc[lo];   // faces of node t
          x[4 + 4 * d] = sqc[hi];
        }
        const float sc = a.somega ? a.somega[p] : kSdef;
        a.betan[ic] = ff_add_f(a.beta[ic], ts * ((a.z[ic] - 1.f) + x[0]));
#pragma unroll
        for (int j = 1; j < K3 - 1; ++j) {
          const int o = j * n0 + ic;
          a.betan[o] = ff_add_f(a.beta[o], ts * fmaf(-sc, x[j], a.z[o]));
        }
        const int o = (K3 - 1) * n0 + ic;
        a.betan[o] = ff_add_f(a.beta[o], ts * ((a.z[o] - 1.f) - x[0]));
      }
      // ---------------- the next iteration's residual at node t ----------------
      if (a.r && write_node) {
        const float2 w0c = t < g.T ? w_time(a, t * P + p, P) : make_float2(0.f, 0.f);
        ff_acc acc{0.f, 0.f};
        if (t >= 1) acc_add_mul(acc, w0p[k], a.ih[0]);
        if (t < g.T) acc_add_mul(acc, w0c, -a.ih[0]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          acc_add_mul(acc, sw[slot_lo(d, cx, cy, cz)], a.ih[1 + d]);
          acc_add_mul(acc, sw[slot_hi(d, cx, cy, cz)], -a.ih[1 + d]);
        }
        if (t == 0) acc_add(acc, ff_neg(ff_mul(a.c0[p], isg)));
        if (t == g.T) acc_add(acc, ff_mul(a.c1[p], isg));
        a.r[t * P + p] = acc.h + acc.c;
        w0p[k] = w0c;
      }
    }
    __syncthreads();
  }
}

}  // namespace

bool fused3d_supported(const Geo& g) { return g.D == 3; }

void launch_fused3d(const Geo& g, int G, const MxFields& f, const MxFields& fn, bool residual, cudaStream_t s,
                    LaunchCounter lc) {
  Fused3Args a;
  for (int d = 0; d < 4; ++d) {
    a.q[d] = f.q[d];
    a.al[d] = f.al[d];
    a.qn[d] = fn.q[d];
    a.aln[d] = fn.al[d];
    a.ih[d] = (float)g.invh[d];
  }
  a.beta = f.beta;
  a.betan = fn.beta;
  a.z = f.z;
  a.phi = f.phi;
  a.somega = f.somega;
  a.sp = f.sp;
  a.r = residual ? f.r : nullptr;
  a.c0 = f.c0;
  a.c1 = f.c1;
  a.tchunk = g.T < kTchunk3 ? g.T : kTchunk3;
  a.nchunk = (g.T + a.tchunk - 1) / a.tchunk;
  const long long n0 = (long long)g.T * g.P;
  long long nb = (n0 + kConeThreads - 1) / kConeThreads;
  if (nb > 152LL * 16) nb = 152LL * 16;
  k_cone3<<<dim3((unsigned)nb, (unsigned)G), kConeThreads, 0, s>>>(g, a);
  lc.launched(KID_PROJECT);
  const unsigned ntx = (unsigned)((g.N[0] + FX - 1) / FX), nty = (unsigned)((g.N[1] + FY - 1) / FY),
                 ntz = (unsigned)((g.N[2] + FZ - 1) / FZ);
  k_face3<<<dim3(nty * ntz, ntx, (unsigned)(a.nchunk * G)), kThreads3, 0, s>>>(g, a);
  lc.launched(KID_FACE3);
}

}  // namespace dot
