// dot_mixed.cuh -- fields and Poisson-solver tables of the mixed-precision path.
#pragma once
#include "dot_internal.cuh"

namespace dot {

// Per-solve scalars of a batch, read by the kernels from device memory so that a
// captured launch sequence serves every penalty value.
struct SlotParam {
  float2 isg;      // 1/sigma (two-float): scales c in the b-assembly
  float2 sg;       // sigma (two-float): turns the stored alpha/sigma, beta/sigma into alpha, beta
  float2 rescale;  // sigma_old / sigma_new, applied to the stored multipliers before the next
                   // iteration after a penalty change (1: nothing to do)
  float tau;       // step length tau of the multiplier updates
  int active;      // 0: the slot holds no solve; its blocks return at once
  int assemble;    // 1: the first iteration of the next check period assembles this slot's
                   // lines 1-2 residual (a new or rewritten state, a penalty change); 0: it
                   // keeps the residual the fused kernel left in f.r
};

// A batch holds G solves of one grid.  Every per-solve field below is stored as
// G consecutive copies (slot_view gives slot b's pointers); the DCT tables and
// eigenvalues are shared.
struct MxFields {
  float* q[kMaxD + 1];     // q_0: T*P; q_d: (T+1)*P padded
  float2* al[kMaxD + 1];   // alpha / sigma (two-float), same shapes as q
  float2* beta;            // beta / sigma (two-float), K * T * P
  float* z;                // K * T * P
  float2* phi;             // (T+1)*P two-float potential
  float* b;                // (T+1)*P right-hand side, high part; reused for the correction delta
  float* blo;              // (T+1)*P right-hand side, low part (b = b + blo as a two-float)
  float* phi1;             // (T+1)*P first Poisson solve
  float* r;                // (T+1)*P refinement residual
  double* bsum;            // kBsumParts FP64 partial sums of b, then mean(b) as a two-float
  const float2* c0;        // P: c on the first time plane (densities, two-float)
  const float2* c1;        // P: -c on the last time plane (rho1 densities, two-float)
  const double* m0;        // P: rho0 densities (FP64, for the reductions)
  const double* m1;        // P: rho1 densities
  const float* omega;      // P or nullptr
  const float* somega;     // P or nullptr: sqrt(omega/2)
  const SlotParam* sp;     // G slot parameters
};

constexpr int kBsumStride = 1024;   // doubles per slot in bsum: partial sums, then mean(b)

// Fields of slot b of a batch.
__host__ __device__ inline MxFields slot_view(MxFields f, const Geo& g, int b) {
  if (b == 0) return f;
  const long long nn = (long long)(g.T + 1) * g.P, n0 = (long long)g.T * g.P, P = g.P;
  f.q[0] += b * n0;
  f.al[0] += b * n0;
  // constant indices (the bound is the array size), so that a kernel's copy of the
  // fields stays in registers instead of local memory
#pragma unroll
  for (int d = 0; d < kMaxD; ++d) {
    if (d < g.D) {
      f.q[1 + d] += b * nn;
      f.al[1 + d] += b * nn;
    }
  }
  f.beta += b * g.K * n0;
  if (f.z) f.z += b * g.K * n0;
  f.phi += b * nn;
  f.b += b * nn;
  f.blo += b * nn;
  f.phi1 += b * nn;
  f.r += b * nn;
  f.bsum += b * kBsumStride;
  f.c0 += b * P;
  f.c1 += b * P;
  f.m0 += b * P;
  f.m1 += b * P;
  if (f.omega) f.omega += b * P;
  if (f.somega) f.somega += b * P;
  return f;
}

// Poisson solver of the mixed path: per-axis DCT matrices (FP32, and their
// TF32 hi/lo split for the tensor-core GEMMs), 1D eigenvalues, scratch.
struct MxPoisson {
  const float* C[kMaxD + 1];      // M x M orthonormal DCT-II, row k = frequency
  const float* CT[kMaxD + 1];     // its transpose (DCT-III)
  const float* Chi[kMaxD + 1];    // TF32 split of C: C = Chi + Clo
  const float* Clo[kMaxD + 1];
  const float* CThi[kMaxD + 1];   // TF32 split of C^T
  const float* CTlo[kMaxD + 1];
  const float* lam[kMaxD + 1];    // M, 1D Neumann eigenvalues
  // time-axis tables for the tensor-core flow, rows padded to time_ld(g) floats:
  // C hi, C lo, C^T hi, C^T lo (nullptr: the SIMT time pass is used)
  const float* tpad[4];
  float* w1;                      // poisson_scratch_elems(g) floats per solve of a batch
  float* w2;
  int* err;                       // set by a tensor-core pass whose pipeline wait timed out
  bool use_tc;                    // run eligible passes on the tensor cores
};

// Row stride of the padded time axis (a multiple of 4 floats: 16-byte TMA rows).
inline int time_ld(const Geo& g) { return (g.T + 1 + 3) / 4 * 4; }
// Whether the whole Poisson solve runs on the tensor cores (the flow a batch of
// several solves needs).
bool poisson_tc_flow(const Geo& g, const MxPoisson& ps);
// Scratch elements per solve for w1 / w2.
size_t poisson_scratch_elems(const Geo& g);

// Shared memory of the fused time-axis pass (C_t and two 64-column tiles).
size_t tsolve_smem_bytes(const Geo& g);

// src -> dst (src is preserved), FP32 in and out, for G solves of grid g stored
// one after the other (G > 1 needs poisson_tc_flow).  accum (nullable, two-float,
// slot-strided like phi): when the tensor-core flow runs, its last pass adds the
// result into accum instead of writing dst and the call returns true.
bool launch_poisson_mx(const Geo& g, int G, const MxPoisson& ps, const float* src, float* dst, cudaStream_t s,
                       LaunchCounter lc, float2* accum);
// Refined solve of f.b (+ f.blo) into out (two-float, slot-strided like phi) for
// the G slots of a batch; f.b is overwritten.  have_bsum: f.bsum already holds
// the partial sums of b.
constexpr int kBsumParts = 608;   // most partial sums per slot
void launch_poisson_refined_mx(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, float2* out,
                               bool have_bsum, cudaStream_t s, LaunchCounter lc);
// Multiply the stored alpha/sigma and beta/sigma of every slot whose rescale
// factor is not 1 by that factor (after a penalty change).
void launch_rescale_mx(const Geo& g, int G, const MxFields& f, cudaStream_t s, LaunchCounter lc);
// Line 2 from a residual already in f.r (written by the fused cone kernel of the
// previous iteration): one solve, phi += delta.
void launch_solve_residual_mx(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, cudaStream_t s,
                              LaunchCounter lc);
// Lines 1-2 of an iteration: b-assembly fused with the warm-start residual
// (b never stored), one solve, phi += delta.
void launch_assemble_solve_mx(const Geo& g, int G, const MxFields& f, const MxPoisson& ps, cudaStream_t s,
                              LaunchCounter lc);
// Stopping-measure sums of every active slot into out[G][R_NSLOTS].  socp_part
// (nullable): per-block sums of |z - BFq - d|^2 written by the fused kernel,
// nsocp per slot; when given, they replace the z-based term.
void launch_kkt_mx(const Geo& g, int G, const MxFields& f, double* partials, double* out,
                   const double* socp_part, int nsocp, cudaStream_t s, LaunchCounter lc);

// Fused lines 3-6 for D = 2 (k_fused2d.cu) for every active slot: reads q, alpha,
// beta of f, writes those of fn; phi, somega, sp from f.  socp_part:
// fused2d_blocks(g) doubles per slot.
bool fused2d_supported(const Geo& g);
long long fused2d_blocks(const Geo& g);
void launch_fused2d(const Geo& g, int G, const MxFields& f, const MxFields& fn, double* socp_part,
                    cudaStream_t s, LaunchCounter lc);
// The same pass with beta staged by TMA (needs N_y even); socp_part:
// fused2d_tma_blocks(g, G) doubles per slot (the time chunking depends on the batch size).  Returns false if the tensor map cannot
// be built.
bool fused2d_tma_supported(const Geo& g);
long long fused2d_tma_blocks(const Geo& g, int G);
// residual: also write the next iteration's lines 1-2 residual into f.r (see
// launch_solve_residual_mx).
bool launch_fused2d_tma(const Geo& g, int G, const MxFields& f, const MxFields& fn, double* socp_part, int* err,
                        bool residual, cudaStream_t s, LaunchCounter lc);
// Fused lines 3-6 for D = 3 (k_fused3d.cu) for every active slot: z and q_0, alpha_0
// by one pass over the cones, then q_d, alpha_d, beta by a time-marching pass over
// tiles of cells; reads q, alpha, beta of f, writes those of fn; f.z is scratch.
// residual: also write the next iteration's lines 1-2 residual into f.r.
bool fused3d_supported(const Geo& g);
void launch_fused3d(const Geo& g, int G, const MxFields& f, const MxFields& fn, bool residual, cudaStream_t s,
                    LaunchCounter lc);
// KKT partial-sum scratch (doubles) per slot.
long long kkt_partials_len_mx(const Geo& g);

}  // namespace dot
