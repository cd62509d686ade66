// dot_mixed.cuh -- fields and Poisson-solver tables of the mixed-precision path.
#pragma once
#include "dot_internal.cuh"

namespace dot {

struct MxFields {
  float* q[kMaxD + 1];     // q_0: T*P; q_d: (T+1)*P padded
  float2* al[kMaxD + 1];   // two-float multipliers, same shapes as q
  float2* beta;            // K * T * P two-float multipliers
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
};

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
  float* w1;                      // (T+1)*P scratch
  float* w2;                      // (T+1)*P scratch
  int* err;                       // set by a tensor-core pass whose pipeline wait timed out
  bool use_tc;                    // run eligible spatial passes on the tensor cores
};

// Shared memory of the fused time-axis pass (C_t and two 64-column tiles).
size_t tsolve_smem_bytes(const Geo& g);

// src -> dst (src is preserved), FP32 in and out.
void launch_poisson_mx(const Geo& g, const MxPoisson& ps, const float* src, float* dst, cudaStream_t s,
                       LaunchCounter lc);
// Refined solve of f.b (+ f.blo) into out (two-float); f.b is overwritten.
// have_bsum: f.bsum already holds the partial sums of b (k_assemble_b writes them).
constexpr int kBsumParts = 608;
void launch_poisson_refined_mx(const Geo& g, const MxFields& f, const MxPoisson& ps, float2* out,
                               bool have_bsum, cudaStream_t s, LaunchCounter lc);
void launch_iterate_mx(const Geo& g, const MxFields& f, const MxPoisson& ps, double sigma, double tau,
                       cudaStream_t s, LaunchCounter lc);
// Stopping-measure sums.  socp_part (nullable): per-block sums of |z - BFq - d|^2
// written by the fused kernel; when given, they replace the z-based term.
void launch_kkt_mx(const Geo& g, const MxFields& f, double* partials, double* out, const double* socp_part,
                   int nsocp, cudaStream_t s, LaunchCounter lc);
void launch_assemble_b_mx(const Geo& g, const MxFields& f, double sigma, cudaStream_t s, LaunchCounter lc);

// Fused lines 3-6 for D = 2 (k_fused2d.cu): reads q, alpha, beta of f, writes
// those of fn; phi, somega from f.  socp_part: fused2d_blocks(g) doubles.
bool fused2d_supported(const Geo& g);
long long fused2d_blocks(const Geo& g);
void launch_fused2d(const Geo& g, const MxFields& f, const MxFields& fn, double sigma, double tau,
                    double* socp_part, cudaStream_t s, LaunchCounter lc);
// The same pass with beta staged by TMA (needs N_y even); socp_part:
// fused2d_tma_blocks(g) doubles.  Returns false if the tensor map cannot be built.
bool fused2d_tma_supported(const Geo& g);
long long fused2d_tma_blocks(const Geo& g);
bool launch_fused2d_tma(const Geo& g, const MxFields& f, const MxFields& fn, double sigma, double tau,
                        double* socp_part, int* err, cudaStream_t s, LaunchCounter lc);
long long kkt_partials_len_mx(const Geo& g);

}  // namespace dot
