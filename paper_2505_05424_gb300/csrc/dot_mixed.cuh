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
  float* b;                // (T+1)*P right-hand side; reused for the correction delta
  float* phi1;             // (T+1)*P first Poisson solve
  float* r;                // (T+1)*P refinement residual
  const float* m0f;        // P masses (FP32, for b)
  const float* m1f;
  const double* m0;        // P masses (FP64, for the reductions)
  const double* m1;
  const float* omega;      // P or nullptr
  const float* somega;     // P or nullptr: sqrt(omega/2)
};

// Poisson solver of the mixed path: per-axis DCT matrices (FP32, and their
// TF32 hi/lo split for the tensor-core GEMMs), 1D eigenvalues, scratch.
struct MxPoisson {
  const float* C[kMaxD + 1];      // M x M, row k = frequency
  const float* lam[kMaxD + 1];    // M
  float* w1;                      // (T+1)*P scratch
  float* w2;                      // (T+1)*P scratch
};

// src -> dst (src is preserved), FP32 in and out.
void launch_poisson_mx(const Geo& g, const MxPoisson& ps, const float* src, float* dst, cudaStream_t s,
                       LaunchCounter lc);
// Refined solve of f.b into out (two-float); f.b is overwritten.
void launch_poisson_refined_mx(const Geo& g, const MxFields& f, const MxPoisson& ps, float2* out,
                               cudaStream_t s, LaunchCounter lc);
void launch_iterate_mx(const Geo& g, const MxFields& f, const MxPoisson& ps, double sigma, double tau,
                       cudaStream_t s, LaunchCounter lc);
void launch_kkt_mx(const Geo& g, const MxFields& f, double* partials, double* out, cudaStream_t s,
                   LaunchCounter lc);
long long kkt_partials_len_mx(const Geo& g);

}  // namespace dot
