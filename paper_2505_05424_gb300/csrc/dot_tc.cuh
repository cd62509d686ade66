// dot_tc.cuh -- tensor-core (tcgen05) DCT pass of the mixed-path Poisson solve.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "dot_internal.cuh"

namespace dot {

// The tcgen05 pass handles axis lengths 1 <= K <= 4096: each CTA computes up to
// 256 output columns in one TMEM accumulator, longer axes use several column
// tiles.  Rows of X and of the tables are stored with strides that are multiples
// of 4 floats (16-byte TMA row strides).
bool tc_pass_supported(int K);

enum TcMode { TC_ROWS_FLAT = 0, TC_ROWS_A = 1, TC_KEEP = 2 };

// One pass (see k_dct_tc.cu for the output layouts of the three modes).
struct TcPass {
  const float* X;       // input rows of K values, row stride ldx
  int ldx;
  const float* Bhi;     // K x K table (row k = output frequency), row stride ldb, TF32 split
  const float* Blo;
  int ldb;
  float* out;
  int K;
  int mode;             // TcMode
  long long R;          // ROWS_FLAT, KEEP: total rows
  int A;                // ROWS_FLAT: rows per group; ROWS_A: extent of a
  int Bd;               // ROWS_A: extent of b
  int G;                // ROWS_A: groups
  int M, ldo;           // ROWS_FLAT: runs of M rows written with stride ldo; KEEP: output row stride
  const Geo* geo;       // KEEP: grid of one group (rows r map to in-plane index r mod P)
  const float* lam[4];  // KEEP: eigenvalues, lam[0] along the transformed axis
  float2* accum;        // ROWS_A (nullable): add the result into this two-float field (same
                        // layout as out) instead of writing out
  int* err;             // set by a CTA whose pipeline wait timed out
  unsigned extra_tx;    // self-test only (dot_selftest_pipeline_timeout): bytes each stage's
                        // barrier expects beyond what its loads deliver; 0 otherwise
};
// Returns false when the pass cannot run on the tensor cores (unsupported K,
// misaligned strides or pointers, tensor maps that cannot be encoded).
bool launch_tc_pass(const TcPass& p, cudaStream_t s);

// Plain (unswizzled) tiled tensor map for TMA loads of other kernels.
bool encode_tensor_map(CUtensorMap* m, CUtensorMapDataType type, int rank, const void* base,
                       const cuuint64_t* dims, const cuuint64_t* strides_bytes, const cuuint32_t* box);

}  // namespace dot
