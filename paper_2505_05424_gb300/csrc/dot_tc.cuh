// dot_tc.cuh -- tensor-core (tcgen05) DCT pass of the mixed-path Poisson solve.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace dot {

// The tcgen05 pass handles axis lengths K with K % 4 == 0 (TMA row strides are
// multiples of 16 bytes) and K <= 256 (one TMEM accumulator tile).
bool tc_pass_supported(int K);
int tc_smem_bytes();
// See k_dct_tc.cu: mode 0 = rows flattened (Out[k][r]), mode 1 = rows along a at
// fixed b (Out[b][k][a]).  Bhi/Blo: K x K matrices, row k = output frequency.
bool launch_dct_pass_tc(const float* X, const float* Bhi, const float* Blo, float* out, int K, int mode,
                        long long R, int A, int Bd, int* err, cudaStream_t s);

// Plain (unswizzled) tiled tensor map for TMA loads of other kernels.
bool encode_tensor_map(CUtensorMap* m, CUtensorMapDataType type, int rank, const void* base,
                       const cuuint64_t* dims, const cuuint64_t* strides_bytes, const cuuint32_t* box);

}  // namespace dot
