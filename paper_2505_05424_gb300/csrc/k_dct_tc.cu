// k_dct_tc.cu -- one DCT pass of the mixed-path Poisson solve on the 5th-generation
// tensor cores (tcgen05, TMEM accumulators, TMA operand staging), in 3xTF32
// split precision with FP32 accumulation.
//
// A pass applies the M x M matrix B (the orthonormal DCT-II matrix C for a forward
// transform, C^T for the inverse) along the innermost axis of a field whose rows
// are K = M contiguous values (row stride ldx >= K, a multiple of 4):
//     Out(k, row) = sum_j X(row, j) B(k, j)
// Rows come in G groups (independent solves of one batch, stored one after the
// other).  Output modes:
//   ROWS_FLAT  tile rows r = 128 consecutive rows; with r = g*A + a and a = a1*M + a0,
//              Out[g][k][a1][a0] with the a0 runs padded to stride ldo (M = 1, ldo = 1:
//              plain Out[g][k][a]): the transformed axis moves outermost in the group
//   ROWS_A     input [G][A][Bd][K]; tile rows = 128 consecutive a at fixed (g, b);
//              Out[g][b][k][a]
//   KEEP       Out[r][k] with row stride ldo, each value divided by the Neumann
//              eigenvalue lam_0(k) + sum_d lam_d(k_d(r mod P)) (the zero mode -> 0):
//              the time-axis forward transform and scaling of the Poisson solve
// In ROWS_FLAT and ROWS_A the 32 lanes of a warp hold 32 consecutive output
// addresses for every column k, so the epilogue stores are coalesced.  Columns of
// X beyond K and rows of B beyond K are zero-filled by the TMA unit.
//
// 3xTF32: x = x_hi + x_lo with x_hi = tf32_rna(x) and x_lo = x - x_hi (exact in
// FP32); B likewise (split once on the host).  Each K-step issues
// x_hi*B_hi + x_hi*B_lo + x_lo*B_hi into one FP32 accumulator; the dropped
// x_lo*B_lo term and the truncation of x_lo to TF32 are O(2^-22) relative.
//
// CTA roles (192 threads): warp 0 issues TMA loads (one elected lane), warp 1
// owns TMEM and issues the MMAs (one elected lane), warps 2-5 split the X tile
// into hi/lo in shared memory and run the epilogue (tcgen05.ld from TMEM).
// Every mbarrier wait is bounded; on timeout the CTA records the failure in
// *err, stops issuing work, and still frees its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <chrono>
#include <cstdint>
#include <cstring>

#include "dot_internal.cuh"
#include "dot_tc.cuh"
#include "ffloat.cuh"

namespace dot {
namespace {

constexpr int kTileM = 128;          // rows per CTA (MMA M)
constexpr int kChunkK = 32;          // K elements per stage (128 bytes: one SW128 row)
constexpr int kStages = 2;
constexpr int kMaxN = 256;           // columns of the accumulator (MMA N)
constexpr int kThreadsTC = 192;

constexpr int kXBytes = kTileM * kChunkK * 4;      // 16 KB
// A stage holds the X tile (hi and lo) and Nout rows of the table (hi and lo);
// shared memory and TMEM columns are sized to Nout so that short axes run two or
// more CTAs per SM.
__host__ __device__ constexpr int stage_bytes(int nout) { return 2 * kXBytes + 2 * nout * kChunkK * 4; }
__host__ __device__ constexpr int smem_bytes(int nout) { return kStages * stage_bytes(nout) + 1024 + 256; }
constexpr int kSmemBytes = smem_bytes(kMaxN);
// TMEM allocation: a power of two >= 32 columns
__host__ __device__ constexpr int tmem_cols(int nout) {
  return nout <= 32 ? 32 : nout <= 64 ? 64 : nout <= 128 ? 128 : 256;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the phase with the given parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  return mbar_wait_bounded(smem_u32(bar), parity);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B
// apart (SBO), LBO unused for this layout (set to 16 B), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                 // LBO (ignored for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // SBO
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct PassArgs {
  float* out;
  int K;           // length of the transformed axis (= reduction length)
  int Nout;        // output columns per CTA (MMA N, multiple of 16, <= 256); CTA column
                   // tile blockIdx.y covers frequencies [256 * blockIdx.y, + Nout)
  int mode;        // TC_ROWS_FLAT, TC_ROWS_A, TC_KEEP
  long long R;     // ROWS_FLAT / KEEP: total rows (all groups)
  int A, Bd, G;    // ROWS_FLAT: rows per group A; ROWS_A: extents of a, b; G groups
  FastDiv fA, fM;  // division by A and by M (ROWS_FLAT)
  int M, ldo;      // ROWS_FLAT: runs of M rows, stride ldo; KEEP: output row stride
  // KEEP: eigenvalue tables (lam[0] along the transformed axis) and the spatial
  // decode of r mod P
  const float* lam[kMaxD + 1];
  int D;
  int N[kMaxD];
  unsigned P;
  FastDiv fP, fS[kMaxD], fN[kMaxD];
  float2* accum;   // ROWS_A: accumulate into a two-float field instead of writing out
  int* err;
  unsigned extra_tx;   // see TcPass::extra_tx
};

__global__ void __launch_bounds__(kThreadsTC, 2)
k_dct_pass_tc(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_bhi,
              const __grid_constant__ CUtensorMap tm_blo, PassArgs pa) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s: X hi, X lo, B hi, B lo (addresses computed, not kept in an indexed array)
  const int sbytes = stage_bytes(pa.Nout);
  auto sx = [&](int s) { return smem + s * sbytes; };
  auto sxlo = [&](int s) { return smem + s * sbytes + kXBytes; };
  auto sbh = [&](int s) { return smem + s * sbytes + 2 * kXBytes; };
  auto sbl = [&](int s) { return smem + s * sbytes + 2 * kXBytes + pa.Nout * kChunkK * 4; };
  uint64_t* bars = (uint64_t*)(smem + kStages * stage_bytes(pa.Nout));
  const uint32_t ncols = (uint32_t)tmem_cols(pa.Nout);
  uint64_t* full = bars;                 // TMA landed
  uint64_t* conv = bars + kStages;       // hi/lo split done
  uint64_t* empty = bars + 2 * kStages;  // MMAs of the stage done
  uint64_t* accf = bars + 3 * kStages;   // accumulator complete
  uint32_t* tmem_slot = (uint32_t*)(bars + 3 * kStages + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (pa.K + kChunkK - 1) / kChunkK;
  // tile coordinates
  long long row0 = 0;
  int a0 = 0, bfix = 0, gfix = 0;
  if (pa.mode != TC_ROWS_A) {
    row0 = (long long)blockIdx.x * kTileM;
  } else {
    const int tiles_a = (pa.A + kTileM - 1) / kTileM;
    const int tb = blockIdx.x / tiles_a;
    a0 = (blockIdx.x - tb * tiles_a) * kTileM;
    gfix = tb / pa.Bd;
    bfix = tb - gfix * pa.Bd;
  }

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 4);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  // this CTA's output columns: [n0, n0 + nout)
  const int n0 = blockIdx.y * kMaxN;
  const int nout = min(pa.Nout, (pa.K - n0 + 15) / 16 * 16);
  if (warp == 0) {
    if (lane == 0) {
      const unsigned bytes = kXBytes + 2u * (unsigned)pa.Nout * kChunkK * 4u + pa.extra_tx;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % kStages, it = c / kStages;
        if (c >= kStages && !mbar_wait(&empty[s], (it - 1) & 1)) { atomicExch(&s_fail, 1); break; }
        if (s_fail) break;
        mbar_expect_tx(&full[s], bytes);
        if (pa.mode != TC_ROWS_A) tma_load_2d(sx(s), &tm_x, &full[s], c * kChunkK, (int)row0);
        else tma_load_4d(sx(s), &tm_x, &full[s], c * kChunkK, bfix, a0, gfix);
        tma_load_2d(sbh(s), &tm_bhi, &full[s], c * kChunkK, n0);
        tma_load_2d(sbl(s), &tm_blo, &full[s], c * kChunkK, n0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(kTileM, nout);
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % kStages, it = c / kStages;
        if (!mbar_wait(&conv[s], it & 1)) { atomicExch(&s_fail, 1); break; }
        if (s_fail) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ax = smem_u32(sx(s)), al = smem_u32(sxlo(s));
        const uint32_t bh = smem_u32(sbh(s)), bl = smem_u32(sbl(s));
#pragma unroll
        for (int kk = 0; kk < kChunkK / 8; ++kk) {
          const uint32_t off = kk * 32;   // 8 TF32 = 32 bytes along K inside the swizzle atom
          const uint32_t accum = (c > 0 || kk > 0) ? 1u : 0u;
          mma_tf32(tmem, sw128_desc(ax + off), sw128_desc(bh + off), idesc, accum);
          mma_tf32(tmem, sw128_desc(ax + off), sw128_desc(bl + off), idesc, 1u);
          mma_tf32(tmem, sw128_desc(al + off), sw128_desc(bh + off), idesc, 1u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(accf);
    }
  } else {
    // warps 2-5: split X into hi/lo, then the epilogue
    const int t = threadIdx.x - 64;   // 0..127
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % kStages, it = c / kStages;
      // warp-uniform decision: every lane waits, the warp leaves together
      const bool got = __all_sync(0xffffffffu, mbar_wait(&full[s], it & 1));
      if (!got) { atomicExch(&s_fail, 1); break; }
      float4* px = reinterpret_cast<float4*>(sx(s));
      float4* pl = reinterpret_cast<float4*>(sxlo(s));
#pragma unroll 4
      for (int e = t; e < kXBytes / 16; e += 128) {
        float4 v = px[e];
        float4 h, l;
        h.x = tf32_rna(v.x); l.x = v.x - h.x;
        h.y = tf32_rna(v.y); l.y = v.y - h.y;
        h.z = tf32_rna(v.z); l.z = v.z - h.z;
        h.w = tf32_rna(v.w); l.w = v.w - h.w;
        px[e] = h;
        pl[e] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
    }
    bool ok = __all_sync(0xffffffffu, mbar_wait(accf, 0));
    if (!ok) atomicExch(&s_fail, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = __all_sync(0xffffffffu, ok && (*(volatile int*)&s_fail == 0));   // tcgen05.ld needs a uniform warp
    if (ok) {
      const int wq = warp & 3;                 // TMEM lane quarter this warp may access
      const int row = wq * 32 + lane;          // row within the tile
      // KEEP: this warp's copy of the time eigenvalues lam_0(n0 .. n0 + nout) in
      // stage 0's X tile, which no TMA load or MMA touches once the accumulator is
      // complete (one copy per warp: no barrier across warps)
      float* slam = reinterpret_cast<float*>(sx(0)) + (warp - 2) * kMaxN;
      if (pa.mode == TC_KEEP) {
        for (int i = lane; i < nout; i += 32) slam[i] = n0 + i < pa.K ? pa.lam[0][n0 + i] : 1.f;
        __syncwarp();
      }
      long long out_base = 0, col_stride = 1;
      bool valid;
      float lsp = 0.f;        // KEEP: spatial part of the eigenvalue
      bool zero_mode = false;
      if (pa.mode == TC_ROWS_FLAT) {
        const long long r = row0 + row;
        valid = r < pa.R;
        if (valid) {
          const unsigned g = fdiv((unsigned)r, pa.fA), a = (unsigned)r - g * (unsigned)pa.A;
          const unsigned a1 = fdiv(a, pa.fM), a0r = a - a1 * (unsigned)pa.M;
          col_stride = (long long)(pa.A / pa.M) * pa.ldo;
          out_base = (long long)g * pa.K * col_stride + (long long)a1 * pa.ldo + a0r;
        }
      } else if (pa.mode == TC_ROWS_A) {
        const int a = a0 + row;
        valid = a < pa.A;
        col_stride = pa.A;
        out_base = ((long long)gfix * pa.Bd + bfix) * pa.K * pa.A + a;
      } else {
        const long long r = row0 + row;
        valid = r < pa.R;
        if (valid) {
          out_base = r * pa.ldo;
          const unsigned sp = (unsigned)r - fdiv((unsigned)r, pa.fP) * pa.P;
          zero_mode = sp == 0;
          for (int d = 0; d < pa.D; ++d) {
            const unsigned q = fdiv(sp, pa.fS[d]);
            const unsigned kd = d == 0 ? q : q - fdiv(q, pa.fN[d]) * (unsigned)pa.N[d];
            lsp += pa.lam[1 + d][kd];
          }
        }
      }
      for (int c0 = 0; c0 < nout; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!valid) continue;
        if (pa.mode == TC_KEEP) {
          float w[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int k = n0 + c0 + j;
            const float lam = slam[c0 + j] + lsp;
            // fast division (within 2 ulp for the eigenvalue range, 0 < lam < 2^126)
            w[j] = (k == 0 && zero_mode) ? 0.f : __fdividef(__uint_as_float(v[j]), lam);
          }
          float* o = pa.out + out_base + n0 + c0;
          if (n0 + c0 + 16 <= pa.K) {
#pragma unroll
            for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(o + j) = make_float4(w[j], w[j + 1], w[j + 2], w[j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (n0 + c0 + j < pa.K) o[j] = w[j];
          }
        } else if (pa.accum) {
          // all 16 loads first, then the stores: no load waits behind a store
          float2 old[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (n0 + c0 + j < pa.K) old[j] = pa.accum[out_base + (long long)(n0 + c0 + j) * col_stride];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (n0 + c0 + j < pa.K)
              pa.accum[out_base + (long long)(n0 + c0 + j) * col_stride] = ff_add_f(old[j], __uint_as_float(v[j]));
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int k = n0 + c0 + j;
            if (k < pa.K) pa.out[out_base + (long long)k * col_stride] = __uint_as_float(v[j]);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(pa.err, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool encode(CUtensorMap* m, const float* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides_bytes,
            const cuuint32_t* box) {
  auto fn = get_encode();
  if (!fn) return false;
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, (void*)base, dims, strides_bytes, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool encode_tensor_map(CUtensorMap* m, CUtensorMapDataType type, int rank, const void* base,
                       const cuuint64_t* dims, const cuuint64_t* strides_bytes, const cuuint32_t* box) {
  auto fn = get_encode();
  if (!fn) return false;
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(m, type, rank, (void*)base, dims, strides_bytes, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_pass_supported(int K) { return K >= 1 && K <= 16 * kMaxN; }


bool launch_tc_pass(const TcPass& p, cudaStream_t s) {
  static std::atomic<unsigned long long> smem_done{0};
  smem_optin((const void*)k_dct_pass_tc, kSmemBytes, &smem_done);
  const int K = p.K;
  if (!tc_pass_supported(K) || p.ldx < K || p.ldx % 4 != 0 || p.ldb < K || p.ldb % 4 != 0) return false;
  if (((uintptr_t)p.X & 15) || ((uintptr_t)p.Bhi & 15) || ((uintptr_t)p.Blo & 15)) return false;
  const int Nout = K < kMaxN ? (K + 15) / 16 * 16 : kMaxN;
  CUtensorMap mx, mh, ml;
  bool ok;
  if (p.mode != TC_ROWS_A) {
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)p.R};
    cuuint64_t str[1] = {(cuuint64_t)p.ldx * 4};
    cuuint32_t box[2] = {kChunkK, kTileM};
    ok = encode(&mx, p.X, 2, dims, str, box);
  } else {
    cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)p.Bd, (cuuint64_t)p.A, (cuuint64_t)p.G};
    cuuint64_t str[3] = {(cuuint64_t)p.ldx * 4, (cuuint64_t)p.ldx * 4 * p.Bd,
                         (cuuint64_t)p.ldx * 4 * p.Bd * p.A};
    cuuint32_t box[4] = {kChunkK, 1, kTileM, 1};
    ok = encode(&mx, p.X, 4, dims, str, box);
  }
  cuuint64_t bdims[2] = {(cuuint64_t)K, (cuuint64_t)K};
  cuuint64_t bstr[1] = {(cuuint64_t)p.ldb * 4};
  cuuint32_t bbox[2] = {kChunkK, (cuuint32_t)Nout};
  ok = ok && encode(&mh, p.Bhi, 2, bdims, bstr, bbox) && encode(&ml, p.Blo, 2, bdims, bstr, bbox);
  if (!ok) return false;
  PassArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.out = p.out;
  pa.K = K;
  pa.Nout = Nout;
  pa.mode = p.mode;
  pa.R = p.R;
  pa.A = p.A > 0 ? p.A : 1;
  pa.Bd = p.Bd > 0 ? p.Bd : 1;
  pa.G = p.G > 0 ? p.G : 1;
  pa.M = p.M > 0 ? p.M : 1;
  pa.ldo = p.ldo > 0 ? p.ldo : 1;
  pa.fA = make_fastdiv((unsigned)pa.A);
  pa.fM = make_fastdiv((unsigned)pa.M);
  pa.err = p.err;
  pa.extra_tx = p.extra_tx;
  pa.accum = p.mode == TC_ROWS_A ? p.accum : nullptr;
  if (p.accum && p.mode != TC_ROWS_A) return false;
  if (p.mode == TC_ROWS_FLAT && (p.R % pa.A != 0 || pa.A % pa.M != 0 || pa.ldo < pa.M)) return false;
  if (p.mode == TC_KEEP) {
    if (!p.geo || pa.ldo < K || pa.ldo % 4 != 0 || ((uintptr_t)p.out & 15)) return false;
    const Geo& g = *p.geo;
    pa.D = g.D;
    for (int a = 0; a <= g.D; ++a) pa.lam[a] = p.lam[a];
    for (int d = 0; d < kMaxD; ++d) {
      pa.N[d] = g.N[d];
      pa.fS[d] = g.fS[d];
      pa.fN[d] = g.fN[d];
    }
    pa.P = (unsigned)g.P;
    pa.fP = g.fP;
  }
  dim3 grid(p.mode != TC_ROWS_A ? (unsigned)((p.R + kTileM - 1) / kTileM)
                                 : (unsigned)(pa.G * pa.Bd * ((p.A + kTileM - 1) / kTileM)),
            (unsigned)((K + kMaxN - 1) / kMaxN));
  k_dct_pass_tc<<<grid, kThreadsTC, smem_bytes(Nout), s>>>(mx, mh, ml, pa);
  return true;
}

}  // namespace dot

// Self-test of the bounded pipeline waits (include/dot_selftest.h).
extern "C" int dot_selftest_pipeline_timeout(int inject, double* seconds, int* flag) {
  using namespace dot;
  if (!seconds || !flag) return -1;
  const int K = 32, R = 128;   // one 128-row tile, one chunk: a single CTA
  float *x = nullptr, *bh = nullptr, *bl = nullptr, *out = nullptr;
  int* err = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaMalloc(&x, sizeof(float) * R * K);
  if (e == cudaSuccess) e = cudaMalloc(&bh, sizeof(float) * K * K);
  if (e == cudaSuccess) e = cudaMalloc(&bl, sizeof(float) * K * K);
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * R * K);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, sizeof(float) * R * K, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bh, 0, sizeof(float) * K * K, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bl, 0, sizeof(float) * K * K, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int rc = e == cudaSuccess ? 0 : -3;
  if (rc == 0) {
    TcPass p;
    std::memset(&p, 0, sizeof(p));
    p.X = x;
    p.ldx = K;
    p.Bhi = bh;
    p.Blo = bl;
    p.ldb = K;
    p.out = out;
    p.K = K;
    p.mode = TC_ROWS_FLAT;
    p.R = R;
    p.A = R;
    p.M = 1;
    p.ldo = 1;
    p.err = err;
    // 16 bytes more than the loads deliver: the stage's barrier never completes
    p.extra_tx = inject ? 16u : 0u;
    const auto t0 = std::chrono::steady_clock::now();
    if (!launch_tc_pass(p, s)) rc = -1;
    if (rc == 0 && cudaStreamSynchronize(s) != cudaSuccess) rc = -3;
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rc == 0 && cudaMemcpy(flag, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = -3;
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(x);
  cudaFree(bh);
  cudaFree(bl);
  cudaFree(out);
  cudaFree(err);
  return rc;
}

