// dot_internal.cuh -- shared declarations of the CUDA path (kernels + host control).
//
// Device layout.  Every field is a stack of time planes of P = N_1 * ... * N_D
// elements in C order ([x_1]...[x_D], x_D fastest):
//   nodes (phi, b, Poisson scratch)   : T+1 planes
//   q_0, alpha_0 (time faces, cones)   : T planes
//   q_d, alpha_d (space faces, d >= 1) : T+1 planes, padded to N_d entries along
//                                        axis d; the entry x_d = N_d - 1 is a pad
//                                        that is kept at exactly 0
//   beta (and z in the FP64 path)      : K = 4D+2 component planes of T*P each
// The padding gives every staggered field the node layout, so a stencil reads
// its neighbours at fixed offsets (P along time, sst[d] along axis d).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace dot {

constexpr int kMaxD = 3;
constexpr int kMaxK = 4 * kMaxD + 2;

// Bounded wait on an mbarrier phase (shared-memory address `bar`): true once the
// phase with the given parity has completed, false after about one second on the
// global timer, so that a pipeline whose producer never arrives returns an error
// status to the host instead of hanging the GPU.  The timer is read on the first
// miss and then every 1024 polls.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, unsigned parity) {
  unsigned long long t0 = 0;
  for (unsigned it = 0; it < 0x80000000u; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 1023u) == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (it == 0) t0 = t;
      else if (t - t0 > kWaitLimitNs) return false;
    }
  }
  return false;
}

// Unsigned division of n < 2^31 by a fixed divisor d >= 2 with one multiply-high
// and a shift: with l = ceil(log2 d) and m = ceil(2^(31 + l) / d) (< 2^32),
// floor(n / d) = umulhi(n, m) >> (l - 1) (the round-up method of Granlund and
// Montgomery, "Division by invariant integers using multiplication", PLDI 1994).
// d = 1 passes n through.
struct FastDiv {
  unsigned d;
  unsigned m;
  unsigned sh;
};

inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  if (d <= 1) {
    f.m = 0;
    f.sh = 0;
    return f;
  }
  unsigned l = 0;
  while ((1ull << l) < d) ++l;                 // l = ceil(log2 d)
  const unsigned long long p = 31ull + l;
  f.m = (unsigned)(((1ull << p) + d - 1) / d);  // ceil(2^p / d) < 2^32
  f.sh = (unsigned)(p - 32);
  return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
  return f.d <= 1 ? n : (__umulhi(n, f.m) >> f.sh);
}

// Opt a kernel into `bytes` of dynamic shared memory on the current device.  The
// attribute belongs to the device, so each call site keeps a bit per device
// (devices 0-63; others set it at every call) in `done`.
inline void smem_optin(const void* kernel, int bytes, std::atomic<unsigned long long>* done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done->load(std::memory_order_acquire) & bit)) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess && bit)
    done->fetch_or(bit, std::memory_order_acq_rel);
}

// Grid geometry passed by value to every kernel.  Element indices of one field
// stay below 2^31 ((T+1) * P * ... is checked at dot_create), so the plane and
// coordinate arithmetic runs on 32-bit fast divisions.
struct Geo {
  int D;                 // spatial dimension
  int T;                 // time intervals
  int K;                 // cone dimension 4D + 2
  int N[kMaxD];          // cells per spatial axis (1 beyond D)
  long long P;           // nodes per time plane
  long long sst[kMaxD];  // element stride of spatial axis d inside a plane
  double invh[kMaxD + 1];  // 1/h: invh[0] = T, invh[1 + d] = N_d
  FastDiv fP;            // division by P
  FastDiv fS[kMaxD];     // division by sst[d]
  FastDiv fN[kMaxD];     // division by N[d]
};

// coordinate along spatial axis d of in-plane index p: (p / sst[d]) % N[d]
__device__ __forceinline__ int coord(const Geo& g, long long p, int d) {
  const unsigned q = fdiv((unsigned)p, g.fS[d]);
  if (d == 0) return (int)q;   // p < P: the outermost coordinate needs no modulo
  return (int)(q - fdiv(q, g.fN[d]) * (unsigned)g.N[d]);
}

// time plane of element index i (i < 2^31)
__device__ __forceinline__ int plane_of(const Geo& g, long long i) { return (int)fdiv((unsigned)i, g.fP); }

// Reduction slots of the stopping measures (sums of squares and inner products).
enum RedSlot {
  R_PRIM = 0,     // sum (A phi - q)^2
  R_APHI,         // sum (A phi)^2
  R_Q,            // sum q^2
  R_DUALRES,      // sum (A^* alpha + c)^2
  R_COMP0,        // sum (alpha_0 - max(0, f + alpha_0))^2
  R_ALPHA0,       // sum alpha_0^2
  R_F,            // sum f^2
  R_COMPD,        // sum (alpha_bar - g)^2
  R_ALPHAB,       // sum alpha_bar^2
  R_G,            // sum g^2
  R_SOCP,         // sum (z - B F q - d)^2
  R_SOCD,         // sum (F^* B^* beta + alpha)^2
  R_FBB,          // sum (F^* B^* beta)^2
  R_CPHI,         // <c, phi>
  R_DUALOBJ,      // -1/2 sum alpha_bar^2 / den over den > 0
  R_NSLOTS
};

// FP64 fields (all device pointers into the workspace).
struct F64Fields {
  double* q[kMaxD + 1];
  double* al[kMaxD + 1];
  double* beta;   // K * T * P
  double* z;      // K * T * P
  double* phi;    // (T+1) * P
  double* b;      // (T+1) * P, also Poisson ping-pong buffer
  double* w1;     // (T+1) * P Poisson ping-pong buffer
  const double* m0;      // P, rho0 cell masses
  const double* m1;      // P, rho1 cell masses
  const double* omega;   // P or nullptr (omega = 1 everywhere)
  const double* somega;  // P or nullptr: sqrt(omega / 2)
};

// DCT tables per axis (axis 0 = time): orthonormal DCT-II matrix (M x M,
// row k = frequency) and the 1D Neumann eigenvalues (4/h^2) sin^2(pi k / (2M)).
struct DctTables64 {
  const double* C[kMaxD + 1];
  const double* lam[kMaxD + 1];
};

// ---- launch helpers (defined in the .cu files) ----------------------------
// Kernel ids for launch accounting and per-kernel timing (names in dot_api.cu).
enum KernelId {
  KID_ASSEMBLE_B = 0, KID_DCT_AXIS, KID_SCALE, KID_RESIDUAL, KID_COMBINE, KID_PROJECT,
  KID_UPDATE_Q0, KID_UPDATE_QD, KID_UPDATE_BETA, KID_KKT, KID_DCT_TC, KID_FUSED, KID_FACE3, KID_COUNT
};

// Counts launches; when `mark` is set, it is called after every launch with the
// kernel id so the caller can record a CUDA event on the launching stream.
struct LaunchCounter {
  long* n;
  void (*mark)(void*, int) = nullptr;
  void* user = nullptr;
  void tick(int k = 1) const { if (n) *n += k; }
  void launched(int kid, int k = 1) const {
    tick(k);
    if (mark) mark(user, kid);
  }
};

void launch_assemble_b_f64(const Geo& g, const F64Fields& f, double sigma, cudaStream_t s, LaunchCounter lc);
void launch_project_f64(const Geo& g, const F64Fields& f, double sigma, cudaStream_t s, LaunchCounter lc);
void launch_update_q_alpha_f64(const Geo& g, const F64Fields& f, double sigma, double tau, cudaStream_t s, LaunchCounter lc);
void launch_update_beta_f64(const Geo& g, const F64Fields& f, double sigma, double tau, cudaStream_t s, LaunchCounter lc);
// Poisson solve in place of (b -> phi), using w1 as scratch.  b is overwritten.
void launch_poisson_f64(const Geo& g, const DctTables64& t, double* b, double* w1, double* phi,
                        cudaStream_t s, LaunchCounter lc);
// Stopping-measure sums into out[R_NSLOTS] (device), using `partials` scratch of
// kkt_partials_len(g) doubles.
long long kkt_partials_len(const Geo& g);
void launch_kkt_f64(const Geo& g, const F64Fields& f, double* partials, double* out, cudaStream_t s,
                    LaunchCounter lc);

}  // namespace dot
