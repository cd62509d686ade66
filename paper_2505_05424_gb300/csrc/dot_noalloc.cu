// dot_noalloc.cu -- the mixed-precision refined Poisson solve for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating runtime: plugins of hosts
// that forbid allocation on their worker threads, processes whose device memory
// is already fully reserved by another allocator, and loops with a fixed memory
// budget that must not risk an allocation failing part way through a run.
// dot_poisson_f32_noalloc serves
// them: the caller passes the right-hand side and the output buffer, and every
// scratch buffer the solve needs (four node-sized FP32 fields, the FP64 partial
// sums of the zero mode, the DCT tables and the pipeline error flag) lives in one
// file-scope __device__ array of fixed size, which every GPU that loads this
// library holds until the process exits.
//
// The array is shared by every call: a call overwrites what the previous one
// left there, and two calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race on it.  Serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/dot.h"
#include "dot_mixed.cuh"
#include "dot_paths.cuh"

namespace dot {
namespace {

constexpr long long kMaxNodes = 1LL << 20;  // (T+1) * N_1 * ... * N_D
constexpr int kMaxAxis = 256;               // largest node count along one spatial axis
// Here the time axis runs the SIMT time pass of the mixed path (no padded time
// tables), which is built for at most 160 time nodes, as DOT_MIXED contexts are.
constexpr int kMaxTimeNodes = 160;

// Layout of the scratch array (256-byte aligned pieces, sizes in bytes).
constexpr size_t kField = (size_t)kMaxNodes * sizeof(float);
constexpr size_t kTable = (size_t)kMaxAxis * kMaxAxis * sizeof(float);
constexpr size_t kLam = (size_t)kMaxAxis * sizeof(float);
constexpr size_t kOffB = 0;
constexpr size_t kOffBlo = kOffB + kField;
constexpr size_t kOffPhi1 = kOffBlo + kField;
constexpr size_t kOffR = kOffPhi1 + kField;
constexpr size_t kOffW1 = kOffR + kField;
constexpr size_t kOffW2 = kOffW1 + kField;
constexpr size_t kOffTables = kOffW2 + kField;                           // (kMaxD+1) axes x 6 tables
constexpr size_t kOffLam = kOffTables + (size_t)(kMaxD + 1) * 6 * kTable; // (kMaxD+1) axes
constexpr size_t kOffSum = kOffLam + (size_t)(kMaxD + 1) * kLam;
constexpr size_t kOffErr = kOffSum + kBsumStride * sizeof(double);  // partial sums of b, then mean(b)
constexpr size_t kOffParam = kOffErr + 256;                            // one SlotParam (active)
constexpr size_t kScratchBytes = kOffParam + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The host-side name g_scratch is a stand-in, not a device address: the address
// is fetched per device with cudaGetSymbolAddress.
std::mutex g_mu;
void* g_dev_ptr[64] = {nullptr};

// Host staging of the DCT tables (static: this path allocates nothing).
float g_host_tab[(kMaxD + 1) * 6][kMaxAxis * kMaxAxis];
float g_host_lam[kMaxD + 1][kMaxAxis];

// error text in a fixed buffer (formatting it allocates nothing)
thread_local char g_err[256];

int fail(int code, const char* m, const char* detail = "") {
  std::snprintf(g_err, sizeof(g_err), "%s%s", m, detail);
  return code;
}

float tf32_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace
}  // namespace dot

extern "C" const char* dot_noalloc_last_error(void) { return dot::g_err; }

extern "C" int dot_poisson_f32_noalloc(const dot_grid* grid, const float* b, float* phi, void* stream) {
  using namespace dot;
  if (!grid || !b || !phi) return fail(DOT_EINVAL, "grid, b and phi are required");
  if (grid->D != 2 && grid->D != 3) return fail(DOT_EINVAL, "D must be 2 or 3");
  if (grid->T < 1 || grid->T + 1 > kMaxTimeNodes) return fail(DOT_EINVAL, "T + 1 must lie in [2, 160]");
  long long nn = grid->T + 1;
  for (int d = 0; d < grid->D; ++d) {
    if (grid->N[d] < 2 || grid->N[d] > kMaxAxis) return fail(DOT_EINVAL, "every N[d] must lie in [2, 256]");
    nn *= grid->N[d];
  }
  if (nn > kMaxNodes) {
    std::snprintf(g_err, sizeof(g_err),
                  "grid has %lld nodes; this entry point handles at most %lld ((T+1) * N_1 * ... * N_D)", nn,
                  kMaxNodes);
    return DOT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(DOT_ECUDA, "cudaGetDevice: ", cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return fail(DOT_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  // set-up once per device, with that device current (the first call on a device;
  // make it before any stream capture)
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return fail(DOT_ECUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
    g_dev_ptr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_dev_ptr[dev];
  dot_grid gr = *grid;
  Geo g = make_geo(gr);

  MxFields f;
  std::memset(&f, 0, sizeof(f));
  f.b = (float*)(base + kOffB);
  f.blo = (float*)(base + kOffBlo);
  f.phi1 = (float*)(base + kOffPhi1);
  f.r = (float*)(base + kOffR);
  f.bsum = (double*)(base + kOffSum);
  MxPoisson ps;
  std::memset(&ps, 0, sizeof(ps));
  ps.w1 = (float*)(base + kOffW1);
  ps.w2 = (float*)(base + kOffW2);
  ps.err = (int*)(base + kOffErr);
  ps.use_tc = true;
  f.sp = (const SlotParam*)(base + kOffParam);

  // DCT tables of this grid (orthonormal DCT-II, its transpose and their TF32 splits)
  for (int a = 0; a <= g.D; ++a) {
    const int M = a == 0 ? g.T + 1 : g.N[a - 1];
    const double pi = 3.14159265358979323846;
    const double h = a == 0 ? 1.0 / g.T : 1.0 / g.N[a - 1];
    float* t[6];
    for (int j = 0; j < 6; ++j) t[j] = g_host_tab[a * 6 + j];
    for (int k = 0; k < M; ++k) {
      const double sk = k == 0 ? std::sqrt(1.0 / M) : std::sqrt(2.0 / M);
      for (int n = 0; n < M; ++n) {
        const double c = sk * std::cos(pi * k * (n + 0.5) / M);
        const float hi = tf32_round((float)c);
        const float lo = (float)(c - (double)hi);
        t[0][k * M + n] = (float)c;
        t[1][n * M + k] = (float)c;
        t[2][k * M + n] = hi;
        t[3][k * M + n] = lo;
        t[4][n * M + k] = hi;
        t[5][n * M + k] = lo;
      }
      const double sv = std::sin(pi * k / (2.0 * M));
      g_host_lam[a][k] = (float)(4.0 / (h * h) * sv * sv);
    }
    float* dst[6];
    for (int j = 0; j < 6; ++j) {
      dst[j] = (float*)(base + kOffTables + (size_t)(a * 6 + j) * kTable);
      e = cudaMemcpyAsync(dst[j], t[j], (size_t)M * M * sizeof(float), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return fail(DOT_ECUDA, "table upload: ", cudaGetErrorString(e));
    }
    float* ldst = (float*)(base + kOffLam + (size_t)a * kLam);
    e = cudaMemcpyAsync(ldst, g_host_lam[a], (size_t)M * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(DOT_ECUDA, "table upload: ", cudaGetErrorString(e));
    ps.C[a] = dst[0];
    ps.CT[a] = dst[1];
    ps.Chi[a] = dst[2];
    ps.Clo[a] = dst[3];
    ps.CThi[a] = dst[4];
    ps.CTlo[a] = dst[5];
    ps.lam[a] = ldst;
  }
  // the right-hand side is copied in (the solve overwrites it with the correction);
  // its low part and the error flag must start at zero
  SlotParam one;
  std::memset(&one, 0, sizeof(one));
  one.rescale = make_float2(1.f, 0.f);
  one.active = 1;
  static SlotParam kOne;
  kOne = one;
  e = cudaMemcpyAsync(f.b, b, (size_t)nn * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.blo, 0, (size_t)nn * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ps.err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + kOffParam, &kOne, sizeof(kOne), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(DOT_ECUDA, "scratch set-up: ", cudaGetErrorString(e));
  long launches = 0;
  LaunchCounter lc{&launches};
  static_assert(kBsumParts + 2 <= kBsumStride, "the partial sums and the mean fit one slot's stride");
  launch_poisson_refined_mx(g, 1, f, ps, reinterpret_cast<float2*>(phi), false, s, lc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DOT_ECUDA, "launch: ", cudaGetErrorString(e));
  int flag = 0;
  e = cudaMemcpyAsync(&flag, ps.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(DOT_ECUDA, "poisson: ", cudaGetErrorString(e));
  if (flag) return fail(DOT_ECUDA, "a tensor-core pipeline wait timed out (kernel returned early)");
  return DOT_OK;
}
