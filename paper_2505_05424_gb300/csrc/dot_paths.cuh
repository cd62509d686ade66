// dot_paths.cuh -- one implementation of Algorithm 2 per precision mode behind a
// small interface used by the C ABI layer (dot_api.cu).
#pragma once
#include <cstddef>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dot.h"
#include "dot_internal.cuh"

namespace dot {

Geo make_geo(const dot_grid& gr);
bool grid_valid(const dot_grid* g, std::string* why);
int check_options(const dot_options& o, std::string* why);
// Densities -> c (cell-average densities, each of mass 1) and omega; DOT_EINVAL
// with a message for non-finite, negative or massless input.
int prepare_densities(const Geo& g, const double* rho0, const double* rho1, const uint8_t* mask,
                      double obstacle_weight, std::vector<double>* m0, std::vector<double>* m1,
                      std::vector<double>* omega, bool* any_mask, std::string* why);
// The problem a context solves: grid, options, stream, densities (c, any scale)
// and the obstacle mask (cells whose weight is not 1).
void problem_of(const dot_ctx* c, dot_grid* g, dot_options* opt, void** stream, std::vector<double>* rho0,
                std::vector<double>* rho1, std::vector<uint8_t>* mask, bool* has_mask);
// The device a context was created on; every entry point makes it current for
// the duration of the call (DeviceScope) and restores the caller's device.
int context_device(const dot_ctx* c);
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev_) == cudaSuccess && prev_ != dev && cudaSetDevice(dev) == cudaSuccess) set_ = true;
  }
  ~DeviceScope() {
    if (set_) cudaSetDevice(prev_);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;

 private:
  int prev_ = 0;
  bool set_ = false;
};
// The multilevel strategy of Sec. 5 (dot_multilevel.cu): densities averaged over
// 2 x ... x 2 blocks (a block is an obstacle if any of its cells is); whether a grid
// can be coarsened `levels` times; level v's tolerance (coarse_tol when given, else
// the paper's max(tol 10^-v, 1e-6)).
void coarsen(const dot_grid& gf, const std::vector<double>& rf, const std::vector<uint8_t>* mf, dot_grid* gc,
             std::vector<double>* rc, std::vector<uint8_t>* mc);
bool multilevel_ok(const dot_grid& g, int levels, std::string* why);
double level_tol(double tol, double coarse_tol, int v);
// Stopping measures of Sec. 5.3 (kkt[DOT_KKT_LEN]) from the reduction slots r;
// cn2 = sum of squares of c.
void kkt_measures(const Geo& g, double cn2, const double* r, long iters, double sigma, double* kkt);

// Bump allocator over the caller's workspace; with base == nullptr it only
// measures (used by dot_workspace_bytes).
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(char* b) : base(b) {}
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

class Path {
 public:
  virtual ~Path() {}
  // Carve buffers, upload masses/omega/DCT tables, zero the iterate.
  virtual int init(char* ws, size_t bytes, const std::vector<double>& m0, const std::vector<double>& m1,
                   const std::vector<double>* omega, cudaStream_t s, std::string* err) = 0;
  // One iteration of Algorithm 2 (lines 1-6) with penalty sigma and step tau.
  virtual void iterate(double sigma, double tau, cudaStream_t s, LaunchCounter lc) = 0;
  // Stopping-measure sums into red_out() (device, R_NSLOTS doubles).
  virtual void kkt(cudaStream_t s, LaunchCounter lc) = 0;
  virtual const double* red_out() const = 0;
  // alpha_0 (natural layout) into rho, alpha_bar (natural layout) into m, phi; NULL = skip.
  virtual int read_fields(double* rho, double* m, double* phi, cudaStream_t s, std::string* err) = 0;
  virtual int read_state(double* q, double* al, double* beta, cudaStream_t s, std::string* err) = 0;
  // The state with the penalty sigma it belongs to (the next iterate uses sigma).
  virtual int write_state(const double* q, const double* al, const double* beta, double sigma, cudaStream_t s,
                          std::string* err) = 0;
  virtual int poisson_op(const double* b, double* phi, cudaStream_t s, LaunchCounter lc, std::string* err) = 0;
  // Device flag that a kernel sets when a bounded pipeline wait gave up (or nullptr).
  virtual const int* error_flag() const { return nullptr; }
  // Mixed path: whether eligible DCT passes run on the tensor cores.
  virtual void set_tensor_cores(bool) {}

  // Replay of whole check periods from a CUDA graph (the mixed path, whose kernels
  // read the penalty and step from device memory).  set_penalty applies sigma and
  // tau for the next iterations (and rescales the stored multipliers when sigma
  // changed) outside the graph; parity says which of the two iterate buffers is
  // current (a capture flips it without running anything); residual_carried says
  // that the next iteration reuses a residual left by the previous one, which a
  // period captured right after a stopping-measure check does not expect.
  virtual bool graphable() const { return false; }
  virtual void set_penalty(double, double, cudaStream_t, LaunchCounter) {}
  virtual int parity() const { return 0; }
  virtual void set_parity(int) {}
  virtual bool residual_carried() const { return false; }
  // Called once after every check period (host bookkeeping between periods).
  virtual void end_period() {}
};

size_t path_workspace_bytes(const Geo& g, dot_precision prec);
std::unique_ptr<Path> make_path(dot_precision prec, const Geo& g);
// The mixed-precision path (path_mixed.cu).
void carve_mixed_size(const Geo& g, Carver& cv);
std::unique_ptr<Path> make_mixed_path(const Geo& g);

// Shared host helpers (defined in path_f64.cu).
void dct_tables_host(const Geo& g, int axis, std::vector<double>* C, std::vector<double>* lam);
// Geometry of face family fam >= 1 for the natural <-> padded copies:
// width / pitch in elements, height in rows.
void face_copy_shape(const Geo& g, int fam, size_t* width, size_t* pitch, size_t* height);
long long natural_face_count(const Geo& g, int fam);

}  // namespace dot
