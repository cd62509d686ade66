// dot_api.cu -- the C ABI of include/dot.h: validation, the workspace plan,
// Algorithm 2's outer loop with the penalty rule and stopping test of Sec. 5.3,
// and host<->device layout conversion.  All per-element work runs in the kernels
// of the sibling .cu files; the host only moves scalars and copies buffers.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dot.h"
#include "dot_internal.cuh"
#include "dot_paths.cuh"

using namespace dot;

namespace {

thread_local std::string g_thread_err;

double elapsed_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

bool grid_ok(const dot_grid* g, std::string* why) {
  if (!g) { *why = "grid is NULL"; return false; }
  if (g->D != 2 && g->D != 3) { *why = "D must be 2 or 3"; return false; }
  if (g->T < 1 || g->T > 65535) { *why = "T must be in [1, 65535]"; return false; }
  long double n = (long double)(g->T + 1);
  for (int d = 0; d < g->D; ++d) {
    if (g->N[d] < 2 || g->N[d] > 65536) { *why = "every N[d] must be in [2, 65536]"; return false; }
    n *= g->N[d];
  }
  // every field's element index, including 4D+2 stacked cone components, stays
  // below 2^31 (32-bit index arithmetic in the kernels)
  if (n * (long double)(4 * g->D + 2) >= 2147483648.0L) { *why = "grid too large"; return false; }
  return true;
}

}  // namespace

Geo dot::make_geo(const dot_grid& gr) {
  Geo g;
  std::memset(&g, 0, sizeof(g));
  g.D = gr.D;
  g.T = gr.T;
  g.K = 4 * gr.D + 2;
  for (int d = 0; d < kMaxD; ++d) g.N[d] = d < gr.D ? gr.N[d] : 1;
  long long st = 1;
  for (int d = gr.D - 1; d >= 0; --d) {
    g.sst[d] = st;
    st *= g.N[d];
  }
  for (int d = gr.D; d < kMaxD; ++d) g.sst[d] = st;
  g.P = st;
  g.invh[0] = (double)gr.T;
  for (int d = 0; d < gr.D; ++d) g.invh[1 + d] = (double)gr.N[d];
  g.fP = make_fastdiv((unsigned)g.P);
  for (int d = 0; d < kMaxD; ++d) {
    g.fS[d] = make_fastdiv((unsigned)g.sst[d]);
    g.fN[d] = make_fastdiv((unsigned)g.N[d]);
  }
  return g;
}

// Stopping measures from the reduction slots (Sec. 5.3), discrete L2 norms with
// the space-time cell volume h_0 h_1 ... h_D.
void dot::kkt_measures(const Geo& g, double cn2, const double* r, long iters, double sigma, double* kkt) {
  double vol = 1.0 / g.T;
  for (int d = 0; d < g.D; ++d) vol *= 1.0 / g.N[d];
  auto L2 = [vol](double s) { return std::sqrt(vol * s); };
  const double dn2 = 2.0 * (double)g.T * (double)g.P;
  const double etaP = L2(r[R_PRIM]) / (1.0 + L2(r[R_APHI]) + L2(r[R_Q]));
  const double etaD = L2(r[R_DUALRES]) / (1.0 + L2(cn2));
  const double c1 = L2(r[R_COMP0]) / (1.0 + L2(r[R_ALPHA0]) + L2(r[R_F]));
  const double c2 = L2(r[R_COMPD]) / (1.0 + L2(r[R_ALPHAB]) + L2(r[R_G]));
  const double etaC = c1 > c2 ? c1 : c2;
  const double psoc = L2(r[R_SOCP]) / (1.0 + L2(dn2));
  const double dsoc = L2(r[R_SOCD]) / (1.0 + L2(r[R_FBB]) + L2(r[R_ALPHA0] + r[R_ALPHAB]));
  double eta = etaP;
  if (etaD > eta) eta = etaD;
  if (etaC > eta) eta = etaC;
  if (std::isnan(etaD) || std::isnan(etaC) || std::isnan(etaP)) eta = NAN;
  kkt[DOT_KKT_ETA] = eta;
  kkt[DOT_KKT_ETA_P] = etaP;
  kkt[DOT_KKT_ETA_D] = etaD;
  kkt[DOT_KKT_ETA_C] = etaC;
  kkt[DOT_KKT_ETA_P_SOC] = etaP > psoc ? etaP : psoc;
  kkt[DOT_KKT_ETA_D_SOC] = etaD > dsoc ? etaD : dsoc;
  kkt[DOT_KKT_PRIMAL] = r[R_CPHI];
  kkt[DOT_KKT_DUAL] = r[R_DUALOBJ];
  kkt[DOT_KKT_GAP] = std::fabs(r[R_CPHI] - r[R_DUALOBJ]) / (1.0 + std::fabs(r[R_CPHI]) + std::fabs(r[R_DUALOBJ]));
  kkt[DOT_KKT_ITERS] = (double)iters;
  kkt[DOT_KKT_SIGMA] = sigma;
}

// Validate the densities and the mask and turn them into c of eq. (defc) as
// cell-average densities (mass / (h_1 ... h_D), each density normalised to mass
// 1: the data scaling of Sec. 5.3; it leaves phi and q unchanged and makes
// alpha_0 / h_0 the density) and the obstacle weights omega.
int dot::prepare_densities(const Geo& g, const double* rho0, const double* rho1, const uint8_t* mask,
                           double obstacle_weight, std::vector<double>* m0, std::vector<double>* m1,
                           std::vector<double>* omega, bool* any_mask, std::string* why) {
  const long long P = g.P;
  double s0 = 0.0, s1 = 0.0;
  for (long long i = 0; i < P; ++i) {
    if (!std::isfinite(rho0[i]) || !std::isfinite(rho1[i]) || rho0[i] < 0.0 || rho1[i] < 0.0) {
      *why = "densities must be finite and non-negative";
      return DOT_EINVAL;
    }
    s0 += rho0[i];
    s1 += rho1[i];
  }
  if (!(s0 > 0.0) || !(s1 > 0.0) || !std::isfinite(s0) || !std::isfinite(s1)) {
    *why = "densities must have positive finite mass";
    return DOT_EINVAL;
  }
  m0->resize(P);
  m1->resize(P);
  omega->resize(P);
  *any_mask = false;
  const double inv_cell = (double)P;
  for (long long i = 0; i < P; ++i) {
    (*m0)[i] = rho0[i] / s0 * inv_cell;
    (*m1)[i] = rho1[i] / s1 * inv_cell;
    const bool ob = mask && mask[i];
    *any_mask = *any_mask || ob;
    (*omega)[i] = ob ? obstacle_weight : 1.0;
  }
  return DOT_OK;
}

bool dot::grid_valid(const dot_grid* g, std::string* why) { return grid_ok(g, why); }

int dot::check_options(const dot_options& o, std::string* why) {
  if (!(o.tau > 0.0 && o.tau < 2.0)) { *why = "tau must lie in (0, 2)"; return DOT_EINVAL; }
  if (!(o.sigma0 > 0.0 && std::isfinite(o.sigma0))) { *why = "sigma0 must be > 0"; return DOT_EINVAL; }
  if (!(o.s_sigma > 1.0) || !(o.s_r > 1.0)) { *why = "s_sigma and s_r must be > 1"; return DOT_EINVAL; }
  if (o.check_every < 0) { *why = "check_every must be >= 0"; return DOT_EINVAL; }
  if (!(o.obstacle_weight > 0.0 && std::isfinite(o.obstacle_weight))) {
    *why = "obstacle_weight must be > 0";
    return DOT_EINVAL;
  }
  if (o.prec != DOT_FP64 && o.prec != DOT_MIXED) { *why = "unknown precision"; return DOT_EINVAL; }
  if (!(o.tau_switch_below >= 0.0 && std::isfinite(o.tau_switch_below))) {
    *why = "tau_switch_below must be >= 0";
    return DOT_EINVAL;
  }
  return DOT_OK;
}

struct dot_ctx {
  dot_grid grid;
  dot_options opt;
  Geo geo;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  std::unique_ptr<Path> path;
  double* h_red = nullptr;  // pinned R_NSLOTS doubles + one int (device error flag)
  std::vector<double> m0, m1, omega;
  double sigma = 1.0;
  double tau_cur = 1.9;   // dual step length in use (opt.tau, or 1 after tau_switch_below)
  long iters = 0;
  double kkt[DOT_KKT_LEN];
  std::string err;
  long launches = 0;
  // per-kernel timing (dot_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kid;
  size_t ev_n = 0;
  double prof_ms[KID_COUNT] = {0};
  long prof_cnt[KID_COUNT] = {0};
  // CUDA-graph replay of check periods (dot_solve): the private stream the period
  // is captured on (the caller's stream may be the legacy default stream, which
  // cannot be captured)
  cudaStream_t cap = nullptr;
  int device = 0;           // the device of dot_create; made current by every entry point
};

int dot::context_device(const dot_ctx* c) { return c->device; }

void dot::problem_of(const dot_ctx* c, dot_grid* g, dot_options* opt, void** stream, std::vector<double>* rho0,
                     std::vector<double>* rho1, std::vector<uint8_t>* mask, bool* has_mask) {
  *g = c->grid;
  *opt = c->opt;
  *stream = (void*)c->stream;
  *rho0 = c->m0;
  *rho1 = c->m1;
  mask->assign(c->omega.size(), 0);
  *has_mask = false;
  for (size_t i = 0; i < c->omega.size(); ++i)
    if (c->omega[i] != 1.0) {
      (*mask)[i] = 1;
      *has_mask = true;
    }
}

namespace {

const char* const kKernelNames[KID_COUNT] = {
    "assemble_b", "dct_axis", "dct_scale", "poisson_residual", "poisson_combine", "cone_project",
    "update_q0_alpha0", "update_qd_alphad", "update_beta", "kkt_reductions", "dct_tcgen05", "fused_cone_update",
    "face_beta_residual"};

// Record a CUDA event on the context's stream; kid < 0 marks a start point.
void prof_record(dot_ctx* c, int kid) {
  if (c->ev_n == c->ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->ev.push_back(e);
    c->ev_kid.push_back(-1);
  }
  cudaEventRecord(c->ev[c->ev_n], c->stream);
  c->ev_kid[c->ev_n] = kid;
  ++c->ev_n;
}

void prof_mark(void* user, int kid) { prof_record(static_cast<dot_ctx*>(user), kid); }

// After a stream synchronisation: attribute each interval between consecutive
// events to the kernel launched at its end.
void prof_flush(dot_ctx* c) {
  for (size_t i = 1; i < c->ev_n; ++i) {
    const int kid = c->ev_kid[i];
    if (kid < 0 || kid >= KID_COUNT) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[i - 1], c->ev[i]) == cudaSuccess) {
      c->prof_ms[kid] += ms;
      c->prof_cnt[kid] += 1;
    } else {
      cudaGetLastError();   // a timing query never fails the solve
    }
  }
  c->ev_n = 0;
}

LaunchCounter counter(dot_ctx* c) {
  LaunchCounter lc{&c->launches};
  if (c->prof) {
    lc.mark = prof_mark;
    lc.user = c;
  }
  return lc;
}

int fail(dot_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_thread_err = msg;
  return code;
}

int cuda_fail(dot_ctx* c, cudaError_t e, const char* where) {
  return fail(c, DOT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define DOT_CK(ctx, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

void finish_kkt(dot_ctx* c, const double* r) {
  double cn2 = 0.0;
  for (double v : c->m0) cn2 += v * v;
  for (double v : c->m1) cn2 += v * v;
  kkt_measures(c->geo, cn2, r, c->iters, c->sigma, c->kkt);
}

int compute_kkt(dot_ctx* c) {
  LaunchCounter lc = counter(c);
  if (c->prof) prof_record(c, -1);
  c->path->kkt(c->stream, lc);
  DOT_CK(c, cudaGetLastError());
  DOT_CK(c, cudaMemcpyAsync(c->h_red, c->path->red_out(), sizeof(double) * R_NSLOTS, cudaMemcpyDeviceToHost,
                            c->stream));
  int* hflag = reinterpret_cast<int*>(c->h_red + R_NSLOTS);
  *hflag = 0;
  if (c->path->error_flag())
    DOT_CK(c, cudaMemcpyAsync(hflag, c->path->error_flag(), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DOT_CK(c, cudaStreamSynchronize(c->stream));
  if (c->prof) prof_flush(c);
  if (*hflag) return fail(c, DOT_ECUDA, "a tensor-core pipeline wait timed out (kernel returned early)");
  finish_kkt(c, c->h_red);
  return DOT_OK;
}

constexpr int kNoGraph = 1000;   // PeriodGraphs::period: no graph, run the period directly

// Check periods of dot_solve replayed from CUDA graphs: one graph per parity of
// the iterate buffers, captured on first use from the path's own launch sequence
// (ce iterations, the stopping-measure kernels, the copies of their sums and of
// the pipeline error flag into pinned host memory) and destroyed when the solve
// returns.  Between periods the penalty is applied outside the graph: the kernels
// read sigma and tau from device memory.  Profiled solves (dot_profile) launch
// kernel by kernel: an event node at every kernel boundary inside the graph costs
// more than the graph saves (1,470 against 1,500 iterations/s on 256^2 x 64).
class PeriodGraphs {
 public:
  explicit PeriodGraphs(dot_ctx* c) : c_(c) {}
  ~PeriodGraphs() {
    if (exec_[0] || exec_[1]) cudaStreamSynchronize(c_->stream);
    for (auto& e : exec_)
      if (e) cudaGraphExecDestroy(e);
  }
  // One period: DOT_OK with the stopping measures in c->kkt, an error code, or
  // kNoGraph when this period cannot come from a graph (the caller then runs it
  // kernel by kernel).
  int period(int ce) {
    dot_ctx* c = c_;
    if (broken_ || c->prof || !c->opt.use_graphs || !c->path->graphable() || c->path->residual_carried())
      return kNoGraph;
    c->path->set_penalty(c->sigma, c->tau_cur, c->stream, counter(c));
    const int par = c->path->parity() & 1;
    if (!exec_[par] && !capture(par, ce)) {
      broken_ = true;
      return kNoGraph;
    }
    int* hflag = reinterpret_cast<int*>(c->h_red + R_NSLOTS);
    *hflag = 0;
    DOT_CK(c, cudaGraphLaunch(exec_[par], c->stream));
    c->path->set_parity(par ^ (ce & 1));
    c->launches += launches_[par];
    c->iters += ce;
    DOT_CK(c, cudaStreamSynchronize(c->stream));
    if (*hflag) return fail(c, DOT_ECUDA, "a tensor-core pipeline wait timed out (kernel returned early)");
    finish_kkt(c, c->h_red);
    return DOT_OK;
  }

 private:
  bool capture(int par, int ce) {
    dot_ctx* c = c_;
    if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
      c->cap = nullptr;
      cudaGetLastError();
      return false;
    }
    long n = 0;
    LaunchCounter lc{&n};
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      for (int it = 0; it < ce; ++it) c->path->iterate(c->sigma, c->tau_cur, c->cap, lc);
      c->path->kkt(c->cap, lc);
      cudaMemcpyAsync(c->h_red, c->path->red_out(), sizeof(double) * R_NSLOTS, cudaMemcpyDeviceToHost, c->cap);
      if (c->path->error_flag())
        cudaMemcpyAsync(c->h_red + R_NSLOTS, c->path->error_flag(), sizeof(int), cudaMemcpyDeviceToHost, c->cap);
      e = cudaStreamEndCapture(c->cap, &graph);
    }
    c->path->set_parity(par);   // the capture ran nothing: the buffers are where they were
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec_[par], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      exec_[par] = nullptr;
      cudaGetLastError();
      return false;
    }
    launches_[par] = n;
    return true;
  }

  dot_ctx* c_;
  cudaGraphExec_t exec_[2] = {nullptr, nullptr};
  long launches_[2] = {0, 0};
  bool broken_ = false;
};

}  // namespace

extern "C" {

void dot_default_options(dot_options* o) {
  if (!o) return;
  o->prec = DOT_MIXED;
  o->tau = 1.9;
  o->sigma0 = 1.0;
  o->s_sigma = 1.25;
  o->s_r = 2.0;
  o->check_every = 10;
  o->obstacle_weight = 1e-6;
  o->max_seconds = 0.0;
  o->use_graphs = 1;
  o->tau_switch_below = 3e-7;
}

const char* dot_version(void) { return "dot-gb300 0.1 (sm_103a)"; }

size_t dot_workspace_bytes(const dot_grid* grid, dot_precision prec) {
  std::string why;
  if (!grid_ok(grid, &why)) return 0;
  Geo g = make_geo(*grid);
  return path_workspace_bytes(g, prec);
}

int dot_create(const dot_grid* grid, const double* rho0, const double* rho1, const uint8_t* mask,
               const dot_options* opt, void* workspace, size_t workspace_bytes, void* stream, dot_ctx** out) {
  if (!out) return fail(nullptr, DOT_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  if (!grid_ok(grid, &why)) return fail(nullptr, DOT_EINVAL, why);
  if (!rho0 || !rho1) return fail(nullptr, DOT_EINVAL, "rho0/rho1 is NULL");
  dot_options o;
  dot_default_options(&o);
  if (opt) o = *opt;
  if (check_options(o, &why) != DOT_OK) return fail(nullptr, DOT_EINVAL, why);

  std::unique_ptr<dot_ctx> c(new dot_ctx());
  c->grid = *grid;
  c->opt = o;
  c->geo = make_geo(*grid);
  const Geo& g = c->geo;
  bool any_mask = false;
  if (prepare_densities(g, rho0, rho1, mask, o.obstacle_weight, &c->m0, &c->m1, &c->omega, &any_mask, &why) !=
      DOT_OK)
    return fail(nullptr, DOT_EINVAL, why);
  // the first device call: after every host-side check
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(nullptr, DOT_ECUDA, "no CUDA device");
  c->stream = (cudaStream_t)stream;
  size_t need = path_workspace_bytes(g, o.prec);
  if (workspace) {
    if (workspace_bytes < need)
      return fail(nullptr, DOT_ENOMEM, "workspace smaller than dot_workspace_bytes()");
    if (((uintptr_t)workspace & 255u) != 0) return fail(nullptr, DOT_EINVAL, "workspace must be 256-byte aligned");
    c->ws = (char*)workspace;
    c->ws_bytes = workspace_bytes;
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) return fail(nullptr, DOT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    c->ws = (char*)p;
    c->ws_bytes = need;
    c->own_ws = true;
  }
  cudaError_t e = cudaMallocHost(&c->h_red, sizeof(double) * (R_NSLOTS + 1));
  if (e != cudaSuccess) {
    if (c->own_ws) cudaFree(c->ws);
    return fail(nullptr, DOT_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
  }
  c->path = make_path(o.prec, g);
  std::string perr;
  int rc = c->path->init(c->ws, c->ws_bytes, c->m0, c->m1, any_mask ? &c->omega : nullptr, c->stream, &perr);
  if (rc != DOT_OK) {
    cudaFreeHost(c->h_red);
    if (c->own_ws) cudaFree(c->ws);
    return fail(nullptr, rc, perr);
  }
  c->sigma = o.sigma0;
  c->tau_cur = o.tau;
  c->iters = 0;
  for (int i = 0; i < DOT_KKT_LEN; ++i) c->kkt[i] = NAN;
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFreeHost(c->h_red);
    if (c->own_ws) cudaFree(c->ws);
    return fail(nullptr, DOT_ECUDA, std::string("dot_create: ") + cudaGetErrorString(e));
  }
  *out = c.release();
  return DOT_OK;
}

int dot_solve(dot_ctx* c, double tol, long maxit) {
  if (!c) return fail(nullptr, DOT_EINVAL, "ctx is NULL");
  DeviceScope dev(c->device);
  if (maxit < 0) return fail(c, DOT_EINVAL, "maxit must be >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  const int ce = c->opt.check_every;
  LaunchCounter lc = counter(c);
  PeriodGraphs graphs(c);
  long k = 0;   // iterations done by this call
  while (k < maxit) {
    bool checked = false;
    // a whole check period from a CUDA graph: ce iterations and the stopping
    // measures, the same kernels in the same order as the loop below
    if (ce > 0 && k % ce == 0 && k + ce <= maxit) {
      const int rc = graphs.period(ce);
      if (rc != kNoGraph) {
        if (rc != DOT_OK) return rc;
        k += ce;
        checked = true;
      }
    }
    if (!checked) {
      if (c->prof) {
        if (c->ev_n > 4096) {
          DOT_CK(c, cudaStreamSynchronize(c->stream));
          prof_flush(c);
        }
        prof_record(c, -1);
      }
      c->path->iterate(c->sigma, c->tau_cur, c->stream, lc);
      ++c->iters;
      ++k;
      if (ce > 0 && k % ce == 0) {
        const int rc = compute_kkt(c);
        if (rc != DOT_OK) return rc;
        checked = true;
      }
    }
    if (checked) {
      c->path->end_period();
      const double eta = c->kkt[DOT_KKT_ETA];
      if (!std::isfinite(eta)) return fail(c, DOT_EDIVERGED, "stopping measure is not finite");
      if (tol > 0.0 && eta <= tol) return DOT_OK;
      // mixed path near its FP32 floor: the ALG2 step from now on
      if (c->opt.prec == DOT_MIXED && c->opt.tau_switch_below > 0.0 && eta <= c->opt.tau_switch_below)
        c->tau_cur = 1.0;
      // penalty rule (Sec. 5.3) on eta_P^soc / eta_D^soc
      const double ratio = c->kkt[DOT_KKT_ETA_P_SOC] / c->kkt[DOT_KKT_ETA_D_SOC];
      if (ratio > c->opt.s_r)
        c->sigma *= c->opt.s_sigma;
      else if (ratio < 1.0 / c->opt.s_r)
        c->sigma /= c->opt.s_sigma;
      if (c->opt.max_seconds > 0.0 && elapsed_s(t0) > c->opt.max_seconds)
        return fail(c, DOT_ETIMEOUT, "max_seconds elapsed");
    }
  }
  DOT_CK(c, cudaGetLastError());
  DOT_CK(c, cudaStreamSynchronize(c->stream));
  if (c->prof) prof_flush(c);
  return DOT_ENOTCONV;
}

int dot_kkt(dot_ctx* c, double* kkt) {
  if (!c) return fail(nullptr, DOT_EINVAL, "ctx is NULL");
  DeviceScope dev(c->device);
  int rc = compute_kkt(c);
  if (rc != DOT_OK) return rc;
  if (kkt) std::memcpy(kkt, c->kkt, sizeof(c->kkt));
  return DOT_OK;
}

int dot_get(dot_ctx* c, double* rho, double* m, double* phi, double* objective, double* kkt) {
  if (!c) return fail(nullptr, DOT_EINVAL, "ctx is NULL");
  DeviceScope dev(c->device);
  const Geo& g = c->geo;
  if (objective || kkt) {
    int rc = compute_kkt(c);
    if (rc != DOT_OK) return rc;
    if (objective) *objective = -2.0 * c->kkt[DOT_KKT_PRIMAL] / (double)c->geo.P;
    if (kkt) std::memcpy(kkt, c->kkt, sizeof(c->kkt));
  }
  std::string perr;
  int rc = c->path->read_fields(rho, m, phi, c->stream, &perr);
  if (rc != DOT_OK) return fail(c, rc, perr);
  const double invh0 = (double)g.T;   // rho = alpha_0 / h_0, m = alpha_bar / h_0
  if (rho) {
    const long long n0 = (long long)g.T * g.P;
    for (long long i = 0; i < n0; ++i) rho[i] *= invh0;
  }
  if (m) {
    long long nm = 0;
    for (int d = 0; d < g.D; ++d) nm += (long long)(g.T + 1) * g.P / g.N[d] * (g.N[d] - 1);
    for (long long i = 0; i < nm; ++i) m[i] *= invh0;
  }
  return DOT_OK;
}

int dot_get_state(dot_ctx* c, double* q, double* alpha, double* beta, double* sigma, long* iters) {
  if (!c) return fail(nullptr, DOT_EINVAL, "ctx is NULL");
  DeviceScope dev(c->device);
  std::string perr;
  int rc = c->path->read_state(q, alpha, beta, c->stream, &perr);
  if (rc != DOT_OK) return fail(c, rc, perr);
  if (sigma) *sigma = c->sigma;
  if (iters) *iters = c->iters;
  return DOT_OK;
}

int dot_set_state(dot_ctx* c, const double* q, const double* alpha, const double* beta, double sigma,
                  long iters) {
  if (!c) return fail(nullptr, DOT_EINVAL, "ctx is NULL");
  DeviceScope dev(c->device);
  if (!q || !alpha || !beta) return fail(c, DOT_EINVAL, "q, alpha and beta are required");
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(c, DOT_EINVAL, "sigma must be > 0");
  std::string perr;
  int rc = c->path->write_state(q, alpha, beta, sigma, c->stream, &perr);
  if (rc != DOT_OK) return fail(c, rc, perr);
  c->sigma = sigma;
  c->iters = iters;
  c->tau_cur = c->opt.tau;
  return DOT_OK;
}

int dot_poisson(dot_ctx* c, const double* b, double* phi) {
  if (!c) return fail(nullptr, DOT_EINVAL, "ctx is NULL");
  DeviceScope dev(c->device);
  if (!b || !phi) return fail(c, DOT_EINVAL, "b and phi are required");
  std::string perr;
  LaunchCounter lc = counter(c);
  if (c->prof) prof_record(c, -1);
  int rc = c->path->poisson_op(b, phi, c->stream, lc, &perr);
  if (c->prof) prof_flush(c);
  if (rc != DOT_OK) return fail(c, rc, perr);
  return DOT_OK;
}

int dot_profile(dot_ctx* c, int enable) {
  if (!c) return fail(nullptr, DOT_EINVAL, "ctx is NULL");
  DeviceScope dev(c->device);
  DOT_CK(c, cudaStreamSynchronize(c->stream));
  if (c->prof) prof_flush(c);
  c->prof = enable != 0;
  if (c->prof) {
    for (int i = 0; i < KID_COUNT; ++i) { c->prof_ms[i] = 0.0; c->prof_cnt[i] = 0; }
    c->ev_n = 0;
  }
  return DOT_OK;
}

int dot_profile_read(dot_ctx* c, double* ms_total, long* launches, int max) {
  if (!c) return fail(nullptr, DOT_EINVAL, "ctx is NULL");
  for (int i = 0; i < max && i < KID_COUNT; ++i) {
    if (ms_total) ms_total[i] = c->prof_ms[i];
    if (launches) launches[i] = c->prof_cnt[i];
  }
  return KID_COUNT;
}

const char* dot_kernel_name(int id) { return (id >= 0 && id < KID_COUNT) ? kKernelNames[id] : ""; }

void dot_destroy(dot_ctx* c) {
  if (!c) return;
  DeviceScope dev(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->cap) cudaStreamDestroy(c->cap);
  c->path.reset();
  if (c->h_red) cudaFreeHost(c->h_red);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  delete c;
}

const char* dot_last_error(const dot_ctx* c) { return c ? c->err.c_str() : g_thread_err.c_str(); }

long dot_launch_count(const dot_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
