// dot_server.cu -- continuous batching of many DOT solves on one GPU (the
// dot_server_* functions of include/dot.h).
//
// One server thread owns the device work.  Requests of one grid share a batch
// (MixedBatch: G slots whose kernels advance together); a batch's period --
// check_every iterations of Algorithm 2 and the stopping measures -- is one CUDA
// graph launch on the batch's stream, followed by a copy of the per-slot
// measures into pinned memory and an event.  The thread polls the events; when a
// period ends it applies the stopping test and penalty rule of Sec. 5.3 per slot
// (the same host code as dot_solve), retires finished slots (copying their
// results out), admits queued requests into free slots and launches the next
// period.  Batches are created while their workspace fits the memory budget and
// freed after idling.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dot.h"
#include "dot_batch.cuh"

using namespace dot;

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2 };

struct Request {
  long long id = 0;
  dot_grid grid;
  Geo geo;
  std::vector<double> m0, m1, omega;
  bool has_mask = false;
  double cn2 = 0.0;
  double tol = 1e-6;
  long maxit = 0;
  bool keep = true;
  ReqState state = Q_QUEUED;
  int status = DOT_OK;
  long iters = 0;
  double sigma = 1.0;
  double tau = 1.9;        // dual step length in use (as dot_solve: 1 after tau_switch_below)
  double kkt[DOT_KKT_LEN];
  double objective = NAN;
  std::vector<double> rho, m, phi;
  double t_submit = 0, t_admit = 0, t_done = 0;
  // multilevel warm start (Sec. 5): the grids and the caller's densities coarsest
  // first, the request's own grid last; lv = the level in progress.  Each level is
  // served like a request of its grid; a finished coarse level's state, prolonged,
  // starts the next one (as dot_solve_multilevel does with contexts).
  std::vector<dot_grid> ml_grid;
  std::vector<std::vector<double>> ml_r0, ml_r1;
  std::vector<std::vector<uint8_t>> ml_mask;
  int lv = 0;
  double tol_final = 1e-6;
  std::vector<double> init_q, init_al, init_beta;   // prolonged state for the next admission
  double init_sigma = 0.0;
};

struct Batch {
  dot_grid grid;
  Geo geo;
  int G = 1;
  char* ws = nullptr;
  size_t bytes = 0;
  std::unique_ptr<MixedBatch> mb;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // by the parity of the double-buffered set
  long graph_launches[2] = {0, 0};
  double* h_red = nullptr;                         // pinned: G x R_NSLOTS doubles + error flag
  std::vector<Request*> slot;
  bool running = false;
  int period = 0;                                  // iterations of the period in flight
  Clock::time_point idle_since;
  int active() const {
    int n = 0;
    for (Request* r : slot) n += r != nullptr;
    return n;
  }
};

bool same_grid(const dot_grid& a, const dot_grid& b) {
  if (a.D != b.D || a.T != b.T) return false;
  for (int d = 0; d < a.D; ++d)
    if (a.N[d] != b.N[d]) return false;
  return true;
}

long long nodes_of(const dot_grid& g) {
  long long n = g.T + 1;
  for (int d = 0; d < g.D; ++d) n *= g.N[d];
  return n;
}

}  // namespace

struct dot_server {
  dot_options opt;
  dot_server_options sopt;
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_done;    // a request finished
  std::condition_variable cv_work;    // a request arrived / stop
  std::deque<Request*> incoming;      // submitted, not yet seen by the thread
  std::deque<Request*> queued;        // seen, waiting for a slot (thread only)
  std::map<long long, std::unique_ptr<Request>> reqs;
  std::vector<std::unique_ptr<Batch>> batches;   // thread only
  long long next_id = 1;
  size_t bytes_held = 0;
  double n_finished = 0, graph_launches = 0, kernel_launches = 0, peak_running = 0, peak_batches = 0;
  double n_queued = 0, n_running = 0, n_batches = 0, n_bytes = 0;
  bool stop = false;
  std::string err;          // last API error (guarded by mu)
  std::string fatal;        // set by the thread when the device failed
  std::thread th;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void run();
  bool admit(Request* r);
  Batch* new_batch(const Request& r);
  void launch_period(Batch& b);
  void finish_period(Batch& b);
  void retire(Batch& b, int k, int status);
  void free_batch(Batch& b);
  void fail_all(const std::string& why);
  bool next_level(Batch& b, int k);
};

namespace {

thread_local std::string g_srv_err;

// Make level lv of request r's multilevel strategy the one it is served at: its
// grid, its densities (prepared as dot_create prepares them) and its tolerance.
int set_level(Request* r, int lv, const dot_options& opt, double coarse_tol, std::string* why) {
  const int L = (int)r->ml_grid.size() - 1;
  r->lv = lv;
  r->grid = r->ml_grid[lv];
  r->geo = make_geo(r->grid);
  const bool masked = !r->ml_mask[lv].empty();
  r->m0.clear();
  r->m1.clear();
  r->omega.clear();
  const int rc = prepare_densities(r->geo, r->ml_r0[lv].data(), r->ml_r1[lv].data(),
                                   masked ? r->ml_mask[lv].data() : nullptr, opt.obstacle_weight, &r->m0, &r->m1,
                                   &r->omega, &r->has_mask, why);
  r->cn2 = 0.0;
  for (double v : r->m0) r->cn2 += v * v;
  for (double v : r->m1) r->cn2 += v * v;
  r->tol = lv == L ? r->tol_final : level_tol(r->tol_final, coarse_tol, L - lv);
  return rc;
}

// Elements of q (and alpha) and of beta in the natural layouts of the C ABI.
long long state_q_len(const dot_grid& g) {
  long long P = 1;
  for (int d = 0; d < g.D; ++d) P *= g.N[d];
  long long n = (long long)g.T * P;
  for (int d = 0; d < g.D; ++d) n += (long long)(g.T + 1) * (P / g.N[d]) * (g.N[d] - 1);
  return n;
}
long long state_beta_len(const dot_grid& g) {
  long long P = 1;
  for (int d = 0; d < g.D; ++d) P *= g.N[d];
  return (long long)(4 * g.D + 2) * g.T * P;
}

int sfail(dot_server* s, int code, const std::string& m) {
  if (s) {
    std::lock_guard<std::mutex> l(s->mu);
    s->err = m;
  } else {
    g_srv_err = m;
  }
  return code;
}

}  // namespace

Batch* dot_server::new_batch(const Request& r) {
  const Geo& g = r.geo;
  int G = 1;
  if (MixedBatch::batchable(g)) {
    const long long per = nodes_of(r.grid);
    long long want = (sopt.target_nodes + per - 1) / per;
    G = (int)std::max(1LL, std::min<long long>(want, sopt.max_slots));
  }
  const bool masks = true;
  size_t bytes = MixedBatch::workspace_bytes(g, G, masks);
  // shrink the batch until it fits what is left of the budget
  while (G > 1 && bytes_held + bytes > sopt.hbm_budget) {
    G = G / 2;
    bytes = MixedBatch::workspace_bytes(g, G, masks);
  }
  if (bytes_held + bytes > sopt.hbm_budget) return nullptr;
  std::unique_ptr<Batch> b(new Batch());
  b->grid = r.grid;
  b->geo = g;
  b->G = G;
  b->bytes = bytes;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  b->ws = (char*)p;
  // batches of small grids get the higher priority: their periods are short
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  const int prio = nodes_of(r.grid) < 1000000 ? hi : lo;
  cudaError_t e = cudaStreamCreateWithPriority(&b->stream, cudaStreamNonBlocking, prio);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_red, sizeof(double) * ((size_t)G * R_NSLOTS + 1));
  if (e != cudaSuccess) {
    free_batch(*b);
    return nullptr;
  }
  b->mb.reset(new MixedBatch(g, G, masks));
  std::string why;
  if (b->mb->init(b->ws, bytes, b->stream, &why) != DOT_OK) {
    free_batch(*b);
    return nullptr;
  }
  b->slot.assign(G, nullptr);
  b->idle_since = Clock::now();
  bytes_held += bytes;
  batches.push_back(std::move(b));
  {
    std::lock_guard<std::mutex> l(mu);
    peak_batches = std::max(peak_batches, (double)batches.size());
  }
  return batches.back().get();
}

void dot_server::free_batch(Batch& b) {
  if (b.stream) cudaStreamSynchronize(b.stream);
  for (int k = 0; k < 2; ++k)
    if (b.graph[k]) cudaGraphExecDestroy(b.graph[k]);
  b.mb.reset();
  if (b.h_red) cudaFreeHost(b.h_red);
  if (b.done) cudaEventDestroy(b.done);
  if (b.stream) cudaStreamDestroy(b.stream);
  if (b.ws) cudaFree(b.ws);
  b.ws = nullptr;
  b.h_red = nullptr;
  b.done = nullptr;
  b.stream = nullptr;
  b.graph[0] = b.graph[1] = nullptr;
}

// Put r into a free slot of a batch of its grid (creating one if memory allows).
bool dot_server::admit(Request* r) {
  Batch* target = nullptr;
  int k = -1;
  for (auto& b : batches) {
    if (b->running || !same_grid(b->grid, r->grid)) continue;
    for (int j = 0; j < b->G; ++j)
      if (!b->slot[j]) { target = b.get(); k = j; break; }
    if (target) break;
  }
  if (!target) {
    // a running batch of this grid with a free slot takes the request after its period
    for (auto& b : batches)
      if (same_grid(b->grid, r->grid) && b->active() < b->G) return false;
    target = new_batch(*r);
    if (!target) return false;
    k = 0;
  }
  std::string why;
  r->tau = opt.tau;
  if (target->mb->load_slot(k, r->m0, r->m1, r->has_mask ? &r->omega : nullptr, opt.sigma0, r->tau,
                            target->stream, &why) != DOT_OK) {
    fail_all("load_slot: " + why);
    return false;
  }
  r->sigma = opt.sigma0;
  if (!r->init_q.empty()) {
    // a finer level of the multilevel strategy: start from the prolonged state
    if (target->mb->write_state(k, r->init_q.data(), r->init_al.data(), r->init_beta.data(), r->init_sigma, r->tau,
                                target->stream, &why) != DOT_OK) {
      fail_all("write_state: " + why);
      return false;
    }
    r->sigma = r->init_sigma;
    r->init_q = std::vector<double>();
    r->init_al = std::vector<double>();
    r->init_beta = std::vector<double>();
  }
  target->slot[k] = r;
  r->iters = 0;
  std::lock_guard<std::mutex> l(mu);
  r->state = Q_RUNNING;
  if (r->t_admit == 0.0) r->t_admit = now();
  return true;
}

void dot_server::launch_period(Batch& b) {
  const int ce = opt.check_every > 0 ? opt.check_every : 10;
  long launches = 0;
  LaunchCounter lc{&launches};
  cudaError_t e = b.mb->upload_params(b.stream);
  const int par = b.mb->parity();
  if (e == cudaSuccess && sopt.use_graphs) {
    if (!b.graph[par]) {
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        b.mb->apply_rescale(b.stream, lc);     // penalty changes since the last period
        for (int it = 0; it < ce; ++it) b.mb->iterate(b.stream, lc);
        b.mb->kkt(b.stream, lc);
        e = cudaStreamEndCapture(b.stream, &graph);
        b.mb->set_parity(par);   // capture ran no kernel: the buffers are where they were
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b.graph[par], graph, 0);
      if (graph) cudaGraphDestroy(graph);
      b.graph_launches[par] = launches;
      launches = 0;
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b.graph[par], b.stream);
    b.mb->set_parity(par ^ (ce & 1));
    launches = b.graph_launches[par];
  } else if (e == cudaSuccess) {
    b.mb->apply_rescale(b.stream, lc);
    for (int it = 0; it < ce; ++it) b.mb->iterate(b.stream, lc);
    b.mb->kkt(b.stream, lc);
    e = cudaGetLastError();
  }
  b.mb->clear_rescale();   // the launched period applied the factors the device holds
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.h_red, b.mb->red_out(), sizeof(double) * (size_t)b.G * R_NSLOTS, cudaMemcpyDeviceToHost,
                        b.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.h_red + (size_t)b.G * R_NSLOTS, b.mb->error_flag(), sizeof(int), cudaMemcpyDeviceToHost,
                        b.stream);
  if (e == cudaSuccess) e = cudaEventRecord(b.done, b.stream);
  if (e != cudaSuccess) {
    fail_all(std::string("launch: ") + cudaGetErrorString(e));
    return;
  }
  b.running = true;
  b.period = ce;
  std::lock_guard<std::mutex> l(mu);
  graph_launches += 1;
  kernel_launches += (double)launches;
}

// A coarse level of slot k's request has finished: its state, prolonged to the next
// finer grid, starts that level, for which the request is queued again.
bool dot_server::next_level(Batch& b, int k) {
  Request* r = b.slot[k];
  const dot_grid gc = r->ml_grid[r->lv], gf = r->ml_grid[r->lv + 1];
  std::vector<double> q(state_q_len(gc)), al(state_q_len(gc)), beta(state_beta_len(gc));
  std::string why;
  if (b.mb->read_state(k, q.data(), al.data(), beta.data(), b.stream, &why) != DOT_OK) return false;
  r->init_q.assign(state_q_len(gf), 0.0);
  r->init_al.assign(state_q_len(gf), 0.0);
  r->init_beta.assign(state_beta_len(gf), 0.0);
  if (dot_prolong_state(&gc, &gf, q.data(), al.data(), beta.data(), r->init_q.data(), r->init_al.data(),
                        r->init_beta.data()) != DOT_OK)
    return false;
  r->init_sigma = r->sigma;
  if (set_level(r, r->lv + 1, opt, sopt.multilevel_coarse_tol, &why) != DOT_OK) return false;
  b.mb->set_active(k, false);
  b.slot[k] = nullptr;
  if (b.active() == 0) b.idle_since = Clock::now();
  queued.push_front(r);   // ahead of later arrivals: it has waited already
  return true;
}

void dot_server::retire(Batch& b, int k, int status) {
  Request* r = b.slot[k];
  if (status >= 0 && r->lv + 1 < (int)r->ml_grid.size()) {
    if (next_level(b, k)) return;
    status = DOT_ECUDA;
  }
  if (status >= 0 && r->keep) {
    const Geo& g = b.geo;
    const long long n0 = (long long)g.T * g.P, nn = (long long)(g.T + 1) * g.P;
    long long nm = 0;
    for (int d = 0; d < g.D; ++d) nm += (long long)(g.T + 1) * g.P / g.N[d] * (g.N[d] - 1);
    r->rho.resize(n0);
    r->m.resize(nm);
    r->phi.resize(nn);
    std::string why;
    if (b.mb->read_fields(k, r->rho.data(), r->m.data(), r->phi.data(), b.stream, &why) != DOT_OK) {
      status = DOT_ECUDA;
    } else {
      const double invh0 = (double)g.T;   // rho = alpha_0 / h_0, m = alpha_bar / h_0
      for (double& v : r->rho) v *= invh0;
      for (double& v : r->m) v *= invh0;
    }
  }
  r->objective = -2.0 * r->kkt[DOT_KKT_PRIMAL] / (double)b.geo.P;
  b.mb->set_active(k, false);
  b.slot[k] = nullptr;
  if (b.active() == 0) b.idle_since = Clock::now();
  std::lock_guard<std::mutex> l(mu);
  r->status = status;
  r->state = Q_DONE;
  r->t_done = now();
  r->m0.clear();
  r->m1.clear();
  r->omega.clear();
  r->m0.shrink_to_fit();
  r->m1.shrink_to_fit();
  r->omega.shrink_to_fit();
  n_finished += 1;
  cv_done.notify_all();
}

void dot_server::finish_period(Batch& b) {
  b.running = false;
  b.mb->end_period();
  const int* flag = reinterpret_cast<const int*>(b.h_red + (size_t)b.G * R_NSLOTS);
  if (*flag) {
    for (int k = 0; k < b.G; ++k)
      if (b.slot[k]) retire(b, k, DOT_ECUDA);
    return;
  }
  for (int k = 0; k < b.G; ++k) {
    Request* r = b.slot[k];
    if (!r) continue;
    r->iters += b.period;
    kkt_measures(b.geo, r->cn2, b.h_red + (size_t)k * R_NSLOTS, r->iters, r->sigma, r->kkt);
    const double eta = r->kkt[DOT_KKT_ETA];
    if (!std::isfinite(eta)) { retire(b, k, DOT_EDIVERGED); continue; }
    if (r->tol > 0.0 && eta <= r->tol) { retire(b, k, DOT_OK); continue; }
    if (r->iters >= r->maxit) { retire(b, k, DOT_ENOTCONV); continue; }
    // near the mixed path's FP32 floor: the ALG2 step from now on (as dot_solve)
    if (opt.tau_switch_below > 0.0 && eta <= opt.tau_switch_below) r->tau = 1.0;
    // penalty rule (Sec. 5.3) on eta_P^soc / eta_D^soc
    const double ratio = r->kkt[DOT_KKT_ETA_P_SOC] / r->kkt[DOT_KKT_ETA_D_SOC];
    if (ratio > opt.s_r)
      r->sigma *= opt.s_sigma;
    else if (ratio < 1.0 / opt.s_r)
      r->sigma /= opt.s_sigma;
    b.mb->set_sigma(k, r->sigma, r->tau, true);
  }
}

void dot_server::fail_all(const std::string& why) {
  std::lock_guard<std::mutex> l(mu);
  fatal = why;
  for (auto& kv : reqs) {
    Request* r = kv.second.get();
    if (r->state != Q_DONE) {
      r->state = Q_DONE;
      r->status = DOT_ECUDA;
      r->t_done = now();
    }
  }
  incoming.clear();
  queued.clear();
  for (auto& b : batches) std::fill(b->slot.begin(), b->slot.end(), nullptr);
  stop = true;
  cv_done.notify_all();
}

void dot_server::run() {
  cudaSetDevice(device);
  for (;;) {
    {
      std::unique_lock<std::mutex> l(mu);
      bool busy = false;
      for (auto& b : batches) busy = busy || b->running || b->active() > 0;
      if (!stop && incoming.empty() && queued.empty() && !busy)
        cv_work.wait_for(l, std::chrono::milliseconds(5));
      if (stop) break;
      while (!incoming.empty()) {
        queued.push_back(incoming.front());
        incoming.pop_front();
      }
    }
    // periods that ended
    for (auto& b : batches)
      if (b->running && cudaEventQuery(b->done) == cudaSuccess) finish_period(*b);
    if (stop) break;
    // admission in arrival order (a request that cannot be placed does not block
    // requests of other grids)
    for (auto it = queued.begin(); it != queued.end();) {
      if (admit(*it)) it = queued.erase(it);
      else ++it;
      if (stop) break;
    }
    if (stop) break;
    // idle batches: launch the next period, or free the memory of empty ones
    for (auto& b : batches)
      if (!b->running && b->active() > 0) launch_period(*b);
    if (stop) break;
    const auto tnow = Clock::now();
    for (size_t i = 0; i < batches.size();) {
      Batch& b = *batches[i];
      const double idle = std::chrono::duration<double, std::milli>(tnow - b.idle_since).count();
      if (!b.running && b.active() == 0 && (idle > sopt.idle_ms || !queued.empty())) {
        bytes_held -= b.bytes;
        free_batch(b);
        batches.erase(batches.begin() + i);
      } else {
        ++i;
      }
    }
    {
      std::lock_guard<std::mutex> l(mu);
      double running = 0;
      for (auto& b : batches) running += b->active();
      n_running = running;
      n_queued = (double)queued.size();
      n_batches = (double)batches.size();
      n_bytes = (double)bytes_held;
      peak_running = std::max(peak_running, running);
    }
    // nothing finished yet: yield briefly instead of spinning on the events
    bool any_running = false;
    for (auto& b : batches) any_running = any_running || b->running;
    if (any_running) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  for (auto& b : batches) free_batch(*b);
  batches.clear();
  bytes_held = 0;
}

extern "C" {

void dot_server_default_options(dot_server_options* o) {
  if (!o) return;
  o->hbm_budget = 0;
  o->max_slots = 64;
  o->target_nodes = 4194304;
  o->use_graphs = 1;
  o->idle_ms = 200;
  o->multilevel = 0;
  o->multilevel_min_nodes = 1000000;
  o->multilevel_coarse_tol = 0.0;
  o->multilevel_masked = 0;
}

int dot_server_create(const dot_options* opt, const dot_server_options* sopt, dot_server** out) {
  if (!out) return sfail(nullptr, DOT_EINVAL, "out is NULL");
  *out = nullptr;
  dot_options o;
  dot_default_options(&o);
  if (opt) o = *opt;
  std::string why;
  if (check_options(o, &why) != DOT_OK) return sfail(nullptr, DOT_EINVAL, why);
  if (o.prec != DOT_MIXED) return sfail(nullptr, DOT_EINVAL, "the server runs DOT_MIXED solves");
  dot_server_options so;
  dot_server_default_options(&so);
  if (sopt) so = *sopt;
  if (so.max_slots < 1 || so.max_slots > 256) return sfail(nullptr, DOT_EINVAL, "max_slots must lie in [1, 256]");
  if (so.target_nodes < 1) return sfail(nullptr, DOT_EINVAL, "target_nodes must be >= 1");
  if (so.multilevel < 0 || so.multilevel > 8) return sfail(nullptr, DOT_EINVAL, "multilevel must lie in [0, 8]");
  if (!(so.multilevel_coarse_tol >= 0.0)) return sfail(nullptr, DOT_EINVAL, "multilevel_coarse_tol must be >= 0");
  std::unique_ptr<dot_server> s(new dot_server());
  s->opt = o;
  if (cudaGetDevice(&s->device) != cudaSuccess) return sfail(nullptr, DOT_ECUDA, "no CUDA device");
  if (so.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return sfail(nullptr, DOT_ECUDA, "cudaMemGetInfo failed");
    so.hbm_budget = (size_t)(0.8 * (double)fr);
  }
  s->sopt = so;
  s->t0 = Clock::now();
  dot_server* raw = s.get();
  s->th = std::thread([raw]() { raw->run(); });
  *out = s.release();
  return DOT_OK;
}

int dot_server_submit(dot_server* s, const dot_grid* grid, const double* rho0, const double* rho1,
                      const uint8_t* mask, double tol, long maxit, int keep_fields, long long* id) {
  if (!s) return sfail(nullptr, DOT_EINVAL, "server is NULL");
  if (!id) return sfail(s, DOT_EINVAL, "id is NULL");
  std::string why;
  if (!grid_valid(grid, &why)) return sfail(s, DOT_EINVAL, why);
  if (!rho0 || !rho1) return sfail(s, DOT_EINVAL, "rho0/rho1 is NULL");
  if (maxit < 0) return sfail(s, DOT_EINVAL, "maxit must be >= 0");
  std::unique_ptr<Request> r(new Request());
  r->grid = *grid;
  r->geo = make_geo(*grid);
  if (r->geo.T + 1 > 160) return sfail(s, DOT_EINVAL, "DOT_MIXED supports T + 1 <= 160 time nodes");
  if (prepare_densities(r->geo, rho0, rho1, mask, s->opt.obstacle_weight, &r->m0, &r->m1, &r->omega, &r->has_mask,
                        &why) != DOT_OK)
    return sfail(s, DOT_EINVAL, why);
  // a request that cannot fit the budget even in a batch of one slot would wait forever
  const size_t need = MixedBatch::workspace_bytes(r->geo, 1, true);
  if (need > s->sopt.hbm_budget)
    return sfail(s, DOT_ENOMEM, "the request needs " + std::to_string(need) +
                                    " bytes of workspace, more than the server's hbm_budget");
  for (double v : r->m0) r->cn2 += v * v;
  for (double v : r->m1) r->cn2 += v * v;
  r->tol = tol;
  r->maxit = maxit;
  r->keep = keep_fields != 0;
  const int L = s->sopt.multilevel;
  std::string mwhy;
  if (L > 0 && nodes_of(*grid) >= s->sopt.multilevel_min_nodes && (!r->has_mask || s->sopt.multilevel_masked) &&
      multilevel_ok(*grid, L, &mwhy)) {
    // the pyramid of the multilevel strategy, served coarsest first: the prepared
    // densities and the obstacle cells (weight != 1) averaged as dot_solve_multilevel
    // averages a context's
    std::vector<dot_grid> gs(L + 1);
    std::vector<std::vector<double>> R0(L + 1), R1(L + 1);
    std::vector<std::vector<uint8_t>> M(L + 1);
    const bool masked = r->has_mask;
    gs[0] = *grid;
    R0[0] = r->m0;
    R1[0] = r->m1;
    if (masked) {
      M[0].assign(r->omega.size(), 0);
      for (size_t i = 0; i < r->omega.size(); ++i) M[0][i] = r->omega[i] != 1.0;
    }
    for (int v = 1; v <= L; ++v) {
      coarsen(gs[v - 1], R0[v - 1], masked ? &M[v - 1] : nullptr, &gs[v], &R0[v], &M[v]);
      dot_grid gtmp;
      std::vector<uint8_t> mtmp;
      coarsen(gs[v - 1], R1[v - 1], nullptr, &gtmp, &R1[v], &mtmp);
    }
    // the caller's own grid keeps the caller's densities, prepared as at submission
    const long long P = r->geo.P;
    R0[0].assign(rho0, rho0 + P);
    R1[0].assign(rho1, rho1 + P);
    M[0] = mask ? std::vector<uint8_t>(mask, mask + P) : std::vector<uint8_t>();
    for (int v = L; v >= 0; --v) {
      r->ml_grid.push_back(gs[v]);
      r->ml_r0.push_back(std::move(R0[v]));
      r->ml_r1.push_back(std::move(R1[v]));
      r->ml_mask.push_back(v == 0 || masked ? std::move(M[v]) : std::vector<uint8_t>());
    }
    r->tol_final = tol;
    if (set_level(r.get(), 0, s->opt, s->sopt.multilevel_coarse_tol, &why) != DOT_OK) return sfail(s, DOT_EINVAL, why);
  }
  for (int i = 0; i < DOT_KKT_LEN; ++i) r->kkt[i] = NAN;
  std::lock_guard<std::mutex> l(s->mu);
  if (!s->fatal.empty()) {
    s->err = "the server stopped: " + s->fatal;
    return DOT_ECUDA;
  }
  r->id = s->next_id++;
  r->t_submit = s->now();
  *id = r->id;
  s->incoming.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  s->cv_work.notify_one();
  return DOT_OK;
}

int dot_server_wait(dot_server* s, long long id, double timeout_s, int* status) {
  if (!s) return sfail(nullptr, DOT_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> l(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    s->err = "unknown request id";
    return DOT_EINVAL;
  }
  Request* r = it->second.get();
  auto done = [r]() { return r->state == Q_DONE; };
  if (timeout_s < 0) s->cv_done.wait(l, done);
  else if (timeout_s > 0) s->cv_done.wait_for(l, std::chrono::duration<double>(timeout_s), done);
  if (!done()) return DOT_ETIMEOUT;
  if (status) *status = r->status;
  return DOT_OK;
}

int dot_server_result(dot_server* s, long long id, double* rho, double* m, double* phi, double* objective,
                      double* kkt, double* times) {
  if (!s) return sfail(nullptr, DOT_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> l(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    s->err = "unknown request id";
    return DOT_EINVAL;
  }
  Request* r = it->second.get();
  if (r->state != Q_DONE) {
    s->err = "request has not finished";
    return DOT_EINVAL;
  }
  if ((rho || m || phi) && (r->rho.empty() || r->phi.empty())) {
    s->err = "fields were not kept (keep_fields = 0, or the solve failed)";
    return DOT_EINVAL;
  }
  if (rho) std::memcpy(rho, r->rho.data(), r->rho.size() * sizeof(double));
  if (m) std::memcpy(m, r->m.data(), r->m.size() * sizeof(double));
  if (phi) std::memcpy(phi, r->phi.data(), r->phi.size() * sizeof(double));
  if (objective) *objective = r->objective;
  if (kkt) std::memcpy(kkt, r->kkt, sizeof(r->kkt));
  if (times) {
    times[0] = r->t_submit;
    times[1] = r->t_admit;
    times[2] = r->t_done;
  }
  return DOT_OK;
}

int dot_server_release(dot_server* s, long long id) {
  if (!s) return sfail(nullptr, DOT_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> l(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second->state != Q_DONE) {
    s->err = "unknown or unfinished request";
    return DOT_EINVAL;
  }
  s->reqs.erase(it);
  return DOT_OK;
}

int dot_server_stats(dot_server* s, double* out, int n) {
  if (!s || !out) return 0;
  std::lock_guard<std::mutex> l(s->mu);
  const double v[9] = {s->n_queued + (double)s->incoming.size(), s->n_running, s->n_finished, s->n_batches,
                       s->n_bytes, s->graph_launches, s->kernel_launches, s->peak_running, s->peak_batches};
  int k = 0;
  for (; k < n && k < 9; ++k) out[k] = v[k];
  return k;
}

void dot_server_destroy(dot_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> l(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  delete s;
}

const char* dot_server_last_error(const dot_server* s) {
  if (!s) return g_srv_err.c_str();
  // the server thread may set `fatal` at any time: copy under the lock into a
  // buffer of the calling thread (valid until its next call)
  thread_local std::string copy;
  {
    std::lock_guard<std::mutex> l(const_cast<dot_server*>(s)->mu);
    copy = s->err.empty() ? s->fatal : s->err;
  }
  return copy.c_str();
}

}  // extern "C"
