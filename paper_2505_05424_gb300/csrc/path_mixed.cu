// path_mixed.cu -- the mixed-precision path of Algorithm 2 (see k_mixed.cu for
// the storage and arithmetic of each field) for a batch of G solves of one grid
// (dot_batch.cuh), and the single-solve Path of the C ABI on top of it.  Host
// side: buffer plan, uploads, and the double <-> (float | two-float) conversions
// of the C ABI's host arrays.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "dot_batch.cuh"

namespace dot {

struct MixedBatch::Buffers {
  MxFields f;        // set 0 of (q, alpha, beta) + the shared fields
  MxFields f2;       // set 1 of (q, alpha, beta) (fused D = 2 path), shared fields as f
  double* socp;      // fused-kernel partial sums of |z - BFq - d|^2, per slot
  float2* phi_op;
  float2* c0;
  float2* c1;
  double* m0;
  double* m1;
  float* omega;
  float* somega;
  float* tab[kMaxD + 1][6];   // C, C^T, C hi, C lo, C^T hi, C^T lo
  float* tpad[4];             // time axis, rows padded to time_ld(g)
  float* lbuf[kMaxD + 1];
  double* partials;
  double* red;
  int* err;
  SlotParam* params;
  float* w1;                  // Poisson scratch, G * poisson_scratch_elems(g) floats each
  float* w2;
};

namespace {

// per-slot partial sums of |z - BFq - d|^2 written by either fused kernel for a batch of G
long long socp_blocks(const Geo& g, int G) { return std::max(fused2d_blocks(g), fused2d_tma_blocks(g, G)); }

void carve(const Geo& g, int G, bool masks, Carver& cv, MixedBatch::Buffers* B) {
  const size_t nn = (size_t)(g.T + 1) * g.P, n0 = (size_t)g.T * g.P, P = (size_t)g.P;
  const size_t Gs = (size_t)G;
  std::memset(B, 0, sizeof(*B));
  B->f.q[0] = cv.take<float>(Gs * n0);
  B->f.al[0] = cv.take<float2>(Gs * n0);
  for (int d = 0; d < g.D; ++d) {
    B->f.q[1 + d] = cv.take<float>(Gs * nn);
    B->f.al[1 + d] = cv.take<float2>(Gs * nn);
  }
  B->f.beta = cv.take<float2>(Gs * g.K * n0);
  B->f2 = B->f;
  if (fused2d_supported(g) || fused3d_supported(g)) {   // q, alpha, beta double-buffered
    B->f2.q[0] = cv.take<float>(Gs * n0);
    B->f2.al[0] = cv.take<float2>(Gs * n0);
    for (int d = 0; d < g.D; ++d) {
      B->f2.q[1 + d] = cv.take<float>(Gs * nn);
      B->f2.al[1 + d] = cv.take<float2>(Gs * nn);
    }
    B->f2.beta = cv.take<float2>(Gs * g.K * n0);
  }
  if (fused2d_supported(g)) {
    B->f.z = nullptr;                       // z never leaves the fused kernel
    B->socp = cv.take<double>(Gs * socp_blocks(g, G));
  } else {
    B->f.z = cv.take<float>(Gs * g.K * n0);
    B->socp = nullptr;
  }
  B->f.phi = cv.take<float2>(Gs * nn);
  B->phi_op = cv.take<float2>(nn);
  B->f.b = cv.take<float>(Gs * nn);
  B->f.blo = cv.take<float>(Gs * nn);
  B->f.phi1 = cv.take<float>(Gs * nn);
  B->f.r = cv.take<float>(Gs * nn);
  B->f.bsum = cv.take<double>(Gs * kBsumStride);
  const size_t ws = poisson_scratch_elems(g);
  B->c0 = cv.take<float2>(Gs * P);
  B->c1 = cv.take<float2>(Gs * P);
  B->m0 = cv.take<double>(Gs * P);
  B->m1 = cv.take<double>(Gs * P);
  B->omega = cv.take<float>((masks ? Gs : 1) * P);
  B->somega = cv.take<float>((masks ? Gs : 1) * P);
  for (int a = 0; a <= g.D; ++a) {
    const size_t M = a == 0 ? (size_t)g.T + 1 : (size_t)g.N[a - 1];
    for (int j = 0; j < 6; ++j) B->tab[a][j] = cv.take<float>(M * M);
    B->lbuf[a] = cv.take<float>(M);
  }
  const size_t ldt = (size_t)time_ld(g);
  for (int j = 0; j < 4; ++j) B->tpad[j] = cv.take<float>((size_t)(g.T + 1) * ldt);
  B->partials = cv.take<double>(Gs * kkt_partials_len_mx(g));
  B->red = cv.take<double>(Gs * R_NSLOTS);
  B->err = cv.take<int>(64);
  B->params = cv.take<SlotParam>(Gs);
  B->w1 = cv.take<float>(Gs * ws);
  B->w2 = cv.take<float>(Gs * ws);
}

// Round to the nearest TF32 value (10 explicit mantissa bits), ties away from zero.
inline float tf32_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

inline float2 split_ff(double v) {
  const float hi = (float)v;
  const float lo = (float)(v - (double)hi);
  return make_float2(hi, lo);
}

cudaError_t up(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}
cudaError_t down(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
}

}  // namespace

MixedBatch::MixedBatch(const Geo& g, int G, bool slot_masks)
    : g_(g), G_(G), slot_masks_(slot_masks), B_(new Buffers()) {
  std::memset(&ps_, 0, sizeof(ps_));
  const SlotParam empty{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(1.f, 0.f), 0.f, 0, 1};
  hp_.assign(G, empty);
  hs_.assign(G, 0.0);
}

MixedBatch::~MixedBatch() {}

size_t MixedBatch::workspace_bytes(const Geo& g, int G, bool slot_masks) {
  Carver cv(nullptr);
  Buffers B;
  carve(g, G, slot_masks, cv, &B);
  return cv.off + 256;
}

bool MixedBatch::batchable(const Geo& g) {
  MxPoisson ps;
  std::memset(&ps, 0, sizeof(ps));
  ps.use_tc = true;
  float dummy = 0.f;
  ps.tpad[0] = &dummy;
  return fused2d_supported(g) && poisson_tc_flow(g, ps);
}

const MxFields& MixedBatch::cur() const { return cur_ == 0 ? B_->f : B_->f2; }
const MxFields& MixedBatch::other() const { return cur_ == 0 ? B_->f2 : B_->f; }

int MixedBatch::init(char* ws, size_t bytes, cudaStream_t s, std::string* err) {
  if (g_.T + 1 > 160) {
    *err = "DOT_MIXED supports T + 1 <= 160 time nodes";
    return DOT_EINVAL;
  }
  const size_t need = workspace_bytes(g_, G_, slot_masks_);
  if (bytes + 256 < need) { *err = "workspace too small"; return DOT_ENOMEM; }
  Carver cv(ws);
  carve(g_, G_, slot_masks_, cv, B_.get());
  ps_.w1 = B_->w1;
  ps_.w2 = B_->w2;
  Buffers& B = *B_;
  fused_ = fused2d_supported(g_);
  tma_ = fused_ && fused2d_tma_supported(g_);
  fused3_ = fused3d_supported(g_);
  if (G_ > 1 && !batchable(g_)) {
    *err = "this grid cannot be batched (needs D = 2 and every axis on the tensor cores)";
    return DOT_EINVAL;
  }
  // shared (not double-buffered) pointers of set 1
  MxFields& f2 = B.f2;
  f2.z = B.f.z;
  f2.phi = B.f.phi;
  f2.b = B.f.b;
  f2.phi1 = B.f.phi1;
  f2.r = B.f.r;
  f2.bsum = B.f.bsum;
  f2.blo = B.f.blo;
  if (!fused_ && !fused3_) {
    for (int d = 0; d <= kMaxD; ++d) { f2.q[d] = B.f.q[d]; f2.al[d] = B.f.al[d]; }
    f2.beta = B.f.beta;
  }
  for (MxFields* f : {&B.f, &B.f2}) {
    f->c0 = B.c0;
    f->c1 = B.c1;
    f->m0 = B.m0;
    f->m1 = B.m1;
    f->omega = slot_masks_ ? B.omega : nullptr;
    f->somega = slot_masks_ ? B.somega : nullptr;
    f->sp = B.params;
  }
  red_ = B.red;
  err_ = B.err;
  dparams_ = B.params;
  cudaError_t e = cudaSuccess;
  // DCT tables: C, C^T and their TF32 splits per axis; the time axis also padded
  hT_.assign((g_.D + 1) * 6 + 4, {});
  const int ldt = time_ld(g_);
  for (int a = 0; a <= g_.D; ++a) {
    std::vector<double> C, l;
    dct_tables_host(g_, a, &C, &l);
    const size_t M = (size_t)(a == 0 ? g_.T + 1 : g_.N[a - 1]);
    std::vector<float>* t = &hT_[a * 6];
    for (int j = 0; j < 6; ++j) t[j].resize(M * M);
    for (size_t k = 0; k < M; ++k)
      for (size_t n = 0; n < M; ++n) {
        const double c = C[k * M + n];
        const float hi = tf32_round_host((float)c);
        const float lo = (float)(c - (double)hi);
        t[0][k * M + n] = (float)c;         // C
        t[1][n * M + k] = (float)c;         // C^T
        t[2][k * M + n] = hi;               // C hi
        t[3][k * M + n] = lo;               // C lo
        t[4][n * M + k] = hi;               // C^T hi
        t[5][n * M + k] = lo;               // C^T lo
      }
    for (int j = 0; j < 6 && e == cudaSuccess; ++j) e = up(B.tab[a][j], t[j].data(), M * M * 4, s);
    std::vector<float> lam(l.begin(), l.end());
    if (e == cudaSuccess) e = up(B.lbuf[a], lam.data(), M * 4, s);
    ps_.C[a] = B.tab[a][0];
    ps_.CT[a] = B.tab[a][1];
    ps_.Chi[a] = B.tab[a][2];
    ps_.Clo[a] = B.tab[a][3];
    ps_.CThi[a] = B.tab[a][4];
    ps_.CTlo[a] = B.tab[a][5];
    ps_.lam[a] = B.lbuf[a];
    if (a == 0) {
      for (int j = 0; j < 4; ++j) {
        std::vector<float>& p = hT_[(g_.D + 1) * 6 + j];
        p.assign(M * ldt, 0.f);
        const std::vector<float>& src = t[2 + j];
        for (size_t k = 0; k < M; ++k)
          for (size_t n = 0; n < M; ++n) p[k * ldt + n] = src[k * M + n];
        if (e == cudaSuccess) e = up(B.tpad[j], p.data(), p.size() * 4, s);
        ps_.tpad[j] = B.tpad[j];
      }
    }
  }
  ps_.err = B.err;
  ps_.use_tc = true;
  if (e == cudaSuccess) e = cudaMemsetAsync(B.err, 0, 64 * sizeof(int), s);
  // zero everything a slot owns (finite scratch for the shared passes) and the params
  const size_t nn = (size_t)(g_.T + 1) * g_.P;
  if (e == cudaSuccess) e = cudaMemsetAsync(ps_.w1, 0, (size_t)G_ * poisson_scratch_elems(g_) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ps_.w2, 0, (size_t)G_ * poisson_scratch_elems(g_) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.f.b, 0, (size_t)G_ * nn * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.f.blo, 0, (size_t)G_ * nn * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.f.phi1, 0, (size_t)G_ * nn * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.f.r, 0, (size_t)G_ * nn * 4, s);
  for (int b = 0; b < G_ && e == cudaSuccess; ++b) e = zero_slot(b, s);
  for (int b = 0; b < G_; ++b) {
    hp_[b] = SlotParam{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(1.f, 0.f), 0.f, 0};
    hs_[b] = 0.0;
  }
  if (e == cudaSuccess) e = upload_params(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { *err = std::string("init: ") + cudaGetErrorString(e); return DOT_ECUDA; }
  return DOT_OK;
}

cudaError_t MixedBatch::zero_slot(int b, cudaStream_t s) {
  const size_t nn = (size_t)(g_.T + 1) * g_.P, n0 = (size_t)g_.T * g_.P;
  Buffers& B = *B_;
  cudaError_t e = cudaMemsetAsync(B.f.phi + b * nn, 0, nn * 8, s);
  const MxFields* sets[2] = {&B.f, &B.f2};
  for (int k = 0; k < (fused_ || fused3_ ? 2 : 1); ++k) {
    const MxFields& f = *sets[k];
    if (e == cudaSuccess) e = cudaMemsetAsync(f.q[0] + b * n0, 0, n0 * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f.al[0] + b * n0, 0, n0 * 8, s);
    for (int d = 0; d < g_.D && e == cudaSuccess; ++d) {
      e = cudaMemsetAsync(f.q[1 + d] + b * nn, 0, nn * 4, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(f.al[1 + d] + b * nn, 0, nn * 8, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(f.beta + b * g_.K * n0, 0, (size_t)g_.K * n0 * 8, s);
  }
  if (e == cudaSuccess && B.f.z) e = cudaMemsetAsync(B.f.z + b * g_.K * n0, 0, (size_t)g_.K * n0 * 4, s);
  if (e == cudaSuccess && B.socp)
    e = cudaMemsetAsync(B.socp + b * socp_blocks(g_, G_), 0, (size_t)socp_blocks(g_, G_) * sizeof(double), s);
  return e;
}

int MixedBatch::load_slot(int b, const std::vector<double>& m0, const std::vector<double>& m1,
                          const std::vector<double>* omega, double sigma, double tau, cudaStream_t s,
                          std::string* err) {
  if (b < 0 || b >= G_) { *err = "slot out of range"; return DOT_EINVAL; }
  if (omega && !slot_masks_ && G_ > 1) { *err = "this batch carries no obstacle weights"; return DOT_EINVAL; }
  Buffers& B = *B_;
  const size_t P = (size_t)g_.P;
  // staging buffers: pageable host memory, copied before cudaMemcpyAsync returns
  std::vector<float2> c0(P), c1(P);
  for (size_t i = 0; i < P; ++i) { c0[i] = split_ff(m0[i]); c1[i] = split_ff(m1[i]); }
  cudaError_t e = up(B.c0 + b * P, c0.data(), P * 8, s);
  if (e == cudaSuccess) e = up(B.c1 + b * P, c1.data(), P * 8, s);
  if (e == cudaSuccess) e = up(B.m0 + b * P, m0.data(), P * 8, s);
  if (e == cudaSuccess) e = up(B.m1 + b * P, m1.data(), P * 8, s);
  const bool keep = slot_masks_ || omega;
  if (keep) {
    std::vector<float> om(P), som(P);
    for (size_t i = 0; i < P; ++i) {
      const double w = omega ? (*omega)[i] : 1.0;
      om[i] = (float)w;
      som[i] = (float)std::sqrt(w / 2.0);
    }
    const size_t off = slot_masks_ ? b * P : 0;
    if (e == cudaSuccess) e = up(B.omega + off, om.data(), P * 4, s);
    if (e == cudaSuccess) e = up(B.somega + off, som.data(), P * 4, s);
  }
  if (!slot_masks_) {
    // a single solve reads omega only when it has an obstacle
    for (MxFields* f : {&B.f, &B.f2}) {
      f->omega = omega ? B.omega : nullptr;
      f->somega = omega ? B.somega : nullptr;
    }
  }
  if (e == cudaSuccess) e = zero_slot(b, s);
  set_sigma(b, sigma, tau, false);
  hp_[b].active = 1;
  r_valid_ = false;
  if (e == cudaSuccess) e = upload_params(s);
  if (e != cudaSuccess) { *err = std::string("load_slot: ") + cudaGetErrorString(e); return DOT_ECUDA; }
  return DOT_OK;
}

void MixedBatch::set_sigma(int b, double sigma, double tau, bool rescale) {
  if (rescale && hs_[b] > 0.0 && sigma != hs_[b]) {
    // compose with a factor not yet applied
    const double pending = (double)hp_[b].rescale.x + (double)hp_[b].rescale.y;
    hp_[b].rescale = split_ff(pending * hs_[b] / sigma);
    hp_[b].assemble = 1;   // c/sigma and the stored multipliers change: the residual too
  } else if (!rescale) {
    hp_[b].rescale = make_float2(1.f, 0.f);
    hp_[b].assemble = 1;
  }
  params_dirty_ = true;
  hp_[b].isg = split_ff(1.0 / sigma);
  hp_[b].sg = split_ff(sigma);
  hp_[b].tau = (float)tau;
  hs_[b] = sigma;
}

bool MixedBatch::rescale_pending() const {
  for (const SlotParam& p : hp_)
    if (p.active && !(p.rescale.x == 1.f && p.rescale.y == 0.f)) return true;
  return false;
}

void MixedBatch::apply_rescale(cudaStream_t s, LaunchCounter lc) {
  launch_rescale_mx(g_, G_, cur(), s, lc);
  r_valid_ = false;
}

void MixedBatch::clear_rescale() {
  for (SlotParam& p : hp_) p.rescale = make_float2(1.f, 0.f);
}

void MixedBatch::set_active(int b, bool on) {
  hp_[b].active = on ? 1 : 0;
  params_dirty_ = true;
}

cudaError_t MixedBatch::upload_params(cudaStream_t s) {
  // pageable source: the runtime stages it before returning, so hp_ may change afterwards
  params_dirty_ = false;
  return up(dparams_, hp_.data(), (size_t)G_ * sizeof(SlotParam), s);
}

void MixedBatch::end_period() {
  // the fused kernels leave every slot's residual in f.r; the last period's first
  // iteration assembled the flagged slots, so the next one reuses them all unless a
  // flag is set again (the D = 2 kernel without TMA, for odd N_y, leaves no residual:
  // flags stay set)
  if (!(tma_ || fused3_)) return;
  for (SlotParam& p : hp_)
    if (p.assemble) {
      p.assemble = 0;
      params_dirty_ = true;
    }
}

void MixedBatch::iterate(cudaStream_t s, LaunchCounter lc) {
  if (fused_) {
    const MxFields& fc = cur();
    const MxFields& fn = other();
    // lines 1-2: the residual is assembled here unless the previous iteration's
    // fused kernel left it in f.r (it cannot after a stopping-measure check, where
    // sigma may change, or after a state or slot change)
    if (r_valid_) launch_solve_residual_mx(g_, G_, fc, ps_, s, lc);
    else launch_assemble_solve_mx(g_, G_, fc, ps_, s, lc);
    // lines 3-6 (the TMA kernel also leaves the next residual in f.r)
    r_valid_ = tma_ && launch_fused2d_tma(g_, G_, fc, fn, B_->socp, B_->err, true, s, lc);
    if (!r_valid_) launch_fused2d(g_, G_, fc, fn, B_->socp, s, lc);
    cur_ ^= 1;
  } else if (fused3_) {
    const MxFields& fc = cur();
    const MxFields& fn = other();
    if (r_valid_) launch_solve_residual_mx(g_, G_, fc, ps_, s, lc);
    else launch_assemble_solve_mx(g_, G_, fc, ps_, s, lc);
    // lines 3-6, and the next iteration's residual in f.r
    launch_fused3d(g_, G_, fc, fn, true, s, lc);
    r_valid_ = true;
    cur_ ^= 1;
  }
}

void MixedBatch::kkt(cudaStream_t s, LaunchCounter lc) {
  // sigma may change after a check: the next iteration assembles the residual of
  // every slot whose assemble flag is set (and reuses f.r for the others)
  r_valid_ = false;
  launch_kkt_mx(g_, G_, cur(), B_->partials, B_->red, fused_ ? B_->socp : nullptr,
                fused_ ? (int)socp_blocks(g_, G_) : 0, s, lc);
}

namespace {

// padded device face field (T+1 planes) <-> natural host layout
cudaError_t face_f_d2h(const Geo& g, int fam, const float* src, double* dst, cudaStream_t s) {
  size_t w, p, h;
  face_copy_shape(g, fam, &w, &p, &h);
  std::vector<float> t(w * h);
  cudaError_t e = cudaMemcpy2DAsync(t.data(), w * 4, src, p * 4, w * 4, h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (size_t i = 0; i < w * h; ++i) dst[i] = t[i];
  return e;
}
cudaError_t face_ff_d2h(const Geo& g, int fam, const float2* src, double* dst, cudaStream_t s) {
  size_t w, p, h;
  face_copy_shape(g, fam, &w, &p, &h);
  std::vector<float2> t(w * h);
  cudaError_t e = cudaMemcpy2DAsync(t.data(), w * 8, src, p * 8, w * 8, h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (size_t i = 0; i < w * h; ++i) dst[i] = (double)t[i].x + (double)t[i].y;
  return e;
}
cudaError_t face_h2d(const Geo& g, int fam, float* qd, float2* ad, const double* q, const double* al,
                     double ascale, cudaStream_t s) {
  size_t w, p, h;
  face_copy_shape(g, fam, &w, &p, &h);
  std::vector<float> tq(w * h);
  std::vector<float2> ta(w * h);
  for (size_t i = 0; i < w * h; ++i) { tq[i] = (float)q[i]; ta[i] = split_ff(al[i] * ascale); }
  cudaError_t e = cudaMemcpy2DAsync(qd, p * 4, tq.data(), w * 4, w * 4, h, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(ad, p * 8, ta.data(), w * 8, w * 8, h, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

int MixedBatch::read_fields(int b, double* rho, double* m, double* phi, cudaStream_t s, std::string* err) {
  cudaError_t e = cudaSuccess;
  const size_t n0 = (size_t)g_.T * g_.P, nn = (size_t)(g_.T + 1) * g_.P;
  const MxFields fc = slot_view(cur(), g_, b);
  const double sig = hs_[b];   // the stored multipliers are alpha / sigma
  if (rho) {
    std::vector<float2> t(n0);
    e = down(t.data(), fc.al[0], n0 * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; i < n0; ++i) rho[i] = sig * ((double)t[i].x + (double)t[i].y);
  }
  if (m && e == cudaSuccess) {
    double* dst = m;
    for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
      e = face_ff_d2h(g_, fam, fc.al[fam], dst, s);
      const long long n = natural_face_count(g_, fam);
      for (long long i = 0; i < n; ++i) dst[i] *= sig;
      dst += n;
    }
  }
  if (phi && e == cudaSuccess) {
    std::vector<float2> t(nn);
    e = down(t.data(), fc.phi, nn * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; i < nn; ++i) phi[i] = (double)t[i].x + (double)t[i].y;
  }
  if (e != cudaSuccess) { *err = std::string("read_fields: ") + cudaGetErrorString(e); return DOT_ECUDA; }
  return DOT_OK;
}

int MixedBatch::read_state(int b, double* q, double* al, double* beta, cudaStream_t s, std::string* err) {
  cudaError_t e = cudaSuccess;
  const size_t n0 = (size_t)g_.T * g_.P;
  const MxFields fc = slot_view(cur(), g_, b);
  if (q) {
    std::vector<float> t(n0);
    e = down(t.data(), fc.q[0], n0 * 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; i < n0; ++i) q[i] = t[i];
    double* dst = q + n0;
    for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
      e = face_f_d2h(g_, fam, fc.q[fam], dst, s);
      dst += natural_face_count(g_, fam);
    }
  }
  const double sig = hs_[b];   // the stored multipliers are alpha / sigma, beta / sigma
  if (al && e == cudaSuccess) {
    std::vector<float2> t(n0);
    e = down(t.data(), fc.al[0], n0 * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; i < n0; ++i) al[i] = sig * ((double)t[i].x + (double)t[i].y);
    double* dst = al + n0;
    for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
      e = face_ff_d2h(g_, fam, fc.al[fam], dst, s);
      const long long n = natural_face_count(g_, fam);
      for (long long i = 0; i < n; ++i) dst[i] *= sig;
      dst += n;
    }
  }
  if (beta && e == cudaSuccess) {
    const size_t nb = (size_t)g_.K * n0;
    std::vector<float2> t(nb);
    e = down(t.data(), fc.beta, nb * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; i < nb; ++i) beta[i] = sig * ((double)t[i].x + (double)t[i].y);
  }
  if (e != cudaSuccess) { *err = std::string("read_state: ") + cudaGetErrorString(e); return DOT_ECUDA; }
  return DOT_OK;
}

int MixedBatch::write_state(int b, const double* q, const double* al, const double* beta, double sigma,
                            double tau, cudaStream_t s, std::string* err) {
  cudaError_t e = zero_slot(b, s);
  r_valid_ = false;
  // both sets were zeroed; write into the current one, the multipliers divided by sigma
  set_sigma(b, sigma, tau, false);
  if (e == cudaSuccess) e = upload_params(s);
  const double is = 1.0 / sigma;
  const MxFields fc = slot_view(cur(), g_, b);
  const size_t n0 = (size_t)g_.T * g_.P;
  std::vector<float> tq(n0);
  std::vector<float2> ta(n0);
  for (size_t i = 0; i < n0; ++i) { tq[i] = (float)q[i]; ta[i] = split_ff(al[i] * is); }
  if (e == cudaSuccess) e = up(fc.q[0], tq.data(), n0 * 4, s);
  if (e == cudaSuccess) e = up(fc.al[0], ta.data(), n0 * 8, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const double* sq = q + n0;
  const double* sa = al + n0;
  for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
    e = face_h2d(g_, fam, fc.q[fam], fc.al[fam], sq, sa, is, s);
    sq += natural_face_count(g_, fam);
    sa += natural_face_count(g_, fam);
  }
  const size_t nb = (size_t)g_.K * n0;
  std::vector<float2> tb(nb);
  for (size_t i = 0; i < nb; ++i) tb[i] = split_ff(beta[i] * is);
  if (e == cudaSuccess) e = up(fc.beta, tb.data(), nb * 8, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { *err = std::string("write_state: ") + cudaGetErrorString(e); return DOT_ECUDA; }
  return DOT_OK;
}

int MixedBatch::poisson_op(const double* b, double* phi, cudaStream_t s, LaunchCounter lc, std::string* err) {
  const size_t nn = (size_t)(g_.T + 1) * g_.P;
  Buffers& B = *B_;
  std::vector<float> tb(nn), tl(nn);
  for (size_t i = 0; i < nn; ++i) {
    const float2 v = split_ff(b[i]);
    tb[i] = v.x;
    tl[i] = v.y;
  }
  r_valid_ = false;   // the solve below uses f.r as scratch
  // slot 0 alone, whatever the batch holds: its parameters are restored afterwards
  std::vector<SlotParam> saved = hp_;
  for (int k = 0; k < G_; ++k) hp_[k].active = k == 0 ? 1 : 0;
  cudaError_t e = upload_params(s);
  if (e == cudaSuccess) e = up(B.f.b, tb.data(), nn * 4, s);
  if (e == cudaSuccess) e = up(B.f.blo, tl.data(), nn * 4, s);
  if (e == cudaSuccess) {
    launch_poisson_refined_mx(g_, 1, B.f, ps_, B.phi_op, false, s, lc);
    e = cudaGetLastError();
  }
  std::vector<float2> t(nn);
  if (e == cudaSuccess) e = down(t.data(), B.phi_op, nn * 8, s);
  hp_ = saved;
  for (SlotParam& p : hp_) p.assemble = 1;   // f.r held the operator's scratch
  if (e == cudaSuccess) e = upload_params(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { *err = std::string("poisson: ") + cudaGetErrorString(e); return DOT_ECUDA; }
  for (size_t i = 0; i < nn; ++i) phi[i] = (double)t[i].x + (double)t[i].y;
  return DOT_OK;
}

namespace {

// The single-solve Path of the C ABI: a batch of one.
class PathMixed : public Path {
 public:
  explicit PathMixed(const Geo& g) : batch_(g, 1, false) {}

  int init(char* ws, size_t bytes, const std::vector<double>& m0, const std::vector<double>& m1,
           const std::vector<double>* omega, cudaStream_t s, std::string* err) override {
    int rc = batch_.init(ws, bytes, s, err);
    if (rc != DOT_OK) return rc;
    m0_ = m0;
    m1_ = m1;
    if (omega) om_ = *omega;
    has_omega_ = omega != nullptr;
    sigma_ = 1.0;
    tau_ = 1.9;
    return batch_.load_slot(0, m0_, m1_, has_omega_ ? &om_ : nullptr, sigma_, tau_, s, err);
  }

  void iterate(double sigma, double tau, cudaStream_t s, LaunchCounter lc) override {
    set_penalty(sigma, tau, s, lc);
    batch_.iterate(s, lc);
  }
  void set_penalty(double sigma, double tau, cudaStream_t s, LaunchCounter lc) override {
    if (sigma != sigma_ || tau != tau_) {
      sigma_ = sigma;
      tau_ = tau;
      batch_.set_sigma(0, sigma, tau, true);
      batch_.upload_params(s);
      if (batch_.rescale_pending()) {
        batch_.apply_rescale(s, lc);
        batch_.clear_rescale();
        batch_.upload_params(s);
      }
    } else if (batch_.params_dirty()) {
      batch_.upload_params(s);   // the assemble flag cleared at the end of the last period
    }
  }
  void end_period() override { batch_.end_period(); }
  bool graphable() const override { return true; }
  int parity() const override { return batch_.parity(); }
  void set_parity(int p) override { batch_.set_parity(p); }
  bool residual_carried() const override { return batch_.residual_valid(); }
  void kkt(cudaStream_t s, LaunchCounter lc) override { batch_.kkt(s, lc); }
  const double* red_out() const override { return batch_.red_out(); }
  const int* error_flag() const override { return batch_.error_flag(); }
  void set_tensor_cores(bool on) override { batch_.set_tensor_cores(on); }
  int read_fields(double* rho, double* m, double* phi, cudaStream_t s, std::string* err) override {
    return batch_.read_fields(0, rho, m, phi, s, err);
  }
  int read_state(double* q, double* al, double* beta, cudaStream_t s, std::string* err) override {
    return batch_.read_state(0, q, al, beta, s, err);
  }
  int write_state(const double* q, const double* al, const double* beta, double sigma, cudaStream_t s,
                  std::string* err) override {
    sigma_ = sigma;
    return batch_.write_state(0, q, al, beta, sigma, tau_, s, err);
  }
  int poisson_op(const double* b, double* phi, cudaStream_t s, LaunchCounter lc, std::string* err) override {
    return batch_.poisson_op(b, phi, s, lc, err);
  }

 private:
  MixedBatch batch_;
  std::vector<double> m0_, m1_, om_;
  bool has_omega_ = false;
  double sigma_ = 1.0, tau_ = 1.9;
};

}  // namespace

void carve_mixed_size(const Geo& g, Carver& cv) { cv.off += MixedBatch::workspace_bytes(g, 1, false); }

std::unique_ptr<Path> make_mixed_path(const Geo& g) { return std::unique_ptr<Path>(new PathMixed(g)); }

}  // namespace dot
