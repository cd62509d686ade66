// path_mixed.cu -- the mixed-precision path of Algorithm 2 (see k_mixed.cu for
// the storage and arithmetic of each field).  Host side: buffer plan, uploads,
// and the double <-> (float | two-float) conversions of the C ABI's host arrays.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "dot_mixed.cuh"
#include "dot_paths.cuh"

namespace dot {
namespace {

struct MxBuffers {
  MxFields f;        // set 0 of (q, alpha, beta) + the shared fields
  MxFields f2;       // set 1 of (q, alpha, beta) (fused D = 2 path), shared fields as f
  double* socp;      // fused-kernel partial sums of |z - BFq - d|^2
  MxPoisson ps;
  float2* phi_op;
  float2* c0;
  float2* c1;
  double* m0;
  double* m1;
  float* omega;
  float* somega;
  float* Cbuf[kMaxD + 1];
  float* CTbuf[kMaxD + 1];
  float* Chi[kMaxD + 1];
  float* Clo[kMaxD + 1];
  float* CThi[kMaxD + 1];
  float* CTlo[kMaxD + 1];
  float* lbuf[kMaxD + 1];
  double* partials;
  double* red;
  int* err;
};

void carve_mx(const Geo& g, Carver& cv, MxBuffers* B) {
  const size_t nn = (size_t)(g.T + 1) * g.P, n0 = (size_t)g.T * g.P, P = (size_t)g.P;
  B->f.q[0] = cv.take<float>(n0);
  B->f.al[0] = cv.take<float2>(n0);
  for (int d = 0; d < g.D; ++d) {
    B->f.q[1 + d] = cv.take<float>(nn);
    B->f.al[1 + d] = cv.take<float2>(nn);
  }
  for (int d = g.D; d < kMaxD; ++d) { B->f.q[1 + d] = nullptr; B->f.al[1 + d] = nullptr; }
  B->f.beta = cv.take<float2>((size_t)g.K * n0);
  B->f2 = B->f;
  const bool fused = fused2d_supported(g);
  if (fused) {
    B->f2.q[0] = cv.take<float>(n0);
    B->f2.al[0] = cv.take<float2>(n0);
    for (int d = 0; d < g.D; ++d) {
      B->f2.q[1 + d] = cv.take<float>(nn);
      B->f2.al[1 + d] = cv.take<float2>(nn);
    }
    B->f2.beta = cv.take<float2>((size_t)g.K * n0);
    B->f.z = nullptr;                       // z never leaves the fused kernel
    B->socp = cv.take<double>((size_t)std::max(fused2d_blocks(g), fused2d_tma_blocks(g)));
  } else {
    B->f.z = cv.take<float>((size_t)g.K * n0);
    B->socp = nullptr;
  }
  B->f.phi = cv.take<float2>(nn);
  B->phi_op = cv.take<float2>(nn);
  B->f.b = cv.take<float>(nn);
  B->f.blo = cv.take<float>(nn);
  B->f.phi1 = cv.take<float>(nn);
  B->f.r = cv.take<float>(nn);
  B->f.bsum = cv.take<double>(kBsumParts + 2);
  B->ps.w1 = cv.take<float>(nn);
  B->ps.w2 = cv.take<float>(nn);
  B->c0 = cv.take<float2>(P);
  B->c1 = cv.take<float2>(P);
  B->m0 = cv.take<double>(P);
  B->m1 = cv.take<double>(P);
  B->omega = cv.take<float>(P);
  B->somega = cv.take<float>(P);
  for (int a = 0; a <= kMaxD; ++a) {
    B->Cbuf[a] = B->CTbuf[a] = B->Chi[a] = B->Clo[a] = B->CThi[a] = B->CTlo[a] = nullptr;
    B->lbuf[a] = nullptr;
  }
  for (int a = 0; a <= g.D; ++a) {
    const size_t M = a == 0 ? (size_t)g.T + 1 : (size_t)g.N[a - 1];
    B->Cbuf[a] = cv.take<float>(M * M);
    B->CTbuf[a] = cv.take<float>(M * M);
    B->Chi[a] = cv.take<float>(M * M);
    B->Clo[a] = cv.take<float>(M * M);
    B->CThi[a] = cv.take<float>(M * M);
    B->CTlo[a] = cv.take<float>(M * M);
    B->lbuf[a] = cv.take<float>(M);
  }
  B->partials = cv.take<double>((size_t)kkt_partials_len_mx(g));
  B->red = cv.take<double>(R_NSLOTS);
  B->err = cv.take<int>(64);
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

class PathMixed : public Path {
 public:
  explicit PathMixed(const Geo& g) : g_(g) {}

  int init(char* ws, size_t bytes, const std::vector<double>& m0, const std::vector<double>& m1,
           const std::vector<double>* omega, cudaStream_t s, std::string* err) override {
    Carver cv(ws);
    carve_mx(g_, cv, &B_);
    if (cv.off > bytes) { *err = "workspace too small"; return DOT_ENOMEM; }
    const size_t P = (size_t)g_.P;
    hc0_.resize(P);
    hc1_.resize(P);
    for (size_t i = 0; i < P; ++i) { hc0_[i] = split_ff(m0[i]); hc1_[i] = split_ff(m1[i]); }
    hm0_ = m0;
    hm1_ = m1;
    cudaError_t e = up(B_.c0, hc0_.data(), P * 8, s);
    if (e == cudaSuccess) e = up(B_.c1, hc1_.data(), P * 8, s);
    if (e == cudaSuccess) e = up(B_.m0, hm0_.data(), P * 8, s);
    if (e == cudaSuccess) e = up(B_.m1, hm1_.data(), P * 8, s);
    if (omega) {
      hom_.resize(P);
      hsom_.resize(P);
      for (size_t i = 0; i < P; ++i) {
        hom_[i] = (float)(*omega)[i];
        hsom_[i] = (float)std::sqrt((*omega)[i] / 2.0);
      }
      if (e == cudaSuccess) e = up(B_.omega, hom_.data(), P * 4, s);
      if (e == cudaSuccess) e = up(B_.somega, hsom_.data(), P * 4, s);
    }
    B_.f.c0 = B_.c0;
    B_.f.c1 = B_.c1;
    B_.f.m0 = B_.m0;
    B_.f.m1 = B_.m1;
    B_.f.omega = omega ? B_.omega : nullptr;
    B_.f.somega = omega ? B_.somega : nullptr;
    hT_.assign((g_.D + 1) * 6, {});
    hl_.resize(g_.D + 1);
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
      float* dst[6] = {B_.Cbuf[a], B_.CTbuf[a], B_.Chi[a], B_.Clo[a], B_.CThi[a], B_.CTlo[a]};
      for (int j = 0; j < 6; ++j)
        if (e == cudaSuccess) e = up(dst[j], t[j].data(), M * M * 4, s);
      hl_[a].assign(l.begin(), l.end());
      if (e == cudaSuccess) e = up(B_.lbuf[a], hl_[a].data(), hl_[a].size() * 4, s);
      B_.ps.C[a] = B_.Cbuf[a];
      B_.ps.CT[a] = B_.CTbuf[a];
      B_.ps.Chi[a] = B_.Chi[a];
      B_.ps.Clo[a] = B_.Clo[a];
      B_.ps.CThi[a] = B_.CThi[a];
      B_.ps.CTlo[a] = B_.CTlo[a];
      B_.ps.lam[a] = B_.lbuf[a];
    }
    B_.ps.err = B_.err;
    B_.ps.use_tc = true;
    fused_ = fused2d_supported(g_);
    tma_ = fused_ && fused2d_tma_supported(g_);
    sync_shared();
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.err, 0, 64 * sizeof(int), s);
    if (g_.T + 1 > 160) {
      *err = "DOT_MIXED supports T + 1 <= 160 time nodes";
      return DOT_EINVAL;
    }
    if (e == cudaSuccess) e = zero_iterate(s);
    if (e != cudaSuccess) { *err = std::string("init: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  void iterate(double sigma, double tau, cudaStream_t s, LaunchCounter lc) override {
    if (fused_) {
      const MxFields& fc = cur();
      const MxFields& fn = other();
      launch_assemble_b_mx(g_, fc, sigma, s, lc);                           // line 1
      launch_poisson_refined_mx(g_, fc, B_.ps, fc.phi, true, s, lc);         // line 2 (+ refinement)
      if (!(tma_ && launch_fused2d_tma(g_, fc, fn, sigma, tau, B_.socp, B_.err, s, lc)))
        launch_fused2d(g_, fc, fn, sigma, tau, B_.socp, s, lc);              // lines 3-6
      cur_ ^= 1;
    } else {
      launch_iterate_mx(g_, B_.f, B_.ps, sigma, tau, s, lc);
    }
  }

  void kkt(cudaStream_t s, LaunchCounter lc) override {
    launch_kkt_mx(g_, cur(), B_.partials, B_.red, fused_ ? B_.socp : nullptr,
                  fused_ ? (int)(tma_ ? fused2d_tma_blocks(g_) : fused2d_blocks(g_)) : 0, s, lc);
  }
  const double* red_out() const override { return B_.red; }
  const int* error_flag() const override { return B_.err; }
  void set_tensor_cores(bool on) override { B_.ps.use_tc = on; }

  int read_fields(double* rho, double* m, double* phi, cudaStream_t s, std::string* err) override {
    cudaError_t e = cudaSuccess;
    const size_t n0 = (size_t)g_.T * g_.P, nn = (size_t)(g_.T + 1) * g_.P;
    if (rho) {
      std::vector<float2> t(n0);
      e = down(t.data(), cur().al[0], n0 * 8, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < n0; ++i) rho[i] = (double)t[i].x + (double)t[i].y;
    }
    if (m && e == cudaSuccess) {
      double* dst = m;
      for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
        e = face_ff_d2h(fam, cur().al[fam], dst, s);
        dst += natural_face_count(g_, fam);
      }
    }
    if (phi && e == cudaSuccess) {
      std::vector<float2> t(nn);
      e = down(t.data(), B_.f.phi, nn * 8, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < nn; ++i) phi[i] = (double)t[i].x + (double)t[i].y;
    }
    if (e != cudaSuccess) { *err = std::string("read_fields: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  int read_state(double* q, double* al, double* beta, cudaStream_t s, std::string* err) override {
    cudaError_t e = cudaSuccess;
    const size_t n0 = (size_t)g_.T * g_.P;
    const MxFields& fc = cur();
    if (q) {
      std::vector<float> t(n0);
      e = down(t.data(), fc.q[0], n0 * 4, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < n0; ++i) q[i] = t[i];
      double* dst = q + n0;
      for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
        e = face_f_d2h(fam, fc.q[fam], dst, s);
        dst += natural_face_count(g_, fam);
      }
    }
    if (al && e == cudaSuccess) {
      std::vector<float2> t(n0);
      e = down(t.data(), fc.al[0], n0 * 8, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < n0; ++i) al[i] = (double)t[i].x + (double)t[i].y;
      double* dst = al + n0;
      for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
        e = face_ff_d2h(fam, fc.al[fam], dst, s);
        dst += natural_face_count(g_, fam);
      }
    }
    if (beta && e == cudaSuccess) {
      const size_t nb = (size_t)g_.K * n0;
      std::vector<float2> t(nb);
      e = down(t.data(), fc.beta, nb * 8, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < nb; ++i) beta[i] = (double)t[i].x + (double)t[i].y;
    }
    if (e != cudaSuccess) { *err = std::string("read_state: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  int write_state(const double* q, const double* al, const double* beta, cudaStream_t s,
                  std::string* err) override {
    cudaError_t e = zero_iterate(s);
    cur_ = 0;
    const size_t n0 = (size_t)g_.T * g_.P;
    std::vector<float> tq(n0);
    std::vector<float2> ta(n0);
    for (size_t i = 0; i < n0; ++i) { tq[i] = (float)q[i]; ta[i] = split_ff(al[i]); }
    if (e == cudaSuccess) e = up(B_.f.q[0], tq.data(), n0 * 4, s);
    if (e == cudaSuccess) e = up(B_.f.al[0], ta.data(), n0 * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const double* sq = q + n0;
    const double* sa = al + n0;
    for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
      e = face_h2d(fam, sq, sa, s);
      sq += natural_face_count(g_, fam);
      sa += natural_face_count(g_, fam);
    }
    const size_t nb = (size_t)g_.K * n0;
    std::vector<float2> tb(nb);
    for (size_t i = 0; i < nb; ++i) tb[i] = split_ff(beta[i]);
    if (e == cudaSuccess) e = up(B_.f.beta, tb.data(), nb * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = std::string("write_state: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  int poisson_op(const double* b, double* phi, cudaStream_t s, LaunchCounter lc, std::string* err) override {
    const size_t nn = (size_t)(g_.T + 1) * g_.P;
    std::vector<float> tb(nn), tl(nn);
    for (size_t i = 0; i < nn; ++i) {
      const float2 v = split_ff(b[i]);
      tb[i] = v.x;
      tl[i] = v.y;
    }
    cudaError_t e = up(B_.f.b, tb.data(), nn * 4, s);
    if (e == cudaSuccess) e = up(B_.f.blo, tl.data(), nn * 4, s);
    if (e == cudaSuccess) {
      launch_poisson_refined_mx(g_, B_.f, B_.ps, B_.phi_op, false, s, lc);
      e = cudaGetLastError();
    }
    std::vector<float2> t(nn);
    if (e == cudaSuccess) e = down(t.data(), B_.phi_op, nn * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = std::string("poisson: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    for (size_t i = 0; i < nn; ++i) phi[i] = (double)t[i].x + (double)t[i].y;
    return DOT_OK;
  }

 private:
  static cudaError_t up(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  }
  static cudaError_t down(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
  }

  cudaError_t zero_iterate(cudaStream_t s) {
    const size_t nn = (size_t)(g_.T + 1) * g_.P, n0 = (size_t)g_.T * g_.P;
    cudaError_t e = cudaMemsetAsync(B_.f.phi, 0, nn * 8, s);
    const MxFields* sets[2] = {&B_.f, &B_.f2};
    for (int k = 0; k < (fused_ ? 2 : 1); ++k) {
      const MxFields& f = *sets[k];
      if (e == cudaSuccess) e = cudaMemsetAsync(f.q[0], 0, n0 * 4, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(f.al[0], 0, n0 * 8, s);
      for (int d = 0; d < g_.D && e == cudaSuccess; ++d) {
        e = cudaMemsetAsync(f.q[1 + d], 0, nn * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(f.al[1 + d], 0, nn * 8, s);
      }
      if (e == cudaSuccess) e = cudaMemsetAsync(f.beta, 0, (size_t)g_.K * n0 * 8, s);
    }
    if (e == cudaSuccess && B_.f.z) e = cudaMemsetAsync(B_.f.z, 0, (size_t)g_.K * n0 * 4, s);
    if (e == cudaSuccess && B_.socp)
      e = cudaMemsetAsync(B_.socp, 0, (size_t)std::max(fused2d_blocks(g_), fused2d_tma_blocks(g_)) * sizeof(double), s);
    return e;
  }

  // the current / other (q, alpha, beta) set
  const MxFields& cur() const { return cur_ == 0 ? B_.f : B_.f2; }
  const MxFields& other() const { return cur_ == 0 ? B_.f2 : B_.f; }

  // copy the shared (non double-buffered) pointers of set 0 into set 1
  void sync_shared() {
    MxFields& b = B_.f2;
    const MxFields& a = B_.f;
    b.z = a.z;
    b.phi = a.phi;
    b.b = a.b;
    b.phi1 = a.phi1;
    b.r = a.r;
    b.bsum = a.bsum;
    b.blo = a.blo;
    b.c0 = a.c0;
    b.c1 = a.c1;
    b.m0 = a.m0;
    b.m1 = a.m1;
    b.omega = a.omega;
    b.somega = a.somega;
    if (!fused_) {
      for (int d = 0; d <= kMaxD; ++d) { b.q[d] = a.q[d]; b.al[d] = a.al[d]; }
      b.beta = a.beta;
    }
  }

  // padded device face field (T+1 planes) -> natural host layout
  cudaError_t face_f_d2h(int fam, const float* src, double* dst, cudaStream_t s) {
    size_t w, p, h;
    face_copy_shape(g_, fam, &w, &p, &h);
    std::vector<float> t(w * h);
    cudaError_t e = cudaMemcpy2DAsync(t.data(), w * 4, src, p * 4, w * 4, h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; i < w * h; ++i) dst[i] = t[i];
    return e;
  }
  cudaError_t face_ff_d2h(int fam, const float2* src, double* dst, cudaStream_t s) {
    size_t w, p, h;
    face_copy_shape(g_, fam, &w, &p, &h);
    std::vector<float2> t(w * h);
    cudaError_t e = cudaMemcpy2DAsync(t.data(), w * 8, src, p * 8, w * 8, h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; i < w * h; ++i) dst[i] = (double)t[i].x + (double)t[i].y;
    return e;
  }
  cudaError_t face_h2d(int fam, const double* q, const double* al, cudaStream_t s) {
    size_t w, p, h;
    face_copy_shape(g_, fam, &w, &p, &h);
    std::vector<float> tq(w * h);
    std::vector<float2> ta(w * h);
    for (size_t i = 0; i < w * h; ++i) { tq[i] = (float)q[i]; ta[i] = split_ff(al[i]); }
    cudaError_t e = cudaMemcpy2DAsync(B_.f.q[fam], p * 4, tq.data(), w * 4, w * 4, h, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(B_.f.al[fam], p * 8, ta.data(), w * 8, w * 8, h, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  }

  Geo g_;
  MxBuffers B_;
  bool fused_ = false;
  bool tma_ = false;
  int cur_ = 0;
  std::vector<float2> hc0_, hc1_;
  std::vector<float> hom_, hsom_;
  std::vector<double> hm0_, hm1_;
  std::vector<std::vector<float>> hT_, hl_;
};

}  // namespace

void carve_mixed_size(const Geo& g, Carver& cv) {
  MxBuffers B;
  carve_mx(g, cv, &B);
}

std::unique_ptr<Path> make_mixed_path(const Geo& g) { return std::unique_ptr<Path>(new PathMixed(g)); }

}  // namespace dot
