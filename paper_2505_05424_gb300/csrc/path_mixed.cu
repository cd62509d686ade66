// path_mixed.cu -- the mixed-precision path of Algorithm 2 (see k_mixed.cu for
// the storage and arithmetic of each field).  Host side: buffer plan, uploads,
// and the double <-> (float | two-float) conversions of the C ABI's host arrays.
#include <cmath>
#include <cstring>

#include "dot_mixed.cuh"
#include "dot_paths.cuh"

namespace dot {
namespace {

struct MxBuffers {
  MxFields f;
  MxPoisson ps;
  float2* phi_op;
  float* m0f;
  float* m1f;
  double* m0;
  double* m1;
  float* omega;
  float* somega;
  float* Cbuf[kMaxD + 1];
  float* lbuf[kMaxD + 1];
  double* partials;
  double* red;
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
  B->f.z = cv.take<float>((size_t)g.K * n0);
  B->f.phi = cv.take<float2>(nn);
  B->phi_op = cv.take<float2>(nn);
  B->f.b = cv.take<float>(nn);
  B->f.phi1 = cv.take<float>(nn);
  B->f.r = cv.take<float>(nn);
  B->ps.w1 = cv.take<float>(nn);
  B->ps.w2 = cv.take<float>(nn);
  B->m0f = cv.take<float>(P);
  B->m1f = cv.take<float>(P);
  B->m0 = cv.take<double>(P);
  B->m1 = cv.take<double>(P);
  B->omega = cv.take<float>(P);
  B->somega = cv.take<float>(P);
  for (int a = 0; a <= kMaxD; ++a) { B->Cbuf[a] = nullptr; B->lbuf[a] = nullptr; }
  for (int a = 0; a <= g.D; ++a) {
    const size_t M = a == 0 ? (size_t)g.T + 1 : (size_t)g.N[a - 1];
    B->Cbuf[a] = cv.take<float>(M * M);
    B->lbuf[a] = cv.take<float>(M);
  }
  B->partials = cv.take<double>((size_t)kkt_partials_len_mx(g));
  B->red = cv.take<double>(R_NSLOTS);
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
    hm0f_.resize(P);
    hm1f_.resize(P);
    for (size_t i = 0; i < P; ++i) { hm0f_[i] = (float)m0[i]; hm1f_[i] = (float)m1[i]; }
    hm0_ = m0;
    hm1_ = m1;
    cudaError_t e = up(B_.m0f, hm0f_.data(), P * 4, s);
    if (e == cudaSuccess) e = up(B_.m1f, hm1f_.data(), P * 4, s);
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
    B_.f.m0f = B_.m0f;
    B_.f.m1f = B_.m1f;
    B_.f.m0 = B_.m0;
    B_.f.m1 = B_.m1;
    B_.f.omega = omega ? B_.omega : nullptr;
    B_.f.somega = omega ? B_.somega : nullptr;
    hC_.resize(g_.D + 1);
    hl_.resize(g_.D + 1);
    for (int a = 0; a <= g_.D; ++a) {
      std::vector<double> C, l;
      dct_tables_host(g_, a, &C, &l);
      hC_[a].assign(C.begin(), C.end());
      hl_[a].assign(l.begin(), l.end());
      if (e == cudaSuccess) e = up(B_.Cbuf[a], hC_[a].data(), hC_[a].size() * 4, s);
      if (e == cudaSuccess) e = up(B_.lbuf[a], hl_[a].data(), hl_[a].size() * 4, s);
      B_.ps.C[a] = B_.Cbuf[a];
      B_.ps.lam[a] = B_.lbuf[a];
    }
    if (e == cudaSuccess) e = zero_iterate(s);
    if (e != cudaSuccess) { *err = std::string("init: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  void iterate(double sigma, double tau, cudaStream_t s, LaunchCounter lc) override {
    launch_iterate_mx(g_, B_.f, B_.ps, sigma, tau, s, lc);
  }

  void kkt(cudaStream_t s, LaunchCounter lc) override { launch_kkt_mx(g_, B_.f, B_.partials, B_.red, s, lc); }
  const double* red_out() const override { return B_.red; }

  int read_fields(double* rho, double* m, double* phi, cudaStream_t s, std::string* err) override {
    cudaError_t e = cudaSuccess;
    const size_t n0 = (size_t)g_.T * g_.P, nn = (size_t)(g_.T + 1) * g_.P;
    if (rho) {
      std::vector<float2> t(n0);
      e = down(t.data(), B_.f.al[0], n0 * 8, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < n0; ++i) rho[i] = (double)t[i].x + (double)t[i].y;
    }
    if (m && e == cudaSuccess) {
      double* dst = m;
      for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
        e = face_ff_d2h(fam, B_.f.al[fam], dst, s);
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
    if (q) {
      std::vector<float> t(n0);
      e = down(t.data(), B_.f.q[0], n0 * 4, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < n0; ++i) q[i] = t[i];
      double* dst = q + n0;
      for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
        e = face_f_d2h(fam, B_.f.q[fam], dst, s);
        dst += natural_face_count(g_, fam);
      }
    }
    if (al && e == cudaSuccess) {
      std::vector<float2> t(n0);
      e = down(t.data(), B_.f.al[0], n0 * 8, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < n0; ++i) al[i] = (double)t[i].x + (double)t[i].y;
      double* dst = al + n0;
      for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
        e = face_ff_d2h(fam, B_.f.al[fam], dst, s);
        dst += natural_face_count(g_, fam);
      }
    }
    if (beta && e == cudaSuccess) {
      const size_t nb = (size_t)g_.K * n0;
      std::vector<float2> t(nb);
      e = down(t.data(), B_.f.beta, nb * 8, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (size_t i = 0; i < nb; ++i) beta[i] = (double)t[i].x + (double)t[i].y;
    }
    if (e != cudaSuccess) { *err = std::string("read_state: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  int write_state(const double* q, const double* al, const double* beta, cudaStream_t s,
                  std::string* err) override {
    cudaError_t e = zero_iterate(s);
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
    std::vector<float> tb(nn);
    for (size_t i = 0; i < nn; ++i) tb[i] = (float)b[i];
    cudaError_t e = up(B_.f.b, tb.data(), nn * 4, s);
    if (e == cudaSuccess) {
      launch_poisson_refined_mx(g_, B_.f, B_.ps, B_.phi_op, s, lc);
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
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.q[0], 0, n0 * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.al[0], 0, n0 * 8, s);
    for (int d = 0; d < g_.D && e == cudaSuccess; ++d) {
      e = cudaMemsetAsync(B_.f.q[1 + d], 0, nn * 4, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.al[1 + d], 0, nn * 8, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.beta, 0, (size_t)g_.K * n0 * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.z, 0, (size_t)g_.K * n0 * 4, s);
    return e;
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
  std::vector<float> hm0f_, hm1f_, hom_, hsom_;
  std::vector<double> hm0_, hm1_;
  std::vector<std::vector<float>> hC_, hl_;
};

}  // namespace

void carve_mixed_size(const Geo& g, Carver& cv) {
  MxBuffers B;
  carve_mx(g, cv, &B);
}

std::unique_ptr<Path> make_mixed_path(const Geo& g) { return std::unique_ptr<Path>(new PathMixed(g)); }

}  // namespace dot
