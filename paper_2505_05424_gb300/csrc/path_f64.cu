// path_f64.cu -- the FP64 reference path: every field and operation in FP64,
// one kernel per line of Algorithm 2, z stored between lines 3 and 4-6.
#include <cmath>
#include <cstring>

#include "dot_paths.cuh"

namespace dot {

void dct_tables_host(const Geo& g, int axis, std::vector<double>* C, std::vector<double>* lam) {
  const double pi = 3.14159265358979323846;
  const int M = axis == 0 ? g.T + 1 : g.N[axis - 1];
  const double h = axis == 0 ? 1.0 / g.T : 1.0 / g.N[axis - 1];
  C->assign((size_t)M * M, 0.0);
  lam->assign(M, 0.0);
  for (int k = 0; k < M; ++k) {
    const double sk = k == 0 ? std::sqrt(1.0 / M) : std::sqrt(2.0 / M);
    for (int n = 0; n < M; ++n) (*C)[(size_t)k * M + n] = sk * std::cos(pi * k * (n + 0.5) / M);
    const double sv = std::sin(pi * k / (2.0 * M));
    (*lam)[k] = 4.0 / (h * h) * sv * sv;
  }
}

void face_copy_shape(const Geo& g, int fam, size_t* width, size_t* pitch, size_t* height) {
  const int d = fam - 1;
  const size_t inner = (size_t)g.sst[d];
  const size_t outer = (size_t)(g.P / (g.N[d] * (long long)inner));
  *width = (size_t)(g.N[d] - 1) * inner;
  *pitch = (size_t)g.N[d] * inner;
  *height = (size_t)(g.T + 1) * outer;
}

long long natural_face_count(const Geo& g, int fam) {
  if (fam == 0) return (long long)g.T * g.P;
  return (long long)(g.T + 1) * (g.P / g.N[fam - 1]) * (g.N[fam - 1] - 1);
}

namespace {

struct F64Buffers {
  F64Fields f;
  double* w2;
  DctTables64 dct;
  double* Cbuf[kMaxD + 1];
  double* lbuf[kMaxD + 1];
  double* m0;
  double* m1;
  double* omega;
  double* somega;
  double* partials;
  double* red;
};

void carve_f64(const Geo& g, Carver& cv, F64Buffers* B) {
  const size_t nn = (size_t)(g.T + 1) * g.P, n0 = (size_t)g.T * g.P;
  B->f.phi = cv.take<double>(nn);
  B->f.b = cv.take<double>(nn);
  B->f.w1 = cv.take<double>(nn);
  B->w2 = cv.take<double>(nn);
  B->f.q[0] = cv.take<double>(n0);
  B->f.al[0] = cv.take<double>(n0);
  for (int d = 0; d < g.D; ++d) {
    B->f.q[1 + d] = cv.take<double>(nn);
    B->f.al[1 + d] = cv.take<double>(nn);
  }
  for (int d = g.D; d < kMaxD; ++d) B->f.q[1 + d] = B->f.al[1 + d] = nullptr;
  B->f.beta = cv.take<double>((size_t)g.K * n0);
  B->f.z = cv.take<double>((size_t)g.K * n0);
  B->m0 = cv.take<double>((size_t)g.P);
  B->m1 = cv.take<double>((size_t)g.P);
  B->omega = cv.take<double>((size_t)g.P);
  B->somega = cv.take<double>((size_t)g.P);
  for (int a = 0; a <= kMaxD; ++a) { B->Cbuf[a] = nullptr; B->lbuf[a] = nullptr; }
  for (int a = 0; a <= g.D; ++a) {
    const size_t M = a == 0 ? (size_t)g.T + 1 : (size_t)g.N[a - 1];
    B->Cbuf[a] = cv.take<double>(M * M);
    B->lbuf[a] = cv.take<double>(M);
  }
  B->partials = cv.take<double>((size_t)kkt_partials_len(g));
  B->red = cv.take<double>(R_NSLOTS);
}

class PathF64 : public Path {
 public:
  explicit PathF64(const Geo& g) : g_(g) {}

  int init(char* ws, size_t bytes, const std::vector<double>& m0, const std::vector<double>& m1,
           const std::vector<double>* omega, cudaStream_t s, std::string* err) override {
    Carver cv(ws);
    carve_f64(g_, cv, &B_);
    if (cv.off > bytes) { *err = "workspace too small"; return DOT_ENOMEM; }
    const size_t P = (size_t)g_.P;
    cudaError_t e = cudaSuccess;
    e = cudaMemcpyAsync(B_.m0, m0.data(), P * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B_.m1, m1.data(), P * sizeof(double), cudaMemcpyHostToDevice, s);
    if (omega) {
      hom_ = *omega;
      hsom_.resize(P);
      for (size_t i = 0; i < P; ++i) hsom_[i] = std::sqrt(hom_[i] / 2.0);
      if (e == cudaSuccess) e = cudaMemcpyAsync(B_.omega, hom_.data(), P * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(B_.somega, hsom_.data(), P * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    B_.f.m0 = B_.m0;
    B_.f.m1 = B_.m1;
    B_.f.omega = omega ? B_.omega : nullptr;
    B_.f.somega = omega ? B_.somega : nullptr;
    hC_.resize(g_.D + 1);
    hl_.resize(g_.D + 1);
    for (int a = 0; a <= g_.D; ++a) {
      dct_tables_host(g_, a, &hC_[a], &hl_[a]);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(B_.Cbuf[a], hC_[a].data(), hC_[a].size() * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(B_.lbuf[a], hl_[a].data(), hl_[a].size() * sizeof(double), cudaMemcpyHostToDevice, s);
      B_.dct.C[a] = B_.Cbuf[a];
      B_.dct.lam[a] = B_.lbuf[a];
    }
    if (e == cudaSuccess) e = zero_iterate(s);
    if (e != cudaSuccess) { *err = std::string("init: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  void iterate(double sigma, double tau, cudaStream_t s, LaunchCounter lc) override {
    launch_assemble_b_f64(g_, B_.f, sigma, s, lc);                         // line 1
    launch_poisson_f64(g_, B_.dct, B_.f.b, B_.f.w1, B_.f.phi, s, lc);     // line 2
    launch_project_f64(g_, B_.f, sigma, s, lc);                            // line 3
    launch_update_q_alpha_f64(g_, B_.f, sigma, tau, s, lc);                // lines 4-5
    launch_update_beta_f64(g_, B_.f, sigma, tau, s, lc);                   // line 6
  }

  void kkt(cudaStream_t s, LaunchCounter lc) override { launch_kkt_f64(g_, B_.f, B_.partials, B_.red, s, lc); }
  const double* red_out() const override { return B_.red; }

  int read_fields(double* rho, double* m, double* phi, cudaStream_t s, std::string* err) override {
    cudaError_t e = cudaSuccess;
    const size_t n0 = (size_t)g_.T * g_.P, nn = (size_t)(g_.T + 1) * g_.P;
    if (rho) e = cudaMemcpyAsync(rho, B_.f.al[0], n0 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (m && e == cudaSuccess) {
      double* dst = m;
      for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
        e = copy_face_d2h(fam, B_.f.al[fam], dst, s);
        dst += natural_face_count(g_, fam);
      }
    }
    if (phi && e == cudaSuccess) e = cudaMemcpyAsync(phi, B_.f.phi, nn * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = std::string("read_fields: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  int read_state(double* q, double* al, double* beta, cudaStream_t s, std::string* err) override {
    cudaError_t e = cudaSuccess;
    if (q) e = read_faces(B_.f.q, q, s);
    if (al && e == cudaSuccess) e = read_faces(B_.f.al, al, s);
    if (beta && e == cudaSuccess)
      e = cudaMemcpyAsync(beta, B_.f.beta, (size_t)g_.K * g_.T * g_.P * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = std::string("read_state: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  int write_state(const double* q, const double* al, const double* beta, double /*sigma*/, cudaStream_t s,
                  std::string* err) override {
    cudaError_t e = zero_iterate(s);
    if (e == cudaSuccess) e = write_faces(q, B_.f.q, s);
    if (e == cudaSuccess) e = write_faces(al, B_.f.al, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(B_.f.beta, beta, (size_t)g_.K * g_.T * g_.P * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = std::string("write_state: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

  int poisson_op(const double* b, double* phi, cudaStream_t s, LaunchCounter lc, std::string* err) override {
    const size_t nn = (size_t)(g_.T + 1) * g_.P;
    // b -> w2, ping-pong w2/w1, result into the right-hand-side buffer (recomputed by
    // every iteration, so the iterate (phi, q, alpha, beta, z) is left untouched).
    cudaError_t e = cudaMemcpyAsync(B_.w2, b, nn * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      launch_poisson_f64(g_, B_.dct, B_.w2, B_.f.w1, B_.f.b, s, lc);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(phi, B_.f.b, nn * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = std::string("poisson: ") + cudaGetErrorString(e); return DOT_ECUDA; }
    return DOT_OK;
  }

 private:
  cudaError_t zero_iterate(cudaStream_t s) {
    const size_t nn = (size_t)(g_.T + 1) * g_.P, n0 = (size_t)g_.T * g_.P;
    cudaError_t e = cudaMemsetAsync(B_.f.phi, 0, nn * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.q[0], 0, n0 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.al[0], 0, n0 * sizeof(double), s);
    for (int d = 0; d < g_.D && e == cudaSuccess; ++d) {
      e = cudaMemsetAsync(B_.f.q[1 + d], 0, nn * sizeof(double), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.al[1 + d], 0, nn * sizeof(double), s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.beta, 0, (size_t)g_.K * n0 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B_.f.z, 0, (size_t)g_.K * n0 * sizeof(double), s);
    return e;
  }

  cudaError_t copy_face_d2h(int fam, const double* src, double* dst, cudaStream_t s) {
    size_t w, p, h;
    face_copy_shape(g_, fam, &w, &p, &h);
    return cudaMemcpy2DAsync(dst, w * sizeof(double), src, p * sizeof(double), w * sizeof(double), h,
                             cudaMemcpyDeviceToHost, s);
  }

  cudaError_t read_faces(double* const* dev, double* host, cudaStream_t s) {
    const size_t n0 = (size_t)g_.T * g_.P;
    cudaError_t e = cudaMemcpyAsync(host, dev[0], n0 * sizeof(double), cudaMemcpyDeviceToHost, s);
    double* dst = host + n0;
    for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
      e = copy_face_d2h(fam, dev[fam], dst, s);
      dst += natural_face_count(g_, fam);
    }
    return e;
  }

  cudaError_t write_faces(const double* host, double* const* dev, cudaStream_t s) {
    const size_t n0 = (size_t)g_.T * g_.P;
    cudaError_t e = cudaMemcpyAsync(dev[0], host, n0 * sizeof(double), cudaMemcpyHostToDevice, s);
    const double* src = host + n0;
    for (int fam = 1; fam <= g_.D && e == cudaSuccess; ++fam) {
      size_t w, p, h;
      face_copy_shape(g_, fam, &w, &p, &h);
      e = cudaMemcpy2DAsync(dev[fam], p * sizeof(double), src, w * sizeof(double), w * sizeof(double), h,
                            cudaMemcpyHostToDevice, s);
      src += natural_face_count(g_, fam);
    }
    return e;
  }

  Geo g_;
  F64Buffers B_;
  std::vector<double> hom_, hsom_;
  std::vector<std::vector<double>> hC_, hl_;
};

}  // namespace

size_t path_workspace_bytes(const Geo& g, dot_precision prec) {
  Carver cv(nullptr);
  if (prec == DOT_FP64) {
    F64Buffers B;
    carve_f64(g, cv, &B);
  } else {
    carve_mixed_size(g, cv);
  }
  return (cv.off + 255) & ~size_t(255);
}

std::unique_ptr<Path> make_path(dot_precision prec, const Geo& g) {
  if (prec == DOT_FP64) return std::unique_ptr<Path>(new PathF64(g));
  return make_mixed_path(g);
}

}  // namespace dot
