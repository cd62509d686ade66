// dot_multilevel.cu -- the multilevel initialisation of Sec. 5 (the experiments'
// "multilevel strategy"): solve the problem on grids coarsened by 2^v in time and
// space, v = levels, ..., 1, each to its own tolerance, and start each finer
// solve from the coarser solution interpolated linearly onto the finer staggered
// grid (dot_prolong_state), ending with the caller's grid.
//
// Interpolation.  Every field is sampled on a tensor grid whose per-axis sample
// positions follow from the staggered discretisation (R2 grid reading):
//   time faces G^s_0 (q_0, alpha_0, every beta component): time (k + 1/2)/T,
//     space cell centres (i + 1/2)/N_d;
//   space faces G^s_d (q_d, alpha_d): time nodes k/T, faces j/N_d (j = 1..N_d-1)
//     along axis d with the no-flux walls j = 0, N_d as zero samples, cell
//     centres along the other axes.
// The interpolant is the tensor product of 1D piecewise-linear interpolation,
// constant beyond the first and last centre.  q approximates A phi (derivatives
// of the potential) and is carried over as is; alpha and beta scale like h_0
// (alpha_0 / h_0 is the density), so they are multiplied by T_coarse / T_fine.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dot.h"
#include "dot_paths.cuh"

using namespace dot;

namespace {

thread_local std::string g_ml_err;

// 1D linear interpolation table from nc coarse samples to nf fine positions.
// value_f[j] = w0 * c[i0] + w1 * c[i1]; an index of -1 stands for a zero sample.
struct Interp1 {
  std::vector<int> i0, i1;
  std::vector<double> w0, w1;
};

// Sample positions of one axis: kind 0 = cell centres (k + 1/2)/n, k < n;
// kind 1 = nodes k/n, k <= n; kind 2 = interior faces j/n, 1 <= j < n, with
// zero samples at 0 and 1.
std::vector<double> positions(int kind, int n) {
  std::vector<double> p;
  if (kind == 0)
    for (int k = 0; k < n; ++k) p.push_back((k + 0.5) / n);
  else if (kind == 1)
    for (int k = 0; k <= n; ++k) p.push_back((double)k / n);
  else
    for (int j = 1; j < n; ++j) p.push_back((double)j / n);
  return p;
}

Interp1 make_interp(int kind, int nc, int nf) {
  std::vector<double> pc = positions(kind, nc), pf = positions(kind, nf);
  Interp1 I;
  const int m = (int)pc.size();
  for (double x : pf) {
    int a = -1, b = -1;
    double wa = 0.0, wb = 0.0;
    // bracketing samples, with the zero walls of kind 2 at 0 and 1
    const double lo = kind == 2 ? 0.0 : pc.front(), hi = kind == 2 ? 1.0 : pc.back();
    if (m == 0) {
      // no interior coarse face: the field is zero
    } else if (x <= pc.front()) {
      if (kind == 2) {
        a = -1;
        b = 0;
        wb = (x - lo) / (pc.front() - lo);
        wa = 1.0 - wb;
      } else {
        a = 0;
        wa = 1.0;
      }
    } else if (x >= pc.back()) {
      if (kind == 2) {
        a = m - 1;
        b = -1;
        wa = (hi - x) / (hi - pc.back());
        wb = 1.0 - wa;
      } else {
        a = m - 1;
        wa = 1.0;
      }
    } else {
      const int k = (int)(std::upper_bound(pc.begin(), pc.end(), x) - pc.begin()) - 1;
      a = k;
      b = k + 1;
      wb = (x - pc[k]) / (pc[k + 1] - pc[k]);
      wa = 1.0 - wb;
    }
    I.i0.push_back(a);
    I.i1.push_back(b);
    I.w0.push_back(wa);
    I.w1.push_back(wb);
  }
  return I;
}

// Interpolate a C-order field of shape dc (rank r) along every axis to shape df.
std::vector<double> interp_field(const double* src, const std::vector<int>& dc, const std::vector<int>& df,
                                 const std::vector<Interp1>& I) {
  std::vector<double> cur(src, src + [&] { size_t n = 1; for (int d : dc) n *= d; return n; }());
  std::vector<int> shape = dc;
  for (size_t ax = 0; ax < dc.size(); ++ax) {
    size_t outer = 1, inner = 1;
    for (size_t a = 0; a < ax; ++a) outer *= shape[a];
    for (size_t a = ax + 1; a < shape.size(); ++a) inner *= shape[a];
    const int nc = shape[ax], nf = df[ax];
    std::vector<double> next(outer * nf * inner);
    const Interp1& T = I[ax];
    for (size_t o = 0; o < outer; ++o)
      for (int j = 0; j < nf; ++j) {
        double* dst = &next[(o * nf + j) * inner];
        const int a = T.i0[j], b = T.i1[j];
        const double wa = T.w0[j], wb = T.w1[j];
        const double* sa = a >= 0 ? &cur[(o * nc + a) * inner] : nullptr;
        const double* sb = b >= 0 ? &cur[(o * nc + b) * inner] : nullptr;
        for (size_t k = 0; k < inner; ++k) dst[k] = (sa ? wa * sa[k] : 0.0) + (sb ? wb * sb[k] : 0.0);
      }
    cur.swap(next);
    shape[ax] = nf;
  }
  return cur;
}

// Shape and per-axis kinds of face family fam (0 = time faces) of grid g.
void family(const dot_grid& g, int fam, std::vector<int>* shape, std::vector<int>* kinds, std::vector<int>* ns) {
  shape->clear();
  kinds->clear();
  ns->clear();
  if (fam == 0) {
    shape->push_back(g.T);
    kinds->push_back(0);
    ns->push_back(g.T);
  } else {
    shape->push_back(g.T + 1);
    kinds->push_back(1);
    ns->push_back(g.T);
  }
  for (int d = 0; d < g.D; ++d) {
    const bool face = fam == d + 1;
    shape->push_back(face ? g.N[d] - 1 : g.N[d]);
    kinds->push_back(face ? 2 : 0);
    ns->push_back(g.N[d]);
  }
}

long long count(const std::vector<int>& s) {
  long long n = 1;
  for (int v : s) n *= v;
  return n;
}

bool grid_cmp_ok(const dot_grid* c, const dot_grid* f) {
  if (c->D != f->D || c->T > f->T) return false;
  for (int d = 0; d < c->D; ++d)
    if (c->N[d] > f->N[d]) return false;
  return true;
}

}  // namespace

extern "C" {

int dot_prolong_state(const dot_grid* gc, const dot_grid* gf, const double* qc, const double* alc,
                      const double* betac, double* qf, double* alf, double* betaf) {
  std::string why;
  if (!grid_valid(gc, &why) || !grid_valid(gf, &why)) {
    g_ml_err = why;
    return DOT_EINVAL;
  }
  if (!grid_cmp_ok(gc, gf)) {
    g_ml_err = "the fine grid must have the coarse grid's D and at least its T and N_d";
    return DOT_EINVAL;
  }
  const double scale = (double)gc->T / (double)gf->T;   // alpha, beta ~ h_0
  long long offc = 0, offf = 0;
  for (int fam = 0; fam <= gc->D; ++fam) {
    std::vector<int> sc, kc, nc, sf, kf, nf;
    family(*gc, fam, &sc, &kc, &nc);
    family(*gf, fam, &sf, &kf, &nf);
    std::vector<Interp1> I;
    for (size_t a = 0; a < sc.size(); ++a) I.push_back(make_interp(kc[a], nc[a], nf[a]));
    if (qc && qf) {
      std::vector<double> v = interp_field(qc + offc, sc, sf, I);
      std::memcpy(qf + offf, v.data(), v.size() * sizeof(double));
    }
    if (alc && alf) {
      std::vector<double> v = interp_field(alc + offc, sc, sf, I);
      for (size_t i = 0; i < v.size(); ++i) alf[offf + i] = scale * v[i];
    }
    if (fam == 0 && betac && betaf) {
      const int K = 4 * gc->D + 2;
      const long long mc = count(sc), mf = count(sf);
      for (int c = 0; c < K; ++c) {
        std::vector<double> v = interp_field(betac + c * mc, sc, sf, I);
        for (long long i = 0; i < mf; ++i) betaf[c * mf + i] = scale * v[i];
      }
    }
    offc += count(sc);
    offf += count(sf);
  }
  return DOT_OK;
}

const char* dot_multilevel_last_error(void) { return g_ml_err.c_str(); }

}  // extern "C"

// Densities (any positive scale) averaged over 2 x ... x 2 blocks of cells, and
// the mask of blocks that contain a masked cell.
void dot::coarsen(const dot_grid& gf, const std::vector<double>& rf, const std::vector<uint8_t>* mf, dot_grid* gc,
                  std::vector<double>* rc, std::vector<uint8_t>* mc) {
  *gc = gf;
  gc->T = gf.T / 2;
  for (int d = 0; d < gf.D; ++d) gc->N[d] = gf.N[d] / 2;
  long long Pc = 1;
  for (int d = 0; d < gf.D; ++d) Pc *= gc->N[d];
  rc->assign(Pc, 0.0);
  if (mf) mc->assign(Pc, 0);
  const int D = gf.D;
  long long Pf = 1;
  for (int d = 0; d < D; ++d) Pf *= gf.N[d];
  for (long long i = 0; i < Pf; ++i) {
    long long rem = i, ci = 0, mul = 1;
    int coord[3] = {0, 0, 0};
    for (int d = D - 1; d >= 0; --d) {
      coord[d] = (int)(rem % gf.N[d]);
      rem /= gf.N[d];
    }
    for (int d = D - 1; d >= 0; --d) {
      ci += (long long)(coord[d] / 2) * mul;
      mul *= gc->N[d];
    }
    (*rc)[ci] += rf[i] / (double)(1 << D);
    if (mf && (*mf)[i]) (*mc)[ci] = 1;
  }
}


bool dot::multilevel_ok(const dot_grid& g, int levels, std::string* why) {
  const int f = 1 << levels;
  if (g.T % f != 0 || g.T / f < 1) {
    *why = "T must be divisible by 2^levels";
    return false;
  }
  for (int d = 0; d < g.D; ++d)
    if (g.N[d] % f != 0 || g.N[d] / f < 2) {
      *why = "every N_d must be divisible by 2^levels with at least 2 coarse cells";
      return false;
    }
  return true;
}

double dot::level_tol(double tol, double coarse_tol, int v) {
  return coarse_tol > 0.0 ? coarse_tol : std::max(tol * std::pow(10.0, -v), 1e-6);
}

extern "C" int dot_solve_multilevel(dot_ctx* ctx, int levels, double tol, double coarse_tol, long maxit,
                                    long* iters) {
  // The context's grid, densities and options define the problem; the coarse
  // levels are solved by temporary contexts of the same precision on the same
  // stream.
  if (!ctx) {
    g_ml_err = "ctx is NULL";
    return DOT_EINVAL;
  }
  DeviceScope dev(context_device(ctx));   // the coarse contexts live on the context's device
  dot_grid g;
  dot_options opt;
  std::vector<double> r0, r1;
  std::vector<uint8_t> mask;
  void* stream = nullptr;
  bool has_mask = false;
  problem_of(ctx, &g, &opt, &stream, &r0, &r1, &mask, &has_mask);
  if (levels < 0 || levels > 8) {
    g_ml_err = "levels must lie in [0, 8]";
    return DOT_EINVAL;
  }
  if (!multilevel_ok(g, levels, &g_ml_err)) return DOT_EINVAL;
  // the pyramid of densities, finest first
  std::vector<dot_grid> grids(levels + 1);
  std::vector<std::vector<double>> R0(levels + 1), R1(levels + 1);
  std::vector<std::vector<uint8_t>> M(levels + 1);
  grids[0] = g;
  R0[0] = r0;
  R1[0] = r1;
  M[0] = mask;
  for (int v = 1; v <= levels; ++v) {
    coarsen(grids[v - 1], R0[v - 1], has_mask ? &M[v - 1] : nullptr, &grids[v], &R0[v], &M[v]);
    dot_grid gtmp;
    std::vector<uint8_t> mtmp;
    coarsen(grids[v - 1], R1[v - 1], nullptr, &gtmp, &R1[v], &mtmp);
  }
  // coarse to fine; the state of the previous level carried in host arrays
  std::vector<double> q, al, beta;
  double sigma = opt.sigma0;
  dot_grid gprev{};
  for (int v = levels; v >= 0; --v) {
    const dot_grid& gv = grids[v];
    dot_ctx* c = ctx;
    if (v > 0) {
      int rc = dot_create(&gv, R0[v].data(), R1[v].data(), has_mask ? M[v].data() : nullptr, &opt, nullptr, 0,
                          stream, &c);
      if (rc != DOT_OK) {
        g_ml_err = std::string("coarse level: ") + dot_last_error(nullptr);
        return rc;
      }
    }
    long long nq = (long long)gv.T;
    long long Pv = 1;
    for (int d = 0; d < gv.D; ++d) Pv *= gv.N[d];
    nq *= Pv;
    for (int d = 0; d < gv.D; ++d) nq += (long long)(gv.T + 1) * (Pv / gv.N[d]) * (gv.N[d] - 1);
    const long long nb = (long long)(4 * gv.D + 2) * gv.T * Pv;
    if (v < levels) {
      std::vector<double> qf(nq), af(nq), bf(nb);
      int rc = dot_prolong_state(&gprev, &gv, q.data(), al.data(), beta.data(), qf.data(), af.data(), bf.data());
      if (rc == DOT_OK) rc = dot_set_state(c, qf.data(), af.data(), bf.data(), sigma, 0);
      if (rc != DOT_OK) {
        if (c != ctx) dot_destroy(c);
        g_ml_err = "warm start failed";
        return rc;
      }
    }
    // per-level tolerance: coarse_tol when given, else the paper's max(tol * 10^-v,
    // 1e-6); the caller's grid tol
    const double tv = v == 0 ? tol : level_tol(tol, coarse_tol, v);
    int rc = dot_solve(c, tv, maxit);
    if (iters) {
      long it = 0;
      if (dot_get_state(c, nullptr, nullptr, nullptr, nullptr, &it) == DOT_OK) iters[v] = it;
    }
    if (rc < 0) {
      if (c != ctx) dot_destroy(c);
      g_ml_err = std::string("level solve: ") + dot_last_error(c == ctx ? ctx : nullptr);
      return rc;
    }
    if (v > 0) {
      q.assign(nq, 0.0);
      al.assign(nq, 0.0);
      beta.assign(nb, 0.0);
      long it = 0;
      rc = dot_get_state(c, q.data(), al.data(), beta.data(), &sigma, &it);
      dot_destroy(c);
      if (rc != DOT_OK) {
        g_ml_err = "reading a coarse state failed";
        return rc;
      }
      gprev = gv;
    } else {
      return rc;
    }
  }
  return DOT_OK;
}
