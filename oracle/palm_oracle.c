/*
 * palm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the inexact proximal ALM (Algorithm 1,
 * explicit steps Algorithm 2, Sec. 4) for the SOCP reformulation (Sec. 3) of the
 * staggered-grid discretised dynamic optimal transport problem (Sec. 2.2, eq. (8)).
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this file.  It shares no code, header, table or helper with the CUDA path.
 *
 * Grid reading (the paper leaves the cell-centred layout implicit): D spatial
 * axes with N_d cells each; the potential lives on the N_d cell centres, so
 * h_d = 1/N_d and each spatial axis has N_d - 1 interior faces.  Time has T
 * intervals, T+1 nodes, h_0 = 1/T.  Every field is a dense C-order array:
 *   nodes G^c      : [T+1][N_1]...[N_D]
 *   faces G^s_0    : [T  ][N_1]...[N_D]                (one cone per entry)
 *   faces G^s_d    : [T+1][N_1]..[N_d - 1]..[N_D]      (d = 1..D)
 * q and alpha are the concatenation (G^s_0; G^s_1; ...; G^s_D); beta and z are
 * K = 4D+2 blocks of |G^s_0| entries each (block-major).
 *
 * Every function cites the passage it follows.  Nothing here is blocked, fused
 * or reordered beyond what the cited definition states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int D;
  int T;
  int N[3];
} og_grid;

typedef struct {
  int nd;       /* D + 1 axes, axis 0 = time */
  int n[4];     /* extent per axis */
  long st[4];   /* C-order strides */
  long size;
} og_shape;

/* fam = -1: node grid G^c; fam = 0..D: staggered grid G^s_fam (Sec. 2.2). */
static og_shape og_shape_of(const og_grid *g, int fam) {
  og_shape s;
  s.nd = g->D + 1;
  s.n[0] = (fam == 0) ? g->T : g->T + 1;
  for (int d = 1; d <= g->D; ++d) s.n[d] = g->N[d - 1] - (fam == d ? 1 : 0);
  long st = 1;
  for (int a = s.nd - 1; a >= 0; --a) {
    s.st[a] = st;
    st *= s.n[a];
  }
  s.size = st;
  return s;
}

static void og_unravel(const og_shape *s, long lin, int idx[4]) {
  for (int a = 0; a < s->nd; ++a) {
    idx[a] = (int)(lin / s->st[a]);
    lin -= (long)idx[a] * s->st[a];
  }
}

static long og_ravel(const og_shape *s, const int idx[4]) {
  long lin = 0;
  for (int a = 0; a < s->nd; ++a) lin += (long)idx[a] * s->st[a];
  return lin;
}

static double og_h(const og_grid *g, int axis) {
  return axis == 0 ? 1.0 / g->T : 1.0 / g->N[axis - 1];
}

/* ---- sizes ------------------------------------------------------------ */

long og_num_nodes(const og_grid *g) { return og_shape_of(g, -1).size; }
long og_num_cones(const og_grid *g) { return og_shape_of(g, 0).size; }
long og_num_faces(const og_grid *g, int fam) { return og_shape_of(g, fam).size; }
long og_num_q(const og_grid *g) {
  long n = 0;
  for (int f = 0; f <= g->D; ++f) n += og_shape_of(g, f).size;
  return n;
}
static long og_q_offset(const og_grid *g, int fam) {
  long n = 0;
  for (int f = 0; f < fam; ++f) n += og_shape_of(g, f).size;
  return n;
}
int og_cone_dim(const og_grid *g) { return 4 * g->D + 2; }

/* ---- discrete gradient A and its adjoint (eq. (Amap), Sec. 2.2) -------- */

/* (A_d phi)_i = (phi_{i+e_d/2} - phi_{i-e_d/2}) / h_d for every i in G^s_d. */
void og_apply_A(const og_grid *g, const double *phi, double *q) {
  og_shape sn = og_shape_of(g, -1);
  for (int f = 0; f <= g->D; ++f) {
    og_shape sf = og_shape_of(g, f);
    double *qf = q + og_q_offset(g, f);
    double h = og_h(g, f);
    for (long lin = 0; lin < sf.size; ++lin) {
      int idx[4];
      og_unravel(&sf, lin, idx);
      long lo = og_ravel(&sn, idx);   /* node below the face along axis f */
      idx[f] += 1;
      long hi = og_ravel(&sn, idx);   /* node above the face */
      qf[lin] = (phi[hi] - phi[lo]) / h;
    }
  }
}

/* A^*: the transpose of og_apply_A, scattered face by face. */
void og_apply_At(const og_grid *g, const double *q, double *out) {
  og_shape sn = og_shape_of(g, -1);
  memset(out, 0, sizeof(double) * sn.size);
  for (int f = 0; f <= g->D; ++f) {
    og_shape sf = og_shape_of(g, f);
    const double *qf = q + og_q_offset(g, f);
    double h = og_h(g, f);
    for (long lin = 0; lin < sf.size; ++lin) {
      int idx[4];
      og_unravel(&sf, lin, idx);
      long lo = og_ravel(&sn, idx);
      idx[f] += 1;
      long hi = og_ravel(&sn, idx);
      out[hi] += qf[lin] / h;
      out[lo] -= qf[lin] / h;
    }
  }
}

/* ---- averaging operators L_T, L_X^d and adjoints (eq. (ltlx)) ---------- */

/* fam 0: (L_T y)_i = (y_{i-e0/2} + y_{i+e0/2})/2; fam d: (L_X^d y)_i likewise along d. */
void og_apply_L(const og_grid *g, int fam, const double *y, double *out) {
  og_shape sn = og_shape_of(g, -1), sf = og_shape_of(g, fam);
  for (long lin = 0; lin < sf.size; ++lin) {
    int idx[4];
    og_unravel(&sf, lin, idx);
    long lo = og_ravel(&sn, idx);
    idx[fam] += 1;
    long hi = og_ravel(&sn, idx);
    out[lin] = 0.5 * (y[lo] + y[hi]);
  }
}

/* Adjoint of og_apply_L: face field of family fam -> node field (overwrites out). */
void og_apply_Lt(const og_grid *g, int fam, const double *v, double *out) {
  og_shape sn = og_shape_of(g, -1), sf = og_shape_of(g, fam);
  memset(out, 0, sizeof(double) * sn.size);
  for (long lin = 0; lin < sf.size; ++lin) {
    int idx[4];
    og_unravel(&sf, lin, idx);
    long lo = og_ravel(&sn, idx);
    idx[fam] += 1;
    long hi = og_ravel(&sn, idx);
    out[lo] += 0.5 * v[lin];
    out[hi] += 0.5 * v[lin];
  }
}

/* ---- decoupling operator F (eq. (operatorF), (fdetails)) --------------- */

/* Position of F^d_v's source face for cone (t, xbar), or -1 when the paper's
 * case analysis sets the entry to 0.  v = 1..4:
 *   v=1: q_d at (t,   x_d - 1/2) if x_d >= 1      v=2: (t,   x_d + 1/2) if x_d <= n_d - 1
 *   v=3: q_d at (t+1, x_d - 1/2) if x_d >= 1      v=4: (t+1, x_d + 1/2) if x_d <= n_d - 1
 * With N_d cell centres, n_d = N_d - 1 and face j sits between nodes j and j+1. */
static long og_F_src(const og_grid *g, int d, int v, const int cone[4]) {
  og_shape sd = og_shape_of(g, d);
  int idx[4];
  for (int a = 0; a < 4; ++a) idx[a] = cone[a];
  int xd = cone[d];
  int tt = (v <= 2) ? cone[0] : cone[0] + 1;
  int left = (v == 1 || v == 3);
  if (left) {
    if (xd < 1) return -1;
    idx[d] = xd - 1;
  } else {
    if (xd > g->N[d - 1] - 2) return -1;
    idx[d] = xd;
  }
  idx[0] = tt;
  return og_ravel(&sd, idx);
}

/* out has 4D+1 blocks of |G^s_0|: block 0 = F_0 q_0 = q_0, block 1+4(d-1)+(v-1) = F^d_v q_d. */
void og_apply_F(const og_grid *g, const double *q, double *out) {
  og_shape s0 = og_shape_of(g, 0);
  long n0 = s0.size;
  for (long c = 0; c < n0; ++c) {
    int cone[4];
    og_unravel(&s0, c, cone);
    out[c] = q[c];
    for (int d = 1; d <= g->D; ++d) {
      const double *qd = q + og_q_offset(g, d);
      for (int v = 1; v <= 4; ++v) {
        long src = og_F_src(g, d, v, cone);
        out[(long)(1 + 4 * (d - 1) + (v - 1)) * n0 + c] = (src >= 0) ? qd[src] : 0.0;
      }
    }
  }
}

/* F^*: transpose of og_apply_F (scatter). */
void og_apply_Ft(const og_grid *g, const double *u, double *q) {
  og_shape s0 = og_shape_of(g, 0);
  long n0 = s0.size;
  memset(q, 0, sizeof(double) * og_num_q(g));
  for (long c = 0; c < n0; ++c) {
    int cone[4];
    og_unravel(&s0, c, cone);
    q[c] += u[c];
    for (int d = 1; d <= g->D; ++d) {
      double *qd = q + og_q_offset(g, d);
      for (int v = 1; v <= 4; ++v) {
        long src = og_F_src(g, d, v, cone);
        if (src >= 0) qd[src] += u[(long)(1 + 4 * (d - 1) + (v - 1)) * n0 + c];
      }
    }
  }
}

/* ---- B, d (eq. (socobservation), (bdd)) with the weighted variant ------- */

/* B x = (-x_0; s x_1; ...; s x_{4D}; x_0) per cone with s = sqrt(omega/2); for
 * omega = 1 this is the paper's sqrt(2)/2.  The weighted constraint
 * x_0 + (omega/8) sum x_v^2 <= 0 of P_omega (Sec. 5.4) is (1+x_0)^2 +
 * (omega/2) sum x_v^2 <= (1-x_0)^2, hence s = sqrt(omega/2). */
void og_apply_B(const og_grid *g, const double *omega, const double *x, double *out) {
  long n0 = og_num_cones(g);
  int K = og_cone_dim(g);
  for (long c = 0; c < n0; ++c) {
    double s = sqrt(omega[c] / 2.0);
    out[c] = -x[c];
    for (int j = 1; j <= 4 * g->D; ++j) out[(long)j * n0 + c] = s * x[(long)j * n0 + c];
    out[(long)(K - 1) * n0 + c] = x[c];
  }
}

/* B^*: (u_{K-1} - u_0; s u_1; ...; s u_{4D}). */
void og_apply_Bt(const og_grid *g, const double *omega, const double *u, double *x) {
  long n0 = og_num_cones(g);
  int K = og_cone_dim(g);
  for (long c = 0; c < n0; ++c) {
    double s = sqrt(omega[c] / 2.0);
    x[c] = u[(long)(K - 1) * n0 + c] - u[c];
    for (int j = 1; j <= 4 * g->D; ++j) x[(long)j * n0 + c] = s * u[(long)j * n0 + c];
  }
}

/* d = (1; 0; ...; 0; 1) per cone. */
void og_fill_d(const og_grid *g, double *dvec) {
  long n0 = og_num_cones(g);
  int K = og_cone_dim(g);
  memset(dvec, 0, sizeof(double) * (size_t)K * n0);
  for (long c = 0; c < n0; ++c) {
    dvec[c] = 1.0;
    dvec[(long)(K - 1) * n0 + c] = 1.0;
  }
}

/* ---- projection onto K_soc (eq. (app-proj), Sec. 2) -------------------- */

/* y, z: n entries each, y[0] is the cone axis.  Case order: y if ||ybar|| <= y0;
 * 0 if ||ybar|| <= -y0; otherwise the boundary formula. */
void og_proj_soc(int n, const double *y, double *z) {
  double nb = 0.0;
  for (int j = 1; j < n; ++j) nb += y[j] * y[j];
  nb = sqrt(nb);
  if (nb <= y[0]) {
    for (int j = 0; j < n; ++j) z[j] = y[j];
  } else if (nb <= -y[0]) {
    for (int j = 0; j < n; ++j) z[j] = 0.0;
  } else {
    double a = 0.5 * (y[0] + nb);
    z[0] = a;
    for (int j = 1; j < n; ++j) z[j] = a * y[j] / nb;
  }
}

/* Pi_Q on block-major K x n0 arrays: the projection cone by cone. */
void og_proj_Q(const og_grid *g, const double *Y, double *Z) {
  long n0 = og_num_cones(g);
  int K = og_cone_dim(g);
  double y[14], z[14];
  for (long c = 0; c < n0; ++c) {
    for (int j = 0; j < K; ++j) y[j] = Y[(long)j * n0 + c];
    og_proj_soc(K, y, z);
    for (int j = 0; j < K; ++j) Z[(long)j * n0 + c] = z[j];
  }
}

/* ---- Poisson solve A^*A phi = b on rge(A^*) by DCT (Sec. 4, "Note that the
 * operator A^*A is the standard discrete Laplacian ... DCT") -------------- */

/* Orthonormal DCT-II matrix of order M: C[k][n] = s_k cos(pi k (n + 1/2) / M),
 * s_0 = sqrt(1/M), s_k = sqrt(2/M).  Written from the definition. */
void og_dct_matrix(int M, double *C) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < M; ++k) {
    double s = (k == 0) ? sqrt(1.0 / M) : sqrt(2.0 / M);
    for (int n = 0; n < M; ++n) C[(long)k * M + n] = s * cos(pi * k * (n + 0.5) / M);
  }
}

/* Apply the M x M matrix C (or its transpose) along one axis of a node field. */
static void og_apply_axis(const og_shape *s, int axis, const double *C, int transpose,
                          const double *in, double *out) {
  int M = s->n[axis];
  long st = s->st[axis];
  long lines = s->size / M;
  /* lines are independent; OpenMP over this outermost loop only */
#pragma omp parallel for schedule(static)
  for (long l = 0; l < lines; ++l) {
    double buf[4096];
    /* base index of line l: enumerate all multi-indices with idx[axis] = 0 */
    long rem = l, base = 0;
    for (int a = s->nd - 1; a >= 0; --a) {
      if (a == axis) continue;
      int ia = (int)(rem % s->n[a]);
      rem /= s->n[a];
      base += (long)ia * s->st[a];
    }
    for (int k = 0; k < M; ++k) {
      double acc = 0.0;
      for (int m = 0; m < M; ++m) {
        double cm = transpose ? C[(long)m * M + k] : C[(long)k * M + m];
        acc += cm * in[base + (long)m * st];
      }
      buf[k] = acc;
    }
    for (int k = 0; k < M; ++k) out[base + (long)k * st] = buf[k];
  }
}

/* DCT-II along one axis of a node field (used by the tests to pin the matrix). */
void og_dct_axis(const og_grid *g, int axis, int inverse, const double *in, double *out) {
  og_shape sn = og_shape_of(g, -1);
  int M = sn.n[axis];
  double *C = (double *)malloc(sizeof(double) * M * M);
  og_dct_matrix(M, C);
  og_apply_axis(&sn, axis, C, inverse, in, out);
  free(C);
}

/* Eigenvalue of A^*A for frequency multi-index k: sum_d (4/h_d^2) sin^2(pi k_d / (2 M_d)),
 * M_d = number of nodes on axis d (path-graph Laplacian with Neumann ends). */
static double og_lambda(const og_grid *g, const int k[4]) {
  const double pi = 3.14159265358979323846;
  og_shape sn = og_shape_of(g, -1);
  double lam = 0.0;
  for (int a = 0; a < sn.nd; ++a) {
    double h = og_h(g, a);
    double sv = sin(pi * k[a] / (2.0 * sn.n[a]));
    lam += 4.0 / (h * h) * sv * sv;
  }
  return lam;
}

/* phi = (A^*A)^dagger b: the unique solution in rge(A^*) (mean zero, eq. (32)). */
void og_poisson(const og_grid *g, const double *b, double *phi) {
  og_shape sn = og_shape_of(g, -1);
  double *w0 = (double *)malloc(sizeof(double) * sn.size);
  double *w1 = (double *)malloc(sizeof(double) * sn.size);
  memcpy(w0, b, sizeof(double) * sn.size);
  for (int a = 0; a < sn.nd; ++a) {
    og_dct_axis(g, a, 0, w0, w1);
    memcpy(w0, w1, sizeof(double) * sn.size);
  }
  for (long lin = 0; lin < sn.size; ++lin) {
    int k[4];
    og_unravel(&sn, lin, k);
    if (lin == 0)
      w0[lin] = 0.0; /* zero mode: ker A = constants (eq. (kerA)), phi in rge(A^*) */
    else
      w0[lin] /= og_lambda(g, k);
  }
  for (int a = 0; a < sn.nd; ++a) {
    og_dct_axis(g, a, 1, w0, w1);
    memcpy(w0, w1, sizeof(double) * sn.size);
  }
  memcpy(phi, w0, sizeof(double) * sn.size);
  free(w0);
  free(w1);
}

/* ---- problem data c (eq. (defc)) ---------------------------------------- */

/* c of eq. (defc): rho0 on the i_0 = 0 slice, -rho1 on i_0 = n_0, 0 elsewhere.
 * m0, m1 are cell masses (each summing to 1).  The data enter as cell-average
 * densities, mass / |X_i| with |X_i| = h_1 ... h_D: the initial data are scaled
 * (Sec. 5.3) so that the densities are O(1), the scale on which the uniform lower
 * bounds delta of Sec. 5.4's examples are stated.  The scaling multiplies the
 * objective and the multipliers by 1/|X_i| and leaves phi and q unchanged; without
 * it the volume-weighted L2 norms of A^*alpha + c and of alpha are O(|X_i|) and
 * eta_dot is meaningless on fine grids. */
void og_fill_c(const og_grid *g, const double *m0, const double *m1, double *c) {
  og_shape sn = og_shape_of(g, -1);
  long P = sn.st[0];
  double inv_cell = 1.0;
  for (int d = 1; d <= g->D; ++d) inv_cell *= (double)g->N[d - 1];   /* 1 / (h_1 ... h_D) */
  memset(c, 0, sizeof(double) * sn.size);
  for (long p = 0; p < P; ++p) {
    c[p] = m0[p] * inv_cell;
    c[(long)g->T * P + p] = -m1[p] * inv_cell;
  }
}

/* ---- one iteration of Algorithm 2 ---------------------------------------- */

typedef struct {
  double tau;
  double sigma;
} og_params;

static double *og_alloc(long n) { return (double *)calloc((size_t)n, sizeof(double)); }

/* The six lines of Algorithm 2, in order, on full vectors.
 * (I + F^*B^*BF) is diagonal (Proposition 3.2), so its diagonal is obtained by
 * applying F^*B^*BF to the all-ones vector. */
void og_iterate(const og_grid *g, const og_params *p, const double *c, const double *omega,
                double *phi, double *z, double *q, double *alpha, double *beta) {
  long nn = og_num_nodes(g), nq = og_num_q(g), n0 = og_num_cones(g);
  int K = og_cone_dim(g);
  long nz = (long)K * n0, nf = (long)(K - 1) * n0;
  double sigma = p->sigma, tau = p->tau;
  double *wq = og_alloc(nq), *b = og_alloc(nn), *Fq = og_alloc(nf), *BFq = og_alloc(nz);
  double *dv = og_alloc(nz), *y = og_alloc(nz), *u = og_alloc(nz), *Bu = og_alloc(nf);
  double *FBu = og_alloc(nq), *Aphi = og_alloc(nq), *ones = og_alloc(nq), *diag = og_alloc(nq);
  og_fill_d(g, dv);

  /* line 1: b = A^*(q - alpha/sigma) - c/sigma */
  for (long i = 0; i < nq; ++i) wq[i] = q[i] - alpha[i] / sigma;
  og_apply_At(g, wq, b);
  for (long i = 0; i < nn; ++i) b[i] -= c[i] / sigma;

  /* line 2: solve A^*A phi = b (DCT) */
  og_poisson(g, b, phi);

  /* line 3: z = Pi_Q(B F q + d - beta/sigma) */
  og_apply_F(g, q, Fq);
  og_apply_B(g, omega, Fq, BFq);
  for (long i = 0; i < nz; ++i) y[i] = BFq[i] + dv[i] - beta[i] / sigma;
  og_proj_Q(g, y, z);

  /* line 4: q = (I + F^*B^*BF)^{-1} (A phi + alpha/sigma + F^*B^*(z - d + beta/sigma)) */
  for (long i = 0; i < nq; ++i) ones[i] = 1.0;
  og_apply_F(g, ones, Fq);
  og_apply_B(g, omega, Fq, BFq);
  og_apply_Bt(g, omega, BFq, Bu);
  og_apply_Ft(g, Bu, diag);
  for (long i = 0; i < nz; ++i) u[i] = z[i] - dv[i] + beta[i] / sigma;
  og_apply_Bt(g, omega, u, Bu);
  og_apply_Ft(g, Bu, FBu);
  og_apply_A(g, phi, Aphi);
  for (long i = 0; i < nq; ++i) q[i] = (Aphi[i] + alpha[i] / sigma + FBu[i]) / (1.0 + diag[i]);

  /* line 5: alpha += tau sigma (A phi - q) */
  for (long i = 0; i < nq; ++i) alpha[i] += tau * sigma * (Aphi[i] - q[i]);

  /* line 6: beta += tau sigma (z - B F q - d) */
  og_apply_F(g, q, Fq);
  og_apply_B(g, omega, Fq, BFq);
  for (long i = 0; i < nz; ++i) beta[i] += tau * sigma * (z[i] - BFq[i] - dv[i]);

  free(wq); free(b); free(Fq); free(BFq); free(dv); free(y); free(u); free(Bu);
  free(FBu); free(Aphi); free(ones); free(diag);
}

/* ---- stopping measures (Sec. 5.3) ---------------------------------------- */

/* Discrete L2 norm: sqrt(h_0 h_1 ... h_D * sum v_i^2), every grid point carrying
 * the volume of one space-time cell. */
static double og_l2(const og_grid *g, const double *v, long n) {
  double vol = og_h(g, 0);
  for (int d = 1; d <= g->D; ++d) vol *= og_h(g, d);
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += v[i] * v[i];
  return sqrt(vol * s);
}

enum {
  OG_ETA_DOT = 0, OG_ETA_P, OG_ETA_D, OG_ETA_C, OG_ETA_PSOC, OG_ETA_DSOC,
  OG_PRIMAL_OBJ, OG_DUAL_OBJ, OG_GAP, OG_NUM_KKT
};

/* eta_P, eta_D, eta_C (KKT system (12) of problem (8)), eta_P^soc, eta_D^soc
 * (KKT system (29)), the primal objective <c, phi>, the dual objective (11) and
 * the relative gap.  Weighted problems use f = q_0 + 1/2 omega o L_T L_X^*(|q|^2)
 * and g_d = (L_X^d L_T^*(omega o alpha_0)) o q_d, the same derivation as (12)
 * with the constraint of P_omega. */
void og_kkt(const og_grid *g, const double *c, const double *omega, const double *phi,
            const double *z, const double *q, const double *alpha, const double *beta,
            double *out) {
  long nn = og_num_nodes(g), nq = og_num_q(g), n0 = og_num_cones(g);
  int K = og_cone_dim(g), D = g->D;
  long nz = (long)K * n0, nf = (long)(K - 1) * n0;
  double *Aphi = og_alloc(nq), *r = og_alloc(nq > nz ? nq : nz), *Atal = og_alloc(nn);
  double *tmpn = og_alloc(nn), *acc = og_alloc(nn), *f = og_alloc(n0), *rc = og_alloc(n0);
  double *Fq = og_alloc(nf), *BFq = og_alloc(nz), *dv = og_alloc(nz), *Bb = og_alloc(nf);
  double *FBb = og_alloc(nq), *wa0 = og_alloc(n0);

  /* eta_P */
  og_apply_A(g, phi, Aphi);
  for (long i = 0; i < nq; ++i) r[i] = Aphi[i] - q[i];
  double etaP = og_l2(g, r, nq) / (1.0 + og_l2(g, Aphi, nq) + og_l2(g, q, nq));

  /* eta_D */
  og_apply_At(g, alpha, Atal);
  for (long i = 0; i < nn; ++i) Atal[i] += c[i];
  double etaD = og_l2(g, Atal, nn) / (1.0 + og_l2(g, c, nn));

  /* eta_C, first part: f(q) = q_0 + 1/2 omega o L_T L_X^*(|q_1|^2; ...; |q_D|^2) */
  memset(acc, 0, sizeof(double) * nn);
  for (int d = 1; d <= D; ++d) {
    long off = og_q_offset(g, d), nd = og_num_faces(g, d);
    double *sq = og_alloc(nd);
    for (long i = 0; i < nd; ++i) sq[i] = q[off + i] * q[off + i];
    og_apply_Lt(g, d, sq, tmpn);
    for (long i = 0; i < nn; ++i) acc[i] += tmpn[i];
    free(sq);
  }
  og_apply_L(g, 0, acc, f);
  for (long i = 0; i < n0; ++i) f[i] = q[i] + 0.5 * omega[i] * f[i];
  for (long i = 0; i < n0; ++i) {
    double m = f[i] + alpha[i];
    rc[i] = alpha[i] - (m > 0.0 ? m : 0.0);
  }
  double etaC1 = og_l2(g, rc, n0) / (1.0 + og_l2(g, alpha, n0) + og_l2(g, f, n0));

  /* eta_C, second part: g_d = (L_X^d L_T^*(omega o alpha_0)) o q_d; dual objective (11) */
  for (long i = 0; i < n0; ++i) wa0[i] = omega[i] * alpha[i];
  og_apply_Lt(g, 0, wa0, tmpn);
  long nbar = nq - n0;
  double *gv = og_alloc(nbar), *rb = og_alloc(nbar);
  double dual = 0.0;
  for (int d = 1; d <= D; ++d) {
    long off = og_q_offset(g, d), nd = og_num_faces(g, d);
    double *den = og_alloc(nd);
    og_apply_L(g, d, tmpn, den);
    for (long i = 0; i < nd; ++i) {
      gv[off - n0 + i] = den[i] * q[off + i];
      rb[off - n0 + i] = alpha[off + i] - gv[off - n0 + i];
      if (den[i] > 0.0) dual -= 0.5 * alpha[off + i] * alpha[off + i] / den[i];
    }
    free(den);
  }
  double etaC2 = og_l2(g, rb, nbar) / (1.0 + og_l2(g, alpha + n0, nbar) + og_l2(g, gv, nbar));
  double etaC = etaC1 > etaC2 ? etaC1 : etaC2;

  /* eta_P^soc: ||z - B F q - d|| / (1 + ||d||) */
  og_fill_d(g, dv);
  og_apply_F(g, q, Fq);
  og_apply_B(g, omega, Fq, BFq);
  for (long i = 0; i < nz; ++i) r[i] = z[i] - BFq[i] - dv[i];
  double psoc = og_l2(g, r, nz) / (1.0 + og_l2(g, dv, nz));
  double etaPsoc = etaP > psoc ? etaP : psoc;

  /* eta_D^soc: ||F^*B^*beta + alpha|| / (1 + ||F^*B^*beta|| + ||alpha||) */
  og_apply_Bt(g, omega, beta, Bb);
  og_apply_Ft(g, Bb, FBb);
  for (long i = 0; i < nq; ++i) r[i] = FBb[i] + alpha[i];
  double dsoc = og_l2(g, r, nq) / (1.0 + og_l2(g, FBb, nq) + og_l2(g, alpha, nq));
  double etaDsoc = etaD > dsoc ? etaD : dsoc;

  double primal = 0.0;
  for (long i = 0; i < nn; ++i) primal += c[i] * phi[i];

  double eta = etaP;
  if (etaD > eta) eta = etaD;
  if (etaC > eta) eta = etaC;
  out[OG_ETA_DOT] = eta;
  out[OG_ETA_P] = etaP;
  out[OG_ETA_D] = etaD;
  out[OG_ETA_C] = etaC;
  out[OG_ETA_PSOC] = etaPsoc;
  out[OG_ETA_DSOC] = etaDsoc;
  out[OG_PRIMAL_OBJ] = primal;
  out[OG_DUAL_OBJ] = dual;
  out[OG_GAP] = fabs(primal - dual) / (1.0 + fabs(primal) + fabs(dual));

  free(Aphi); free(r); free(Atal); free(tmpn); free(acc); free(f); free(rc); free(Fq);
  free(BFq); free(dv); free(Bb); free(FBb); free(wa0); free(gv); free(rb);
}

/* ---- the solve loop with the sigma rule (Sec. 5.3) ------------------------ */

/* Runs Algorithm 2 from the given state.  Every check_every iterations (0 = never)
 * it evaluates og_kkt, stops when eta_dot <= tol, and otherwise updates sigma:
 * sigma *= s_sigma if eta_P^soc/eta_D^soc > s_r, sigma /= s_sigma if the ratio is
 * below 1/s_r.  hist (may be NULL) receives OG_NUM_KKT+2 doubles per check:
 * (iteration, sigma used, kkt...).  Returns the number of iterations run;
 * *sigma_io is updated in place. */
long og_solve(const og_grid *g, double tau, double *sigma_io, double s_sigma, double s_r,
              int check_every, double tol, long maxit, const double *c, const double *omega,
              double *phi, double *z, double *q, double *alpha, double *beta, double *kkt_out,
              double *hist, long hist_cap, long *hist_len) {
  og_params p;
  p.tau = tau;
  p.sigma = *sigma_io;
  long nh = 0;
  long k = 0;
  double kk[OG_NUM_KKT];
  for (int i = 0; i < OG_NUM_KKT; ++i) kk[i] = NAN;
  while (k < maxit) {
    og_iterate(g, &p, c, omega, phi, z, q, alpha, beta);
    ++k;
    if (check_every > 0 && k % check_every == 0) {
      og_kkt(g, c, omega, phi, z, q, alpha, beta, kk);
      if (hist && nh < hist_cap) {
        double *row = hist + nh * (OG_NUM_KKT + 2);
        row[0] = (double)k;
        row[1] = p.sigma;
        for (int i = 0; i < OG_NUM_KKT; ++i) row[2 + i] = kk[i];
        ++nh;
      }
      if (kk[OG_ETA_DOT] <= tol) break;
      double ratio = kk[OG_ETA_PSOC] / kk[OG_ETA_DSOC];
      if (ratio > s_r)
        p.sigma *= s_sigma;
      else if (ratio < 1.0 / s_r)
        p.sigma /= s_sigma;
    }
  }
  if (kkt_out) {
    og_kkt(g, c, omega, phi, z, q, alpha, beta, kk);
    for (int i = 0; i < OG_NUM_KKT; ++i) kkt_out[i] = kk[i];
  }
  if (hist_len) *hist_len = nh;
  *sigma_io = p.sigma;
  return k;
}
