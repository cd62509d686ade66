/*
 * dot.h -- C ABI of the GB300 (sm_103a) dynamic optimal transport solver.
 *
 * The solver runs the inexact proximal ALM of arXiv 2505.05424 (Algorithm 1,
 * explicit steps Algorithm 2, Sec. 4) on the linear SOCP reformulation (Sec. 3,
 * eq. (opt-dualsocalm-ran)) of the staggered-grid discretisation (Sec. 2.2,
 * eq. (opt-disdualori)) of the Benamou-Brenier problem with quadratic cost, or of
 * its weighted variant with obstacles (Sec. 5.4, eq. (opt-weightdualori)).
 * Stopping test and penalty rule: Sec. 5.3.
 *
 * Grid.  D spatial axes (2 or 3) on [0,1]^D with N_d cells each; the potential
 * phi lives on the cell centres (h_d = 1/N_d) so each spatial axis has N_d - 1
 * interior faces; time [0,1] has T intervals and T+1 nodes (h_0 = 1/T).
 *
 * Host array layouts (all C-order, float64, owned by the caller; the library
 * copies what it needs and never keeps a caller pointer after a call returns):
 *   rho0, rho1, mask : [N_1]...[N_D]                    (cell-centred samples)
 *   phi              : [T+1][N_1]...[N_D]                (nodes G^c)
 *   rho              : [T][N_1]...[N_D]                  (time faces G^s_0)
 *   m                : D blocks, block d of shape [T+1][..][N_d - 1][..]  (G^s_d)
 *   q, alpha         : the concatenation (G^s_0; G^s_1; ...; G^s_D)
 *   beta             : [4D+2][T][N_1]...[N_D]            (one cone per time face)
 *
 * Status codes: 0 success; < 0 error (the context, if any, stays valid unless
 * the code is DOT_ECUDA); > 0 soft status with valid results.
 * dot_last_error() returns a human-readable message for the last failing call on
 * that context (or on the calling thread when ctx is NULL).
 *
 * Threading: contexts are independent; calls on different contexts may run
 * concurrently from different threads, calls on one context must not.
 */
#ifndef DOT_GB300_H
#define DOT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DOT_OK 0
#define DOT_EINVAL (-1)     /* bad argument: shape, non-finite or negative density, mass */
#define DOT_ENOMEM (-2)     /* workspace too small or device allocation failed */
#define DOT_ECUDA (-3)      /* a CUDA call failed; the context must be destroyed */
#define DOT_EDIVERGED (-4)  /* a stopping measure became non-finite */
#define DOT_ETIMEOUT (-5)   /* dot_options.max_seconds elapsed; state is readable */
#define DOT_ENOTCONV 1      /* maxit reached before the tolerance; state is readable */

typedef struct {
  int D;      /* spatial dimension: 2 or 3 */
  int T;      /* time intervals, >= 1 */
  int N[3];   /* cells per spatial axis, each >= 2; N[d] for d >= D is ignored */
} dot_grid;

typedef enum {
  DOT_FP64 = 0,   /* every field and every operation in FP64 (the reference path) */
  DOT_MIXED = 1   /* FP32 stencils/projection, 3xTF32 DCT GEMMs on the tensor cores,
                     two-float (48-bit) multipliers and potential, FP64 reductions,
                     one refinement step of the Poisson solve per iteration */
} dot_precision;

typedef struct {
  dot_precision prec;
  double tau;              /* dual step length in (0, 2); Algorithm 1; default 1.9 (Sec. 5.2) */
  double sigma0;           /* initial penalty sigma > 0; default 1 */
  double s_sigma;          /* penalty factor s_sigma > 1; default 1.25 (Sec. 5.3) */
  double s_r;              /* ratio threshold s_r > 1; default 2 (Sec. 5.3) */
  int check_every;         /* evaluate the stopping measures and update sigma every
                              check_every iterations; 0 = never; default 10 */
  double obstacle_weight;  /* omega on masked cells (Sec. 5.4); default 1e-6 */
  double max_seconds;      /* wall-clock limit per dot_solve call; 0 = none */
  int use_graphs;          /* mixed path: replay each check period of dot_solve (the
                              check_every iterations and the stopping measures) from
                              a CUDA graph captured on first use; 0 = launch kernel by
                              kernel, as solves under dot_profile always do.  The
                              results are the same bit for bit; default 1 */
  double tau_switch_below; /* mixed path: once a stopping-measure check finds eta_dot
                              <= tau_switch_below, the dual step length becomes 1 (the
                              tau of ALG2, Sec. 5.2) for the rest of the solve.  With
                              tau near 2 the dual residual A^*alpha + c keeps a share
                              (1 - tau) of itself each iteration and sums the FP32
                              rounding of q and z (about 1e-7 relative) over ~1/(2 - tau)
                              iterations, which stalls eta_dot near 2e-7; with tau = 1
                              it does not.  0 = never; the FP64 path ignores it (it runs
                              the oracle's fixed-tau recurrence); default 3e-7 */
} dot_options;

/* Index of each value in the kkt[] array filled by dot_get / dot_kkt. */
enum {
  DOT_KKT_ETA = 0,        /* eta_dot = max(eta_P, eta_D, eta_C) (Sec. 5.3) */
  DOT_KKT_ETA_P = 1,
  DOT_KKT_ETA_D = 2,
  DOT_KKT_ETA_C = 3,
  DOT_KKT_ETA_P_SOC = 4,
  DOT_KKT_ETA_D_SOC = 5,
  DOT_KKT_PRIMAL = 6,     /* <c, phi>, the objective of problem (8), c in densities */
  DOT_KKT_DUAL = 7,       /* dual objective (11) at the current alpha */
  DOT_KKT_GAP = 8,        /* |primal - dual| / (1 + |primal| + |dual|) */
  DOT_KKT_ITERS = 9,      /* iterations run since dot_create / dot_set_state */
  DOT_KKT_SIGMA = 10,     /* current penalty */
  DOT_KKT_LEN = 11
};

typedef struct dot_ctx dot_ctx;

/* Fill *opt with the defaults listed above (prec = DOT_MIXED). */
void dot_default_options(dot_options *opt);

/* Device bytes a context of this grid and precision needs (for admission by HBM
 * footprint).  Returns 0 for an invalid grid. */
size_t dot_workspace_bytes(const dot_grid *grid, dot_precision prec);

/* Create a solve.  rho0/rho1: non-negative finite samples, each with positive
 * total mass; they are normalised to mass 1 and enter the problem as the vector
 * c of eq. (defc).  mask: NULL or one byte per cell, non-zero = obstacle
 * (omega = obstacle_weight there, Sec. 5.4).  opt: NULL = defaults.
 * workspace: device memory of at least dot_workspace_bytes() bytes, 256-byte
 * aligned, owned by the caller and kept alive until dot_destroy; NULL = the
 * library allocates (and frees) it itself.  stream: cudaStream_t to run on;
 * NULL = the legacy default stream.  The context belongs to the CUDA device
 * current at this call: every later call on it runs on that device and restores
 * the caller's current device on return.  The initial point is q = alpha =
 * beta = 0, sigma = sigma0 (0 lies in Q, Algorithm 1's input condition).
 * Returns DOT_EINVAL for bad shapes/densities, DOT_ENOMEM, or DOT_ECUDA. */
int dot_create(const dot_grid *grid, const double *rho0, const double *rho1,
               const uint8_t *mask, const dot_options *opt, void *workspace,
               size_t workspace_bytes, void *stream, dot_ctx **out);

/* Run Algorithm 2 until eta_dot <= tol at a check (Sec. 5.3) or maxit more
 * iterations.  tol <= 0 never stops early.  Returns DOT_OK when converged,
 * DOT_ENOTCONV at maxit, DOT_ETIMEOUT, DOT_EDIVERGED or DOT_ECUDA.  Blocks the
 * calling thread at every check (it reads the stopping measures).  With
 * opt.use_graphs (DOT_MIXED, not under dot_profile) each whole check period is
 * replayed from a CUDA graph captured on the first period; the results are the
 * same bit for bit as with kernel-by-kernel launches. */
int dot_solve(dot_ctx *ctx, double tol, long maxit);

/* Results.  Any pointer may be NULL.  rho = alpha_0 / h_0 and m_d = alpha_d / h_0
 * (Proposition 3.3: (Lambda_0, Lambda_bar) = (alpha_0, alpha_bar) solve (12)), as
 * densities: each time slice of rho integrates to 1, sum(rho) * h_1...h_D = 1.
 * c enters eq. (defc) as cell-average densities (mass / h_1...h_D), so
 * objective = -2 h_1...h_D <c, phi>, the squared Wasserstein-2 distance of the
 * discrete problem; kkt: DOT_KKT_LEN values measured at the current iterate. */
int dot_get(dot_ctx *ctx, double *rho, double *m, double *phi, double *objective, double *kkt);

/* Stopping measures of the current iterate (Sec. 5.3) into kkt[DOT_KKT_LEN]. */
int dot_kkt(dot_ctx *ctx, double *kkt);

/* Checkpoint / warm start: the iterate (q, alpha, beta), sigma and the iteration
 * count.  Layouts as in the file header; any output pointer may be NULL.  After
 * dot_set_state the next iteration starts from the given point (phi and z are
 * recomputed by Algorithm 2's first lines). */
int dot_get_state(dot_ctx *ctx, double *q, double *alpha, double *beta, double *sigma, long *iters);
int dot_set_state(dot_ctx *ctx, const double *q, const double *alpha, const double *beta,
                  double sigma, long iters);

/* Operator entry point: phi = (A^*A)^dagger b on rge(A^*) with the context's
 * Poisson solver (DCT-II along every axis as dense GEMMs, scale by the inverse
 * Neumann eigenvalues with the zero mode set to 0, DCT-III back; Sec. 4, the
 * phi-subproblem of Algorithm 2).  b, phi: [T+1][N_1]...[N_D] host arrays. */
int dot_poisson(dot_ctx *ctx, const double *b, double *phi);

/* Per-kernel timing.  dot_profile(ctx, 1) resets the counters and makes every
 * later launch on this context bracketed by CUDA events recorded on the
 * context's stream; the elapsed times are accumulated per kernel id at every
 * synchronisation point (stopping-measure checks, end of dot_solve).
 * dot_profile(ctx, 0) stops.  Profiled solves launch kernel by kernel (no graph
 * replay), so that every kernel is bracketed.  dot_profile_read copies, for kernel ids
 * 0..max-1, the total milliseconds and launch counts; it returns the number of
 * kernel ids (DOT_NUM_KERNELS).  dot_kernel_name(id) names each id. */
#define DOT_NUM_KERNELS 13
int dot_profile(dot_ctx *ctx, int enable);
int dot_profile_read(dot_ctx *ctx, double *ms_total, long *launches, int max);
const char *dot_kernel_name(int id);

/* Refined Poisson solve for callers that cannot allocate device memory (no
 * counterpart in the paper; it serves plugins of hosts that forbid allocation on
 * their worker threads, processes whose device memory is reserved by another
 * allocator, and loops with a fixed memory budget that must not risk an
 * allocation failing part way through).  It computes what dot_poisson computes for a DOT_MIXED
 * context -- phi = (A^*A)^dagger b by FP32/3xTF32 DCT solves with one refinement
 * step -- on caller-owned device buffers, and allocates nothing: all scratch
 * lives in one fixed __device__ array of the library (about 31 MB, held by every
 * GPU that loads the library until the process exits).
 *   b    : device, FP32, [T+1][N_1]...[N_D]           (read only)
 *   phi  : device, 2 floats per node (hi, lo) in the same order; phi = hi + lo
 *   stream: cudaStream_t or NULL; the call synchronises it before returning.
 * Limits: D in {2, 3}, T+1 in [2, 160] (the time axis runs the SIMT time pass,
 * built for at most 160 time nodes, as in DOT_MIXED contexts), every N_d in
 * [2, 256], (T+1) N_1...N_D <= 2^20 nodes; larger grids return DOT_EINVAL with a message from
 * dot_noalloc_last_error().  The first call on a device fetches the array's
 * device address and should come before any stream capture.  Every call shares
 * the array: calls whose work overlaps on the GPU race and must be serialised. */
int dot_poisson_f32_noalloc(const dot_grid *grid, const float *b, float *phi, void *stream);
const char *dot_noalloc_last_error(void);

void dot_destroy(dot_ctx *ctx);
const char *dot_last_error(const dot_ctx *ctx);

/* Library version string and the number of kernel launches issued by this
 * context so far (for launch accounting). */
const char *dot_version(void);
long dot_launch_count(const dot_ctx *ctx);

/* ---- Multilevel initialisation (Sec. 5, the "multilevel strategy") ----------
 *
 * dot_solve_multilevel solves the context's problem on grids coarsened by 2^v in
 * time and in every spatial axis, v = levels, ..., 1 (densities averaged over
 * 2^D-cell blocks, a block is an obstacle if any of its cells is), each level to
 * coarse_tol, or for coarse_tol <= 0 to the paper's max(tol * 10^-v, 1e-6),
 * starting every finer level -- and finally the context
 * itself, solved to tol -- from the coarser solution interpolated by
 * dot_prolong_state.  The context's state, sigma and iteration count are those of
 * a dot_set_state followed by dot_solve.  Coarse levels use temporary contexts of
 * the same precision and options on the same stream (their workspaces are
 * allocated with cudaMalloc and freed before the call returns).
 *   levels: 0..8; T and every N_d divisible by 2^levels, N_d / 2^levels >= 2.
 *   iters (nullable): levels + 1 entries, iters[v] = iterations on level v
 *   (iters[0] = the context's).
 * Returns dot_solve's status for the finest level, or an error.
 *
 * dot_prolong_state interpolates a state (q, alpha, beta in the host layouts of
 * dot_get_state) from grid gc to a grid gf of the same D with T and N_d at least
 * gc's: multilinear interpolation on each field's staggered sample positions
 * (time faces at (k + 1/2)/T and cell centres; space faces at time nodes k/T and
 * face positions j/N_d, with zero flux at the walls), constant beyond the
 * outermost centres; alpha and beta are scaled by gc.T / gf.T (they scale like
 * h_0).  Host only (no device work); any pointer pair may be NULL. */
int dot_solve_multilevel(dot_ctx *ctx, int levels, double tol, double coarse_tol, long maxit, long *iters);
int dot_prolong_state(const dot_grid *gc, const dot_grid *gf, const double *qc, const double *alc,
                      const double *betac, double *qf, double *alf, double *betaf);
const char *dot_multilevel_last_error(void);

/* ---- Serving: many solves advanced together (continuous batching) -----------
 *
 * The paper solves one problem at a time; this layer runs Algorithm 2 for many
 * independent DOT problems on one GPU.  Requests of the same grid share a batch:
 * a device workspace holding G solves whose per-iteration kernels advance every
 * active slot in one launch (one CUDA graph per batch covers check_every
 * iterations and the stopping measures).  After each such period the server
 * thread applies the stopping test and the penalty rule of Sec. 5.3 to every
 * slot, retires the slots that finished and admits queued requests into free
 * slots; a request for a grid with no free slot gets a new batch if its
 * workspace fits the memory budget, otherwise it waits (admission by device
 * memory footprint).  Batches of different grids run on separate streams and
 * overlap on the device.  Every slot runs the same recurrence, schedule and
 * kernels as a dot_create/dot_solve context of precision DOT_MIXED, so a
 * request's result does not depend on which other requests share its batch.
 *
 * Grids: D = 2 with every N_d a multiple of 4 (and at most 4096) are batched;
 * other grids get batches of one slot.
 * Threading: every function may be called from any thread. */
typedef struct dot_server dot_server;

typedef struct {
  size_t hbm_budget;   /* device bytes the batches may hold; 0 = 80% of free memory at creation */
  int max_slots;       /* most solves in one batch (1..256; default 64) */
  long target_nodes;   /* a batch gets about this many grid nodes, (T+1) N_1..N_D per slot,
                          within [1, max_slots] slots (default 4,194,304) */
  int use_graphs;      /* 1: one captured CUDA graph per batch and period (default); 0: plain launches */
  int idle_ms;         /* a batch with no solve for this long returns its memory (default 200) */
  int multilevel;      /* > 0: warm-start each large request by the multilevel strategy of Sec. 5 over
                          this many coarse levels, every level served as a request of its own grid
                          (as dot_solve_multilevel); 0 = off (default) */
  long long multilevel_min_nodes;  /* only requests with at least this many nodes (T+1) N_1..N_D and a
                                      grid divisible by 2^multilevel (default 1,000,000) */
  double multilevel_coarse_tol;    /* tolerance of the coarse levels; 0 = max(tol 10^-v, 1e-6) */
  int multilevel_masked;           /* 1: warm-start requests with obstacles too; 0 (default): serve them
                                      cold (their coarse levels, with obstacles grown to whole blocks,
                                      measured slower than a cold start) */
} dot_server_options;

void dot_server_default_options(dot_server_options *o);
/* opt: algorithm options (NULL = defaults; prec must be DOT_MIXED); sopt: NULL = defaults.
 * Starts the server thread on the calling thread's current device. */
int dot_server_create(const dot_options *opt, const dot_server_options *sopt, dot_server **out);
/* Queue a solve.  rho0, rho1, mask as for dot_create (copied before the call
 * returns); tol, maxit as for dot_solve; keep_fields: 1 = keep rho, m, phi for
 * dot_server_result, 0 = only the objective and the stopping measures.
 * *id receives the request id (> 0).  Returns DOT_EINVAL for bad arguments and
 * DOT_ENOMEM when a batch of one slot of this grid (dot_workspace_bytes-like
 * footprint) exceeds the server's hbm_budget, so that it could never run. */
int dot_server_submit(dot_server *srv, const dot_grid *grid, const double *rho0, const double *rho1,
                      const uint8_t *mask, double tol, long maxit, int keep_fields, long long *id);
/* Wait up to timeout_s seconds (< 0: forever, 0: poll) for request id.  Returns
 * DOT_OK when it has finished, with its solve status (as dot_solve's return) in
 * *status; DOT_ETIMEOUT when it has not; DOT_EINVAL for an unknown id. */
int dot_server_wait(dot_server *srv, long long id, double timeout_s, int *status);
/* Results of a finished request (any pointer may be NULL): rho, m, phi as for
 * dot_get (only with keep_fields), objective, kkt[DOT_KKT_LEN], and times[3] =
 * seconds since the server started at submission, admission and completion. */
int dot_server_result(dot_server *srv, long long id, double *rho, double *m, double *phi, double *objective,
                      double *kkt, double *times);
/* Forget a finished request and free its host copies. */
int dot_server_release(dot_server *srv, long long id);
/* Counters: out[0] queued, [1] running, [2] finished, [3] batches, [4] device
 * bytes held, [5] graph (or period) launches, [6] kernel launches, [7] most solves
 * running at once, [8] most batches at once.  Returns the number written (<= n). */
int dot_server_stats(dot_server *srv, double *out, int n);
/* Stops the server thread (queued and running requests are abandoned) and frees
 * every device buffer. */
void dot_server_destroy(dot_server *srv);
/* Message of the server's last failing call (or of the server thread's fatal
 * error); with srv NULL, of the calling thread's last failing dot_server_create.
 * The string stays valid until the calling thread's next call of this function. */
const char *dot_server_last_error(const dot_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* DOT_GB300_H */
