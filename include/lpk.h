/*
 * lpk.h -- C ABI of the GB300 (sm_103a) library for the interior-point method
 * of Cui, Morikuni, Tsuchiya and Hayami, "Implementation of interior-point
 * methods for LP based on Krylov subspace iterative solvers with
 * inner-iteration preconditioning" (arXiv:1604.07491).
 *
 * Problem (Sec. 1, primal-dual pair): min c^T x s.t. A x = b, x >= 0, and its
 * dual max b^T y s.t. A^T y + s = c, s >= 0, with A an m x n sparse matrix.
 *
 * Conventions for every entry point:
 *  - The caller owns every input and output buffer.  Vector arguments are
 *    host pointers when on_device == 0 and CUDA device pointers of the
 *    context's device when on_device != 0 (for instance torch tensors).
 *  - All vectors are contiguous double arrays in the caller's (natural) row
 *    and column numbering.  Matrices are CSR with 0-based int32 column
 *    indices and int64 row pointers.
 *  - Work is ordered on the context's CUDA stream; every call returns after
 *    its results are written (the stream is synchronised before return).
 *  - No call aborts or exits.  Errors are returned as lpk_status and a
 *    message is available from lpk_last_error().  A context is not
 *    thread-safe: use one context per host thread.
 *  - Device-side waits (grid barriers of the persistent kernels) are bounded;
 *    when a bound is hit the call returns LPK_TIMEOUT and the context stays
 *    usable.
 */
#ifndef LPK_H
#define LPK_H

#include <stdint.h>

#ifdef __cplusplus
#define LPK_API extern "C"
#else
#define LPK_API
#endif

typedef enum lpk_status {
  LPK_OK = 0,
  LPK_MAX_IPM_ITER = 1,           /* interior-point iteration cap (99, Sec. 4.2) hit  */
  LPK_KRYLOV_STALL = 2,           /* a Krylov solve ended above its tolerance         */
  LPK_DIVERGED = 3,               /* interior-point iterates became non-finite ('f')  */
  LPK_BREAKDOWN = 4,              /* Krylov recurrence produced a non-positive divisor */
  LPK_TIMEOUT = 5,                /* a bounded device-side wait expired               */
  LPK_EMPTY_ROW_INCONSISTENT = 6, /* empty row i of A with b_i != 0: infeasible       */
  LPK_EMPTY_COL_UNBOUNDED = 7,    /* empty column j of A with c_j < 0: unbounded      */
  LPK_INVALID_ARG = 8,            /* bad size, pointer, index or non-finite value     */
  LPK_OOM = 9,                    /* device allocation failed                         */
  LPK_CUDA_ERROR = 10             /* a CUDA runtime call failed                       */
} lpk_status;

/* Krylov method for the search-direction solve (Sec. 3).  MRNE and CGNE are
 * preconditioned by NE-SSOR inner iterations (Algorithm 5), AB-GMRES by NE-SOR
 * inner iterations (Algorithm 6). */
typedef enum lpk_krylov { LPK_MRNE = 0, LPK_CGNE = 1, LPK_ABGMRES = 2 } lpk_krylov;

/* LPK_FP64: everything in double.  LPK_MIXED: the inner sweeps read an FP32
 * copy of the scaled matrix (4-byte values) and accumulate in double, so the
 * preconditioner stays a fixed linear (for NE-SSOR, SPD) operator; the w-space
 * images A_hat^T z, the outer Krylov recurrences, scaling, residuals and step
 * logic are double. */
typedef enum lpk_precision { LPK_FP64 = 0, LPK_MIXED = 1 } lpk_precision;

/* Inner sweep kind for lpk_sweep: Algorithm 5 or Algorithm 6. */
typedef enum lpk_sweep_kind { LPK_NE_SSOR = 0, LPK_NE_SOR = 1 } lpk_sweep_kind;

typedef struct lpk_ctx lpk_ctx;
typedef struct lpk_problem lpk_problem;

/* Sparse A in CSR.  row_ptr[m+1] (int64, row_ptr[0] = 0, nondecreasing),
 * col_idx[nnz] (int32 in [0, n)), val[nnz] (finite doubles).  Duplicate
 * (row, column) pairs are rejected.  on_device selects host or device
 * pointers for the three arrays. */
typedef struct lpk_matrix {
  int32_t m, n;
  int64_t nnz;
  const int64_t *row_ptr;
  const int32_t *col_idx;
  const double *val;
  int32_t on_device;
  int32_t reserved;
} lpk_matrix;

/* Options of lpk_lp_solve.  Defaults (lpk_default_options) follow Sec. 2.1
 * and Sec. 4.2: tol = 1e-8 (eps_out), eta = 0.9995 in [0.9, 1), phi = 1e-5,
 * sigma_max = 0.208, eps_in0 = 1e-6 (clamped to [1e-14, 1e-4]), max_ipm = 99,
 * max_krylov = 0 (means m).  inner_sweeps (ell) and omega are the inner
 * iteration parameters (odd ell keeps the NE-SSOR preconditioner SPD,
 * Sec. 3.3). */
typedef struct lpk_options {
  double tol;
  double eta;
  double phi;
  double sigma_max;
  double eps_in0;
  double omega;
  double start_tol;   /* Krylov tolerance of the two starting-point solves */
  double backtrack;   /* shrink factor of the centrality backtracking       */
  int32_t max_ipm;
  int32_t max_krylov;
  int32_t inner_sweeps;
  int32_t solver;     /* lpk_krylov    */
  int32_t precision;  /* lpk_precision */
  int32_t verbose;    /* 1: one line per interior-point iteration on stderr */
  uint64_t color_seed;
  int32_t corrector;  /* 0: corrector stage by `solver`; 1: by BA-GMRES with
                         NR-SOR on its least-squares form (Sec. 3.2)       */
  int32_t max_correctors; /* 0..10 multiple centrality correctors per
                         iteration after the predictor-corrector direction
                         (the multi-corrector framework Sec. 4.3 and 5 name;
                         Gondzio's method), each one more Krylov solve;
                         0 = the paper's single corrector (default)        */
} lpk_options;

/* Result summary of lpk_lp_solve.  gamma is the error measure of
 * Eq. (errorMeasureDef); pinf = ||b - Ax|| / max(||b||, 1),
 * dinf = ||c - A^T y - s|| / max(||c||, 1),
 * rel_gap = |c^T x - b^T y| / (1 + |c^T x|). */
typedef struct lpk_info {
  int32_t status;
  int32_t ipm_iters;
  int64_t krylov_iters_total;
  int32_t n_colors;
  int32_t krylov_failures;
  double gamma, rel_gap, pinf, dinf, mu, obj_primal, obj_dual;
  double solve_ms;
  int32_t correctors;  /* centrality correctors accepted over the solve */
  int32_t reserved;
} lpk_info;

/* Result of one Krylov solve: iterations over all restarts, whether the
 * explicit scaled residual ||f_hat - A_hat dw|| <= tol ||f_hat|| holds, and
 * both residual norms. */
typedef struct lpk_krylov_info {
  int32_t iters;
  int32_t converged;
  int32_t restarts;
  int32_t breakdown;
  double res0;
  double res;
} lpk_krylov_info;

/* Counters of one context since its creation or the last lpk_reset_stats:
 * every kernel launch the library issued, and for the persistent Krylov
 * kernel (the dominant kernel) its launches, their device time measured with
 * CUDA events on the context stream, the Krylov iterations, inner-sweep
 * passes (one forward or backward pass over all colors), FP64 row passes
 * over A_hat (products and residuals) and CSC passes (w-space images). */
typedef struct lpk_stats {
  int64_t launches;
  int64_t krylov_launches;
  double krylov_ms;
  int64_t krylov_iters;
  int64_t sweep_passes;
  int64_t row_passes;
  int64_t csc_passes;
  int64_t barriers;
  int32_t last_cluster_size;  /* 0: the last Krylov launch used the grid path */
  int32_t last_resident;      /* 1: it kept every warp's rows in shared memory */
  int64_t basis_passes;       /* AB-GMRES: m-row passes over one basis vector
                                 (four per vector and iteration in the two
                                 Gram-Schmidt passes, one per vector in V p) */
  int64_t spmv_launches;      /* sparse-product kernels launched by lpk_spmv */
  double spmv_ms;             /* their CUDA-event time on the context stream
                                 (the product kernel alone, without the
                                 gather/scatter between numberings) */
  double phase_ms[4];         /* with phase timing on (lpk_set_phase_timing):
                                 the persistent kernel's time between barriers,
                                 by what the phase did: [0] vector updates,
                                 reductions and the rest, [1] inner-sweep color
                                 phases, [2] AB-GMRES/BA-GMRES orthogonalisation
                                 (with the product w = A_hat z before it),
                                 [3] the w-space image A_hat^T z */
  int32_t last_u_global;      /* 1: the last cluster launch kept u in global memory */
  int32_t reserved;
  int64_t tune_probes;        /* timing probes the autotuner launched */
  int64_t tune_cache_hits;    /* problems whose path came from the tuning cache */
} lpk_stats;

/* Execution path of the persistent Krylov kernel.
 *  LPK_EXEC_AUTO:    on the first Krylov solve of each problem, a few
 *                    iterations of every path (grid; clusters of 16, 8, 4
 *                    CTAs with u in shared or in global memory) are timed on
 *                    the actual system and the fastest is kept for that
 *                    problem.  The choice is cached by problem shape (rows,
 *                    columns, nonzeros, colors, longest row, solver, value
 *                    precision, SM count) for the process; when the
 *                    environment variable LPK_TUNE_CACHE names a file, the
 *                    choices are appended to it and read back by later
 *                    processes, so known shapes skip the probes.
 *  LPK_EXEC_GRID:    every SM, software grid barrier, u in global memory.
 *  LPK_EXEC_CLUSTER: the cluster path (LPK_INVALID_ARG at solve time if u does
 *                    not fit).
 *  LPK_EXEC_BATCH:   the cluster path with a cluster size fixed by the problem
 *                    alone (no timing): the smallest of 4, 8, 16 CTAs that
 *                    gives every warp at most three rows per color and keeps
 *                    the rows resident.  For solves that share the GPU
 *                    (batched and serving modes): small clusters leave room
 *                    for many problems at once, and a problem gives bitwise
 *                    the same result alone and among others.  LPK_INVALID_ARG
 *                    at solve time if u does not fit in 16 CTAs.
 * Or-ing LPK_EXEC_NO_RESIDENT disables the shared-memory row cache (by
 * default each warp keeps the column indices and values of its rows in shared
 * memory for the whole launch when they fit).  On the cluster path the sweep
 * vector u lives in the CTAs' shared memory or in global memory (L2): by
 * default in global memory when a color carries 512 or more entries per CTA
 * (the autotuner, in LPK_EXEC_AUTO, times both); or-ing LPK_EXEC_U_SHARED or
 * LPK_EXEC_U_GLOBAL fixes the choice.
 * cluster_size: 0 = chosen from nnz, else 2, 4, 8 or 16 CTAs. */
typedef enum lpk_exec {
  LPK_EXEC_AUTO = 0,
  LPK_EXEC_GRID = 1,
  LPK_EXEC_CLUSTER = 2,
  LPK_EXEC_BATCH = 3,
  LPK_EXEC_NO_RESIDENT = 4,
  LPK_EXEC_U_SHARED = 8,
  LPK_EXEC_U_GLOBAL = 16
} lpk_exec;

/* Create a context on CUDA device `device`, ordered on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The context owns its
 * device workspace; the stream stays owned by the caller. */
LPK_API lpk_status lpk_create(lpk_ctx **ctx, int32_t device, void *cuda_stream);
LPK_API void lpk_destroy(lpk_ctx *ctx);
LPK_API const char *lpk_last_error(const lpk_ctx *ctx);
LPK_API void lpk_default_options(lpk_options *opt);
LPK_API lpk_status lpk_get_stats(const lpk_ctx *ctx, lpk_stats *out);
LPK_API lpk_status lpk_reset_stats(lpk_ctx *ctx);
LPK_API lpk_status lpk_set_exec(lpk_ctx *ctx, int32_t exec, int32_t cluster_size);

/* Failure detection of the grid path (the paper has no counterpart).  Every
 * wait of the persistent kernel's software grid barrier is bounded by
 * `seconds` of %globaltimer (default 5; must be > 0): when it runs out, the
 * CTA records LPK_TIMEOUT, every CTA leaves the kernel at its next barrier,
 * and the call returns LPK_TIMEOUT with the context still usable.
 * test_stall_barrier (testing only, 0 = off): in each grid-path launch, CTA 0
 * withholds its arrival at the grid barrier with that number (counted from 1
 * in the launch), so every wait on it runs out; this is how the timeout path
 * is exercised without faulting the GPU.  The cluster path's hardware
 * barriers have no software wait and are not affected. */
LPK_API lpk_status lpk_set_wait_limit(lpk_ctx *ctx, double seconds, int64_t test_stall_barrier);

/* Phase timing of the persistent Krylov kernel (on != 0; default off): the
 * first CTA reads %globaltimer at every barrier and charges the interval to
 * the kind of phase that ended there (lpk_stats.phase_ms).  Costs one timer
 * read and a shared-memory update per barrier in one thread. */
LPK_API lpk_status lpk_set_phase_timing(lpk_ctx *ctx, int32_t on);

/* Copy A to the device, validate it, remove empty rows and columns (the only
 * preprocessing of Sec. 4.2) and compute the multicolor row order on the
 * device: rows are colored greedily in decreasing priority
 * splitmix64(color_seed ^ row), each taking the smallest color not used by a
 * higher-priority row sharing a column, so rows of one color share no column
 * and NE-(S)SOR can update them in parallel (the paper sweeps rows in natural
 * order, Algorithms 5-6).  The problem owns device copies of A (permuted CSR,
 * CSC, scaled FP64 and FP32 values) and is immutable afterwards. */
LPK_API lpk_status lpk_prepare(lpk_ctx *ctx, const lpk_matrix *A, uint64_t color_seed,
                               lpk_problem **P);
/* Frees a problem.  Destroying a context releases the device memory of its
 * remaining problems; their handles must then still be passed to
 * lpk_problem_free (which only releases the host handle) and nothing else. */
LPK_API void lpk_problem_free(lpk_problem *P);

/* Sizes of the prepared problem: m, n, nnz of the input and the number of
 * colors.  Any output pointer may be NULL. */
LPK_API lpk_status lpk_problem_dims(const lpk_problem *P, int32_t *m, int32_t *n, int64_t *nnz,
                                    int32_t *n_colors);

/* Copy the coloring to host arrays: color[m] (color of each input row; -1 for
 * a removed empty row), color_ptr[n_colors+1] and perm[m'] (kept rows in
 * sweep order, input numbering).  Any output pointer may be NULL. */
LPK_API lpk_status lpk_problem_coloring(lpk_ctx *ctx, const lpk_problem *P, int32_t *color,
                                        int32_t *perm, int32_t *color_ptr);

/* Row scaling of Sec. 3.5 for D = diag(sqrt(d2)): rho[i] = ||(A D)_i||_2 and
 * ahat[k] = a_k sqrt(d2_col(k)) / rho_row(k) in the input CSR order.  d2[n]
 * > 0; rho[m]; ahat[nnz]. ahat may be NULL. */
LPK_API lpk_status lpk_scale_rows(lpk_ctx *ctx, lpk_problem *P, const double *d2, double *rho,
                                  double *ahat, int32_t on_device);

/* y = A x (transpose == 0; x[n], y[m]) or y = A^T x (transpose != 0; x[m],
 * y[n]) with the unscaled A, in double. */
LPK_API lpk_status lpk_spmv(lpk_ctx *ctx, lpk_problem *P, int32_t transpose, const double *x,
                            double *y, int32_t on_device);

/* Inner iterations on the row-scaled matrix A_hat = D_cal^-1 A D (Sec. 3.5,
 * unit row norms), rows visited in the multicolor order:
 *  LPK_NE_SSOR (Algorithm 5): z[m] = C^<ell> g, u[n] = A_hat^T z.
 *  LPK_NE_SOR  (Algorithm 6): u[n] = B^<ell> g, z[m] = the accumulated row
 *                             corrections, u = A_hat^T z.
 * g[m] is in the scaled space.  precision LPK_MIXED runs the sweep in FP32. */
LPK_API lpk_status lpk_sweep(lpk_ctx *ctx, lpk_problem *P, const double *d2, const double *g,
                             int32_t kind, int32_t inner_sweeps, double omega, int32_t precision,
                             double *z, double *u, int32_t on_device);

/* Search-direction solve of Sec. 2.2: A diag(d2) A^T dy = f through the
 * minimum-norm problem min ||dw|| s.t. A D dw = f, D = diag(sqrt(d2))
 * (Eq. minnrmprob), row-scaled (Sec. 3.5), solved by `solver` (Algorithms
 * 2-4) with `inner_sweeps` inner iterations of relaxation `omega`, to the
 * scaled tolerance ||f_hat - A_hat dw|| <= tol ||f_hat|| or max_iter
 * iterations (0 -> m).  Outputs dy[m] and dw[n] = D A^T dy (dw may be NULL);
 * for rank-deficient A, dy is the one the iteration reaches from dy = 0.
 * kinfo may be NULL.  Returns LPK_OK even when the tolerance is not reached
 * (kinfo->converged tells). */
LPK_API lpk_status lpk_ne_solve(lpk_ctx *ctx, lpk_problem *P, const double *d2, const double *f,
                                int32_t inner_sweeps, double omega, int32_t solver,
                                int32_t precision, double tol, int32_t max_iter, double *dy,
                                double *dw, lpk_krylov_info *kinfo, int32_t on_device);

/* lpk_ne_solve without any device allocation, for callers that cannot call
 * cudaMalloc while they solve: applications whose device memory belongs to
 * their own allocator (a caching allocator or a fixed arena), and services
 * that must not hit an out-of-memory error mid-solve.  The paper has no
 * counterpart: this is a deployment variant of lpk_ne_solve.
 *  - d2[n], f[m], dy[m] and dw[n] (dw may be NULL) must be device memory of
 *    the context's GPU (or managed memory); anything else is rejected with
 *    LPK_INVALID_ARG.  Lengths are those of lpk_ne_solve.
 *  - solver LPK_MRNE or LPK_CGNE; always runs the grid path (one CTA per SM).
 *  - All temporaries live in one 32 MiB array of device memory, reserved when
 *    the first context on a device is created (lpk_create looks up its
 *    address) and held by that GPU until the process exits.  A problem
 *    needing more (about 8 doubles per row and column, plus 260 KB) is
 *    rejected with LPK_INVALID_ARG and a message giving the size.
 *  - Every call uses the same array and leaves its contents behind: calls
 *    that overlap on the GPU (other streams, other host threads, other
 *    contexts on the same device) race; serialise them.
 *  - The call is synchronous on the context stream, like lpk_ne_solve.
 *  - Same results as lpk_ne_solve on the grid path (lpk_set_exec). */
LPK_API lpk_status lpk_ne_solve_noalloc(lpk_ctx *ctx, lpk_problem *P, const double *d2, const double *f,
                                        int32_t inner_sweeps, double omega, int32_t solver,
                                        int32_t precision, double tol, int32_t max_iter, double *dy,
                                        double *dw, lpk_krylov_info *kinfo);

/* Interior-point solve (Algorithm 1 with the w-recurrence of Sec. 2.2): b[m],
 * c[n] in; x[n], y[m], s[n] out.  opt may be NULL (defaults).  info may be
 * NULL.  Returns LPK_OK when Gamma <= tol and rel_gap <= tol. */
/* The corrector stage in least-squares form (Sec. 3.2, Eq. ba_ne):
 * min || diag(sqrt(d2)) A^T dy - r ||, i.e. the normal equations of the first
 * kind A diag(d2) A^T dy = A diag(sqrt(d2)) r, solved in m-space by BA-GMRES
 * (left-preconditioned GMRES) with NR-SOR inner iterations on the row-scaled
 * matrix of Sec. 3.5.  d2[n] > 0 and r[n] in; dy[m] and dw[n] =
 * diag(sqrt(d2)) A^T dy out (dw, the minimum-norm solution of
 * A diag(sqrt(d2)) dw = A diag(sqrt(d2)) r, may be NULL).  Convergence: the
 * explicit scaled residual ||f_hat - A_hat dw|| <= tol ||f_hat|| with
 * f_hat = A_hat r (kinfo->converged).  inner_sweeps = NR-SOR sweeps per
 * application, max_iter 0 -> m.  Layout and staging as lpk_ne_solve.
 * precision is accepted for symmetry and ignored: BA-GMRES sweeps in FP64
 * (a left preconditioner must have the null space of the scaled matrix; the
 * FP32 copy's differs and the residual stalls near 1e-7). */
LPK_API lpk_status lpk_ls_solve(lpk_ctx *ctx, lpk_problem *P, const double *d2, const double *r,
                                int32_t inner_sweeps, double omega, int32_t precision, double tol,
                                int32_t max_iter, double *dy, double *dw, lpk_krylov_info *kinfo,
                                int32_t on_device);

LPK_API lpk_status lpk_lp_solve(lpk_ctx *ctx, lpk_problem *P, const double *b, const double *c,
                                const lpk_options *opt, double *x, double *y, double *s,
                                lpk_info *info, int32_t on_device);

/* ------------------------------------------------------------------------
 * Many LPs on one GPU (the paper solves one LP at a time and has no
 * counterpart).  Independent LPs run side by side, each on its own context
 * (one host thread and CUDA stream per LP) with its persistent Krylov kernel
 * on a thread-block cluster of its own; contexts in LPK_EXEC_AUTO mode take
 * the LPK_EXEC_BATCH path for these solves, so every LP gives bitwise the
 * result it gives when solved alone on that path.  With more than 8 LPs at
 * once, set the environment variable CUDA_DEVICE_MAX_CONNECTIONS to 32 before
 * the process creates its CUDA context: with the default of 8 hardware work
 * queues, streams share queues and one LP's persistent kernel holds back the
 * launches of another (measured: 2.7 vs 6.4 LPs/s for 16 assignment LPs).
 * ------------------------------------------------------------------------ */

/* Solve `count` LPs at once: LP i is problems[i] with b[i], c[i] (lengths as
 * for lpk_lp_solve), results into x[i], y[i], s[i] and info[i].  Each problem
 * must belong to a different context, and no context may be set to
 * LPK_EXEC_GRID (its barrier spans every SM, so it cannot share the GPU):
 * LPK_INVALID_ARG otherwise, before anything runs (the message is on the
 * offending context).  `opt` (NULL: defaults) applies to all.  Returns LPK_OK
 * if every solve returned LPK_OK, else the status of the first LP (by index)
 * that did not; info[i].status holds each LP's own status.  Blocks until all
 * are done. */
LPK_API lpk_status lpk_lp_solve_batch(int32_t count, lpk_problem *const *problems, const double *const *b,
                                      const double *const *c, const lpk_options *opt, double *const *x,
                                      double *const *y, double *const *s, lpk_info *info,
                                      int32_t on_device);

/* Continuous-batching server.  `lanes` worker threads, each with its own
 * context and non-blocking stream on `device`, take submitted LPs in arrival
 * order as soon as a lane is free and the LP's device memory estimate (the
 * prepared problem, the interior-point and Krylov workspaces and, for
 * AB-GMRES, its basis sized to the iteration cap) fits in what the running
 * LPs leave of `mem_budget` (0: half the free device memory at creation); an
 * LP that does not fit waits while later, smaller ones may start, and the
 * oldest waiting LP starts whenever nothing runs, even if it alone exceeds
 * the budget.  Each LP's matrix, iterate and Krylov state stay on the device
 * from admission to its result. */
typedef struct lpk_server lpk_server;
typedef struct lpk_server_config {
  int32_t device;
  int32_t lanes;        /* 1..256, default 16 */
  int64_t mem_budget;   /* bytes; 0 = half the free device memory */
  uint64_t color_seed;  /* coloring seed of every LP (as lpk_prepare) */
} lpk_server_config;
/* Per-LP outcome.  Times are seconds on the server's steady clock
 * (lpk_server_now): submission, admission to a lane, result ready. */
typedef struct lpk_request_result {
  lpk_info info;
  int32_t status;       /* lpk_prepare / lpk_lp_solve status */
  int32_t lane;
  double t_submit, t_start, t_end;
  int64_t mem_bytes;    /* device memory charged at admission */
  char error[256];      /* lpk_last_error text when status != LPK_OK */
} lpk_request_result;
typedef struct lpk_server_stats_t {
  int64_t pending, running, completed;
  int64_t mem_in_use, mem_peak, mem_budget;
  int32_t lanes, reserved;
} lpk_server_stats_t;

LPK_API void lpk_server_default_config(lpk_server_config *cfg);
/* cfg NULL: defaults.  LPK_CUDA_ERROR if a lane's stream or context cannot
 * be created. */
LPK_API lpk_status lpk_server_create(lpk_server **srv, const lpk_server_config *cfg);
/* Stops taking LPs, drops the ones not yet admitted, waits for the running
 * ones and releases everything.  No other call on srv may run concurrently
 * or follow. */
LPK_API void lpk_server_destroy(lpk_server *srv);
LPK_API double lpk_server_now(const lpk_server *srv);
/* Queue one LP (A in host CSR, A->on_device must be 0; b[m], c[n] host).
 * Everything is copied: the caller's arrays may be reused on return.  Options
 * as lpk_lp_solve (NULL: defaults).  Returns a ticket for lpk_server_wait.
 * Thread-safe. */
LPK_API lpk_status lpk_server_submit(lpk_server *srv, const lpk_matrix *A, const double *b, const double *c,
                                     const lpk_options *opt, int64_t *ticket);
/* Wait up to timeout_s seconds (< 0: no limit) for a ticket's result; copies
 * x[n], y[m], s[n] (each may be NULL) and the outcome, then releases the
 * ticket.  LPK_TIMEOUT if not ready (the ticket stays valid);
 * LPK_INVALID_ARG for an unknown ticket.  The LP's own status is in
 * res->status.  Thread-safe. */
LPK_API lpk_status lpk_server_wait(lpk_server *srv, int64_t ticket, double timeout_s, double *x, double *y,
                                   double *s, lpk_request_result *res);
LPK_API lpk_status lpk_server_stats(lpk_server *srv, lpk_server_stats_t *out);

#endif /* LPK_H */
