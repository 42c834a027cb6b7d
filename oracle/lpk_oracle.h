/*
 * lpk_oracle.h -- plain, slow, FP64 CPU oracle of the interior-point method of
 * Cui, Morikuni, Tsuchiya and Hayami, "Implementation of interior-point methods
 * for LP based on Krylov subspace iterative solvers with inner-iteration
 * preconditioning" (arXiv:1604.07491).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; both are fed by the seeded
 * generators and nothing else.
 *
 * Matrices are CSR: row_ptr[m+1] (int64), col_idx[nnz] (int32, sorted within a
 * row), val[nnz] (double).  All vectors are double.  Every function is
 * single-threaded and allocates its own scratch with malloc.
 */
#ifndef LPK_ORACLE_H
#define LPK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_MRNE = 0, ORC_CGNE = 1, ORC_ABGMRES = 2 };

enum {
  ORC_OK = 0,
  ORC_MAX_IPM_ITER = 1,
  ORC_KRYLOV_STALL = 2,
  ORC_DIVERGED = 3,
  ORC_BREAKDOWN = 4,
  ORC_EMPTY_ROW_INCONSISTENT = 6,
  ORC_EMPTY_COL_UNBOUNDED = 7,
  ORC_INVALID_ARG = 8,
  ORC_OOM = 9
};

typedef struct {
  double tol;          /* eps_out on Gamma and on the relative gap          */
  double eta;          /* step-length damping in [0.9, 1)                    */
  double phi;          /* centrality bound of the backtracking               */
  double sigma_max;    /* 0.208                                               */
  double eps_in0;      /* initial Krylov tolerance                           */
  double omega;        /* relaxation parameter of the inner sweeps           */
  double start_tol;    /* Krylov tolerance of the two starting-point solves  */
  double backtrack;    /* common shrink factor of the centrality backtracking */
  int32_t max_ipm;     /* 99                                                  */
  int32_t max_krylov;  /* 0 -> m                                              */
  int32_t inner_sweeps;/* ell                                                 */
  int32_t method;      /* ORC_MRNE, ORC_CGNE, ORC_ABGMRES                     */
  uint64_t color_seed;
  int32_t verbose;     /* 1: one line per interior-point iteration on stderr */
  int32_t corrector_ba;/* 1: corrector stage by BA-GMRES (NR-SOR), Sec. 3.2   */
  int32_t max_correctors; /* multiple centrality correctors per iteration (0: the
                             paper's single corrector)                       */
  int32_t pad;
} orc_options;

typedef struct {
  int32_t status;
  int32_t ipm_iters;
  int64_t krylov_iters_total;
  int32_t n_colors;
  int32_t krylov_failures;
  double gamma, rel_gap, pinf, dinf, mu, obj_primal, obj_dual;
  int32_t correctors;  /* centrality correctors accepted over the solve      */
  int32_t pad;
} orc_info;

typedef struct {
  int32_t iters;       /* Krylov iterations (all restarts)                   */
  int32_t converged;   /* explicit residual <= tol * ||f_hat||               */
  int32_t restarts;
  int32_t breakdown;
  double res0;         /* ||f_hat||                                           */
  double res;          /* explicit ||f_hat - A_hat dw|| at exit               */
} orc_krylov_info;

/* Multicolor ordering (greedy first fit over rows in decreasing priority
 * pi(i) = splitmix64(seed ^ i), ties broken by lower i).  Rows conflict when
 * they share a column.  Outputs color[m], perm[m] (rows sorted by color, then
 * by row index) and color_ptr[n_colors+1] (needs room for m+1 entries).
 * Returns n_colors, or -1 on allocation failure. */
int32_t orc_color_rows(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       uint64_t seed, int32_t *color, int32_t *perm, int32_t *color_ptr);

/* splitmix64 of x (published constants of the SplitMix64 generator). */
uint64_t orc_splitmix64(uint64_t x);

/* Row scaling of Sec. 3.5: d_j = sqrt(d2_j), rho_i = ||(A D)_i||_2,
 * ahat_ij = a_ij d_j / rho_i. */
void orc_scale_rows(int32_t m, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                    const double *d2, double *ahat, double *rho);

/* NE-SSOR (Algorithm 5): z = C^<ell> g (z[m]) and u = A^T z (u[n]) for the
 * matrix given in CSR; rows are visited in the order perm (forward: colors
 * ascending, rows ascending; backward: the exact reverse). */
void orc_nessor(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                const double *a, const int32_t *perm, const double *g, int32_t ell, double omega,
                double *z, double *u);

/* NE-SOR (Algorithm 6): z = B^<ell> g in R^n, plus the row-space shadow
 * y[m] (sum of the row corrections d_i) with z = A^T y. */
void orc_nesor(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
               const double *a, const int32_t *perm, const double *g, int32_t ell, double omega,
               double *z, double *y);

/* Krylov solve of min ||dw|| s.t. A dw = f on an already scaled matrix.
 * method: ORC_MRNE (Alg. 3, NE-SSOR), ORC_CGNE (Alg. 2, NE-SSOR) or
 * ORC_ABGMRES (Alg. 4, NE-SOR).  Outputs dw[n] and the row-space dy[m] with
 * dw = A^T dy.  Returns 0. */
int32_t orc_krylov(int32_t method, int32_t m, int32_t n, const int64_t *row_ptr,
                   const int32_t *col_idx, const double *a, const int32_t *perm, const double *f,
                   int32_t ell, double omega, double tol, int32_t maxit, double *dw, double *dy,
                   orc_krylov_info *info, double *res_hist /* may be NULL, maxit+1 */);

/* Search-direction solve of Sec. 2.2: A diag(d2) A^T dy = f through the
 * row-scaled w-form.  dw = diag(sqrt(d2)) A^T dy is the minimum-norm solution.
 * perm is the multicolor order of A's rows. */
int32_t orc_ne_solve(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *val, const int32_t *perm, const double *d2, const double *f,
                     int32_t ell, double omega, int32_t method, double tol, int32_t maxit,
                     double *dy, double *dw, orc_krylov_info *info);

/* NR-SOR inner iterations for min ||A^T y - c|| (A in CSR, rows = the columns
 * of A^T, visited in the order perm): y[m] = B^<ell> c. */
void orc_nrsor(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
               const double *a, const int32_t *perm, const double *c, int32_t ell, double omega,
               double *y);

/* BA-GMRES preconditioned by NR-SOR on min ||A^T dy - r|| for an already
 * scaled A (the corrector stage in least-squares form, Sec. 3.2): dy[m],
 * dw[n] = A^T dy.  info->res is the explicit ||A r - A dw||. */
int32_t orc_ls_krylov(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                      const double *a, const int32_t *perm, const double *r, int32_t ell,
                      double omega, double tol, int32_t maxit, double *dw, double *dy,
                      orc_krylov_info *info);

/* The corrector-stage least-squares problem min ||diag(sqrt(d2)) A^T dy - r||
 * through the row scaling of Sec. 3.5 and BA-GMRES; dw = diag(sqrt(d2)) A^T dy
 * is the minimum-norm solution of A diag(sqrt(d2)) dw = A diag(sqrt(d2)) r. */
int32_t orc_ls_solve(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *val, const int32_t *perm, const double *d2, const double *r,
                     int32_t ell, double omega, double tol, int32_t maxit, double *dy, double *dw,
                     orc_krylov_info *info);

void orc_default_options(orc_options *o);

/* Interior-point method (Algorithm 1 with the w-recurrence of Sec. 2.2).
 * x[n], y[m], s[n] outputs.  trace (may be NULL) receives ORC_TRACE_COLS
 * doubles per iteration k < max_ipm, describing the step from iterate k:
 * Gamma, mu, pinf, dinf, eps_in, Krylov iterations (predictor), Krylov
 * iterations (corrector), alpha_p, alpha_d (accepted, after backtracking),
 * sigma, mu_af (0 when the affine direction was taken), alpha_p and alpha_d
 * of the affine direction, the backtracking factor tau, 1 if a Krylov solve
 * of the step did not converge, and the relative gap of iterate k. */
#define ORC_TRACE_COLS 16
int32_t orc_lp_solve(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *val, const double *b, const double *c, const orc_options *opt,
                     double *x, double *y, double *s, orc_info *info, double *trace);

#ifdef __cplusplus
}
#endif
#endif
