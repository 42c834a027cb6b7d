/*
 * lpk_oracle.c -- plain FP64 CPU oracle of arXiv:1604.07491 (Cui, Morikuni,
 * Tsuchiya, Hayami).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke
 * check and the CPU baseline of the benchmark, never by the product path.
 *
 * Everything here is the paper's arithmetic written out in the order the paper
 * states it, single-threaded, with no blocking or fusion:
 *   Sec. 3.5        row scaling                        -> orc_scale_rows
 *   Algorithm 5     NE-SSOR inner iterations           -> orc_nessor
 *   Algorithm 6     NE-SOR inner iterations            -> orc_nesor
 *   Algorithm 2     CGNE preconditioned by inner its   -> cgne_core
 *   Algorithm 3     MRNE preconditioned by inner its   -> mrne_core
 *   Algorithm 4     AB-GMRES preconditioned by NE-SOR  -> abgmres_core
 *   Sec. 2.2        w-form of the normal equations     -> orc_ne_solve
 *   Sec. 3.2        BA-GMRES for the corrector stage,  -> orc_ls_solve, bagmres_core
 *                   least-squares form (eq. ba_ne), NR-SOR inner iterations
 *                                                      -> orc_nrsor
 *   Algorithm 1     Mehrotra predictor-corrector,      -> orc_lp_solve
 *                   Eq. (steplength), sigma rule, Gamma (Eq. errorMeasureDef),
 *                   centrality backtracking, eps_in schedule of Sec. 4.2
 *   Sec. 4.3 / 5    multiple centrality correctors    -> ipm_core (max_correctors)
 *                   (the multi-corrector framework the paper names as the
 *                   way to fewer interior-point iterations; Gondzio 1996)
 * The multicolor row order (rows of one color share no column) is not in the
 * paper, which sweeps rows in natural order; the oracle applies the same
 * order as the GPU so that sweeps can be compared element by element.
 * Readings of garbled or silent passages are marked "reading:".
 */
#include "lpk_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small dense helpers (plain loops)                                          */
/* ------------------------------------------------------------------------ */
static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}
static double nrm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }
static void axpy(int64_t n, double al, const double *x, double *y) {
  for (int64_t i = 0; i < n; ++i) y[i] += al * x[i];
}
/* t = A p (CSR) */
static void spmv(int32_t m, const int64_t *rp, const int32_t *ci, const double *a, const double *p,
                 double *t) {
  for (int32_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += a[k] * p[ci[k]];
    t[i] = s;
  }
}
/* w = A^T y (CSR, scattered) */
static void spmv_t(int32_t m, int32_t n, const int64_t *rp, const int32_t *ci, const double *a,
                   const double *y, double *w) {
  for (int32_t j = 0; j < n; ++j) w[j] = 0.0;
  for (int32_t i = 0; i < m; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) w[ci[k]] += a[k] * y[i];
}
static double *dalloc(int64_t n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

/* ------------------------------------------------------------------------ */
/* multicolor ordering                                                        */
/* ------------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct { uint64_t key; int32_t row; } prio_t;
static int prio_cmp(const void *pa, const void *pb) {
  const prio_t *a = (const prio_t *)pa, *b = (const prio_t *)pb;
  if (a->key != b->key) return a->key > b->key ? -1 : 1;   /* larger priority first */
  return a->row < b->row ? -1 : (a->row > b->row);        /* then lower row first  */
}

int32_t orc_color_rows(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       uint64_t seed, int32_t *color, int32_t *perm, int32_t *color_ptr) {
  int64_t nnz = row_ptr[m];
  /* column -> rows pattern */
  int64_t *cp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t *ri = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
  prio_t *order = (prio_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(prio_t));
  int32_t *stamp = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
  if (!cp || !ri || !order || !stamp) { free(cp); free(ri); free(order); free(stamp); return -1; }
  for (int64_t k = 0; k < nnz; ++k) cp[col_idx[k] + 1]++;
  for (int32_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
  {
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int32_t j = 0; j < n; ++j) fill[j] = cp[j];
    for (int32_t i = 0; i < m; ++i)
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) ri[fill[col_idx[k]]++] = i;
    free(fill);
  }
  for (int32_t i = 0; i < m; ++i) {
    order[i].key = orc_splitmix64(seed ^ (uint64_t)(uint32_t)i);
    order[i].row = i;
    color[i] = -1;
  }
  qsort(order, (size_t)m, sizeof(prio_t), prio_cmp);
  for (int32_t c = 0; c <= m; ++c) stamp[c] = -1;
  int32_t n_colors = 0;
  /* greedy first fit: each row takes the smallest color not used by an
     already colored row that shares a column with it */
  for (int32_t t = 0; t < m; ++t) {
    int32_t r = order[t].row;
    for (int64_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
      int32_t j = col_idx[k];
      for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
        int32_t c = color[ri[q]];
        if (c >= 0) stamp[c] = r;
      }
    }
    int32_t c = 0;
    while (stamp[c] == r) ++c;
    color[r] = c;
    if (c + 1 > n_colors) n_colors = c + 1;
  }
  /* perm: rows sorted by color, then by row index */
  for (int32_t c = 0; c <= n_colors; ++c) color_ptr[c] = 0;
  for (int32_t i = 0; i < m; ++i) color_ptr[color[i] + 1]++;
  for (int32_t c = 0; c < n_colors; ++c) color_ptr[c + 1] += color_ptr[c];
  {
    int32_t *fill = (int32_t *)malloc((size_t)(n_colors > 0 ? n_colors : 1) * sizeof(int32_t));
    for (int32_t c = 0; c < n_colors; ++c) fill[c] = color_ptr[c];
    for (int32_t i = 0; i < m; ++i) perm[fill[color[i]]++] = i;
    free(fill);
  }
  free(cp); free(ri); free(order); free(stamp);
  return n_colors;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.5 row scaling                                                       */
/* ------------------------------------------------------------------------ */
void orc_scale_rows(int32_t m, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                    const double *d2, double *ahat, double *rho) {
  for (int32_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      double e = val[k] * sqrt(d2[col_idx[k]]);   /* entry of A D, D = (X S^-1)^(1/2) */
      s += e * e;
    }
    rho[i] = sqrt(s);                               /* D_cal(i,i) = ||alpha_i||_2 */
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
      ahat[k] = s > 0.0 ? val[k] * sqrt(d2[col_idx[k]]) / rho[i] : 0.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Algorithms 5 and 6: inner iterations                                       */
/* ------------------------------------------------------------------------ */
static double *row_norms2(int32_t m, const int64_t *rp, const double *a) {
  double *r = dalloc(m);
  for (int32_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += a[k] * a[k];
    r[i] = s;
  }
  return r;
}

/* one row update of Algorithm 5: d_i = omega (g_i - (alpha_i, u)) / ||alpha_i||^2,
   z_i += d_i, u += d_i alpha_i */
static void ssor_row(int32_t i, const int64_t *rp, const int32_t *ci, const double *a,
                     const double *nr2, const double *g, double omega, double *z, double *u) {
  if (nr2[i] == 0.0) return;
  double s = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += a[k] * u[ci[k]];
  double d = omega * (g[i] - s) / nr2[i];
  z[i] += d;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) u[ci[k]] += d * a[k];
}

void orc_nessor(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                const double *a, const int32_t *perm, const double *g, int32_t ell, double omega,
                double *z, double *u) {
  double *nr2 = row_norms2(m, row_ptr, a);
  for (int32_t i = 0; i < m; ++i) z[i] = 0.0;
  for (int32_t j = 0; j < n; ++j) u[j] = 0.0;
  for (int32_t k = 0; k < ell; ++k) {
    for (int32_t p = 0; p < m; ++p) ssor_row(perm[p], row_ptr, col_idx, a, nr2, g, omega, z, u);
    for (int32_t p = m - 1; p >= 0; --p) ssor_row(perm[p], row_ptr, col_idx, a, nr2, g, omega, z, u);
  }
  free(nr2);
}

void orc_nesor(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
               const double *a, const int32_t *perm, const double *g, int32_t ell, double omega,
               double *z, double *y) {
  double *nr2 = row_norms2(m, row_ptr, a);
  for (int32_t i = 0; i < m; ++i) y[i] = 0.0;
  for (int32_t j = 0; j < n; ++j) z[j] = 0.0;
  /* Algorithm 6: d_i = omega (g_i - (alpha_i, z)) / ||alpha_i||^2, z += d_i alpha_i;
     y accumulates d_i so that z = A^T y (used to recover dy without a product) */
  for (int32_t k = 0; k < ell; ++k)
    for (int32_t p = 0; p < m; ++p) ssor_row(perm[p], row_ptr, col_idx, a, nr2, g, omega, y, z);
  free(nr2);
}

/* NR-SOR: the SOR method for the normal equations of the first kind
   A A^T y = A c, i.e. for min ||A^T y - c|| (the columns of A^T are the rows
   of A), ell forward sweeps from y = 0 with the residual r = c - A^T y kept
   explicitly: d_i = omega (alpha_i, r) / ||alpha_i||^2, y_i += d_i,
   r -= d_i alpha_i.  Returns y = B c, the inner-iteration left preconditioner
   of BA-GMRES. */
void orc_nrsor(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
               const double *a, const int32_t *perm, const double *c, int32_t ell, double omega,
               double *y) {
  double *nr2 = row_norms2(m, row_ptr, a);
  double *r = dalloc(n);
  memcpy(r, c, sizeof(double) * (size_t)n);
  for (int32_t i = 0; i < m; ++i) y[i] = 0.0;
  for (int32_t k = 0; k < ell; ++k)
    for (int32_t p = 0; p < m; ++p) {
      int32_t i = perm[p];
      if (nr2[i] == 0.0) continue;
      double t = 0.0;
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) t += a[q] * r[col_idx[q]];
      double d = omega * t / nr2[i];
      y[i] += d;
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) r[col_idx[q]] -= d * a[q];
    }
  free(r);
  free(nr2);
}

/* ------------------------------------------------------------------------ */
/* Krylov solvers on the scaled system A dw = f (A = A_hat here)              */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t m, n;
  const int64_t *rp;
  const int32_t *ci;
  const double *a;
  const int32_t *perm;
  int32_t ell;
  double omega;
} sys_t;

enum { EXIT_CONVERGED = 0, EXIT_MAXIT = 1, EXIT_BREAKDOWN = 2 };

/* Algorithm 3 (MRNE).  reading: the loop index starts at 0 and the updates are
   dw_{k+1} = dw_k + a_k p_k, gamma_{k+1} = ||q_{k+1}||^2, beta_k = gamma_{k+1}/gamma_k,
   p_{k+1} = q_{k+1} + beta_k p_k (the printed indices are inconsistent).
   Row-space shadows (pt, qt, vt) follow p, q, v so that dw = A^T dy holds. */
static int mrne_core(const sys_t *S, const double *g0, double target, int32_t maxit, double *dw,
                     double *dy, int32_t *iters, double *hist, int32_t hist_off) {
  int32_t m = S->m, n = S->n;
  double *g = dalloc(m), *t = dalloc(m), *qt = dalloc(m), *pt = dalloc(m), *vt = dalloc(m);
  double *q = dalloc(n), *p = dalloc(n), *v = dalloc(n);
  memcpy(g, g0, sizeof(double) * (size_t)m);
  orc_nessor(m, n, S->rp, S->ci, S->a, S->perm, g, S->ell, S->omega, qt, q); /* q0 = A^T C g0 */
  memcpy(p, q, sizeof(double) * (size_t)n);
  memcpy(pt, qt, sizeof(double) * (size_t)m);
  double gamma = dot(n, q, q);
  int rc = EXIT_MAXIT;
  int32_t k = 0;
  double gn = nrm2(m, g);
  while (1) {
    if (gn <= target) { rc = EXIT_CONVERGED; break; }
    if (k >= maxit) { rc = EXIT_MAXIT; break; }
    spmv(m, S->rp, S->ci, S->a, p, t);                                         /* t = A p */
    orc_nessor(m, n, S->rp, S->ci, S->a, S->perm, t, S->ell, S->omega, vt, v); /* v = A^T C t */
    double vp = dot(n, v, p);
    if (!(vp > 0.0) || !(gamma > 0.0) || !isfinite(vp)) { rc = EXIT_BREAKDOWN; break; }
    double alpha = gamma / vp;
    axpy(n, alpha, p, dw);
    axpy(m, alpha, pt, dy);
    axpy(m, -alpha, t, g);
    axpy(n, -alpha, v, q);
    axpy(m, -alpha, vt, qt);
    double gamma1 = dot(n, q, q);
    double beta = gamma1 / gamma;
    gamma = gamma1;
    for (int32_t j = 0; j < n; ++j) p[j] = q[j] + beta * p[j];
    for (int32_t i = 0; i < m; ++i) pt[i] = qt[i] + beta * pt[i];
    ++k;
    gn = nrm2(m, g);
    if (hist) hist[hist_off + k] = gn;
  }
  *iters = k;
  free(g); free(t); free(qt); free(pt); free(vt); free(q); free(p); free(v);
  return rc;
}

/* Algorithm 2 (CGNE).  reading: alpha on the second line is alpha_k.  The
   iterate with the smallest recurrence residual is kept for the failure case
   (Sec. 4.2: the solution with the minimum residual norm is adopted). */
static int cgne_core(const sys_t *S, const double *g0, double target, int32_t maxit, double *dw,
                     double *dy, int32_t *iters, double *hist, int32_t hist_off) {
  int32_t m = S->m, n = S->n;
  double *g = dalloc(m), *z = dalloc(m), *qt = dalloc(m), *Aq = dalloc(m), *bdy = dalloc(m);
  double *u = dalloc(n), *q = dalloc(n), *bdw = dalloc(n);
  double *dw0 = dalloc(n), *dy0 = dalloc(m);
  memcpy(dw0, dw, sizeof(double) * (size_t)n);
  memcpy(dy0, dy, sizeof(double) * (size_t)m);
  memcpy(g, g0, sizeof(double) * (size_t)m);
  orc_nessor(m, n, S->rp, S->ci, S->a, S->perm, g, S->ell, S->omega, z, u); /* z0 = C g0, u0 = A^T z0 */
  memcpy(q, u, sizeof(double) * (size_t)n);
  memcpy(qt, z, sizeof(double) * (size_t)m);
  double gamma = dot(m, g, z);
  int rc = EXIT_MAXIT;
  int32_t k = 0;
  double gn = nrm2(m, g), best = gn;
  memcpy(bdw, dw, sizeof(double) * (size_t)n);
  memcpy(bdy, dy, sizeof(double) * (size_t)m);
  while (1) {
    if (gn <= target) { rc = EXIT_CONVERGED; break; }
    if (k >= maxit) { rc = EXIT_MAXIT; break; }
    double qq = dot(n, q, q);
    if (!(qq > 0.0) || !(gamma > 0.0) || !isfinite(gamma)) { rc = EXIT_BREAKDOWN; break; }
    double alpha = gamma / qq;
    spmv(m, S->rp, S->ci, S->a, q, Aq);
    axpy(n, alpha, q, dw);
    axpy(m, alpha, qt, dy);
    axpy(m, -alpha, Aq, g);
    orc_nessor(m, n, S->rp, S->ci, S->a, S->perm, g, S->ell, S->omega, z, u);
    double gamma1 = dot(m, g, z);
    double beta = gamma1 / gamma;
    gamma = gamma1;
    for (int32_t j = 0; j < n; ++j) q[j] = u[j] + beta * q[j];
    for (int32_t i = 0; i < m; ++i) qt[i] = z[i] + beta * qt[i];
    ++k;
    gn = nrm2(m, g);
    if (hist) hist[hist_off + k] = gn;
    if (gn < best) {
      best = gn;
      memcpy(bdw, dw, sizeof(double) * (size_t)n);
      memcpy(bdy, dy, sizeof(double) * (size_t)m);
    }
  }
  if (rc != EXIT_CONVERGED) {
    memcpy(dw, bdw, sizeof(double) * (size_t)n);
    memcpy(dy, bdy, sizeof(double) * (size_t)m);
  }
  *iters = k;
  free(g); free(z); free(qt); free(Aq); free(bdy); free(u); free(q); free(bdw); free(dw0); free(dy0);
  return rc;
}

/* Algorithm 4 (AB-GMRES, no restart, modified Gram-Schmidt, Givens rotations
   for the (k+1) x k least-squares problem).  reading: v_1 = g_0 / beta. */
static int abgmres_core(const sys_t *S, const double *g0, double target, int32_t maxit, double *dw,
                        double *dy, int32_t *iters, double *hist, int32_t hist_off) {
  int32_t m = S->m, n = S->n;
  int32_t cap = 16;
  double *V = (double *)malloc(sizeof(double) * (size_t)m * (size_t)(cap + 1));
  double *H = (double *)calloc((size_t)(cap + 1) * (size_t)cap, sizeof(double)); /* H[i + j*(cap+1)] */
  double *cs = dalloc(cap), *sn = dalloc(cap), *gh = dalloc(cap + 1);
  double *z = dalloc(n), *yv = dalloc(m), *u = dalloc(m);
  double beta = nrm2(m, g0);
  int rc = EXIT_MAXIT;
  int32_t k = 0;
  for (int32_t i = 0; i < m; ++i) V[i] = g0[i] / beta;
  gh[0] = beta;
  double res = beta;
  while (1) {
    if (res <= target) { rc = EXIT_CONVERGED; break; }
    if (k >= maxit) { rc = EXIT_MAXIT; break; }
    if (k + 1 > cap) { /* grow storage */
      int32_t nc = cap * 2;
      double *V2 = (double *)realloc(V, sizeof(double) * (size_t)m * (size_t)(nc + 1));
      double *H2 = (double *)calloc((size_t)(nc + 1) * (size_t)nc, sizeof(double));
      for (int32_t j = 0; j < cap; ++j)
        for (int32_t i = 0; i <= cap; ++i) H2[i + (size_t)j * (nc + 1)] = H[i + (size_t)j * (cap + 1)];
      free(H);
      V = V2; H = H2;
      cs = (double *)realloc(cs, sizeof(double) * (size_t)nc);
      sn = (double *)realloc(sn, sizeof(double) * (size_t)nc);
      gh = (double *)realloc(gh, sizeof(double) * (size_t)(nc + 1));
      cap = nc;
    }
    double *vk = V + (size_t)k * m;
    orc_nesor(m, n, S->rp, S->ci, S->a, S->perm, vk, S->ell, S->omega, z, yv); /* z_k = B v_k */
    spmv(m, S->rp, S->ci, S->a, z, u);                                            /* u_k = A z_k */
    double *hk = H + (size_t)k * (cap + 1);
    for (int32_t i = 0; i <= k; ++i) {                     /* modified Gram-Schmidt */
      double *vi = V + (size_t)i * m;
      hk[i] = dot(m, u, vi);
      axpy(m, -hk[i], vi, u);
    }
    hk[k + 1] = nrm2(m, u);
    double hnext = hk[k + 1];
    for (int32_t i = 0; i < k; ++i) {                      /* previous rotations */
      double a = hk[i], b = hk[i + 1];
      hk[i] = cs[i] * a + sn[i] * b;
      hk[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double r = hypot(hk[k], hk[k + 1]);
    if (!(r > 0.0) || !isfinite(r)) { rc = EXIT_BREAKDOWN; break; }
    cs[k] = hk[k] / r;
    sn[k] = hk[k + 1] / r;
    hk[k] = r;
    hk[k + 1] = 0.0;
    gh[k + 1] = -sn[k] * gh[k];
    gh[k] = cs[k] * gh[k];
    res = fabs(gh[k + 1]);
    ++k;
    if (hist) hist[hist_off + k] = res;
    if (hnext == 0.0) { rc = EXIT_CONVERGED; break; }      /* lucky breakdown: exact */
    double *vn = V + (size_t)k * m;
    for (int32_t i = 0; i < m; ++i) vn[i] = u[i] / hnext;
  }
  if (k > 0) {
    /* p_k = argmin ||beta e1 - H_k p||: back substitution on the rotated H */
    double *pk = dalloc(k);
    for (int32_t i = k - 1; i >= 0; --i) {
      double s = gh[i];
      for (int32_t j = i + 1; j < k; ++j) s -= H[i + (size_t)j * (cap + 1)] * pk[j];
      pk[i] = s / H[i + (size_t)i * (cap + 1)];
    }
    double *qv = dalloc(m);                                 /* q_k = V_k p_k */
    for (int32_t j = 0; j < k; ++j) axpy(m, pk[j], V + (size_t)j * m, qv);
    orc_nesor(m, n, S->rp, S->ci, S->a, S->perm, qv, S->ell, S->omega, z, yv); /* z' = B q_k */
    axpy(n, 1.0, z, dw);
    axpy(m, 1.0, yv, dy);
    free(pk); free(qv);
  }
  *iters = k;
  free(V); free(H); free(cs); free(sn); free(gh); free(z); free(yv); free(u);
  return rc;
}

#define ORC_MAX_RESTARTS 3

int32_t orc_krylov(int32_t method, int32_t m, int32_t n, const int64_t *row_ptr,
                   const int32_t *col_idx, const double *a, const int32_t *perm, const double *f,
                   int32_t ell, double omega, double tol, int32_t maxit, double *dw, double *dy,
                   orc_krylov_info *info, double *res_hist) {
  sys_t S = {m, n, row_ptr, col_idx, a, perm, ell, omega};
  double *r = dalloc(m), *t = dalloc(m);
  for (int32_t j = 0; j < n; ++j) dw[j] = 0.0;
  for (int32_t i = 0; i < m; ++i) dy[i] = 0.0;
  double res0 = nrm2(m, f);
  double target = tol * res0;
  memset(info, 0, sizeof(*info));
  info->res0 = res0;
  if (res_hist) res_hist[0] = res0;
  memcpy(r, f, sizeof(double) * (size_t)m);
  double res = res0;
  int32_t used = 0;
  int rc = EXIT_CONVERGED;
  /* reading (Sec. 4.2 stopping test): the recurrence residual ends the
     iteration, the explicit residual ||f - A dw|| decides convergence; a
     recurrence that claims convergence the explicit residual does not confirm
     is restarted from the current iterate (at most ORC_MAX_RESTARTS times). */
  for (int32_t rs = 0; rs <= ORC_MAX_RESTARTS; ++rs) {
    if (res <= target) { rc = EXIT_CONVERGED; break; }
    if (used >= maxit) { rc = EXIT_MAXIT; break; }
    int32_t it = 0;
    if (method == ORC_MRNE)
      rc = mrne_core(&S, r, target, maxit - used, dw, dy, &it, res_hist, used);
    else if (method == ORC_CGNE)
      rc = cgne_core(&S, r, target, maxit - used, dw, dy, &it, res_hist, used);
    else
      rc = abgmres_core(&S, r, target, maxit - used, dw, dy, &it, res_hist, used);
    used += it;
    spmv(m, row_ptr, col_idx, a, dw, t);
    for (int32_t i = 0; i < m; ++i) r[i] = f[i] - t[i];
    res = nrm2(m, r);
    if (rc != EXIT_CONVERGED) break;
    if (res > target && rs < ORC_MAX_RESTARTS) info->restarts++;
  }
  info->iters = used;
  info->res = res;
  info->converged = res <= target;
  info->breakdown = rc == EXIT_BREAKDOWN;
  free(r); free(t);
  return 0;
}

int32_t orc_ne_solve(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *val, const int32_t *perm, const double *d2, const double *f,
                     int32_t ell, double omega, int32_t method, double tol, int32_t maxit,
                     double *dy, double *dw, orc_krylov_info *info) {
  int64_t nnz = row_ptr[m];
  double *ahat = dalloc(nnz), *rho = dalloc(m), *fh = dalloc(m), *dyh = dalloc(m);
  orc_scale_rows(m, row_ptr, col_idx, val, d2, ahat, rho);
  for (int32_t i = 0; i < m; ++i) fh[i] = rho[i] > 0.0 ? f[i] / rho[i] : 0.0;  /* f_hat = D_cal^-1 f */
  orc_krylov(method, m, n, row_ptr, col_idx, ahat, perm, fh, ell, omega, tol, maxit, dw, dyh, info,
             NULL);
  /* A_hat^T dy_hat = A^T D D_cal^-1 dy_hat, so dy = D_cal^-1 dy_hat */
  for (int32_t i = 0; i < m; ++i) dy[i] = rho[i] > 0.0 ? dyh[i] / rho[i] : 0.0;
  free(ahat); free(rho); free(fh); free(dyh);
  return 0;
}

/* BA-GMRES (left-preconditioned GMRES) on min ||A^T y - r0||: GMRES applied
   to B A^T y = B r0 with B = NR-SOR, in m-space, from y = 0 (the caller
   passes r0 = the residual of its current iterate), modified Gram-Schmidt and
   Givens rotations as in Algorithm 4.  Stops when the preconditioned residual
   estimate |g_{k+1}| <= ratio * ||B r0||.  Adds V_k p_k to y. */
static int bagmres_core(const sys_t *S, const double *r0, double ratio, int32_t maxit, double *y,
                        int32_t *iters) {
  int32_t m = S->m, n = S->n;
  int32_t cap = 16;
  double *V = (double *)malloc(sizeof(double) * (size_t)m * (size_t)(cap + 1));
  double *H = (double *)calloc((size_t)(cap + 1) * (size_t)cap, sizeof(double));
  double *cs = dalloc(cap), *sn = dalloc(cap), *gh = dalloc(cap + 1);
  double *w = dalloc(m), *t = dalloc(n);
  orc_nrsor(m, n, S->rp, S->ci, S->a, S->perm, r0, S->ell, S->omega, w);   /* B r0 */
  double beta = nrm2(m, w);
  int rc = EXIT_MAXIT;
  int32_t k = 0;
  if (beta == 0.0) { rc = EXIT_CONVERGED; goto done; }
  for (int32_t i = 0; i < m; ++i) V[i] = w[i] / beta;
  gh[0] = beta;
  double target = ratio * beta, res = beta;
  while (1) {
    if (res <= target) { rc = EXIT_CONVERGED; break; }
    if (k >= maxit) { rc = EXIT_MAXIT; break; }
    if (k + 1 > cap) {
      int32_t nc = cap * 2;
      double *V2 = (double *)realloc(V, sizeof(double) * (size_t)m * (size_t)(nc + 1));
      double *H2 = (double *)calloc((size_t)(nc + 1) * (size_t)nc, sizeof(double));
      for (int32_t j = 0; j < cap; ++j)
        for (int32_t i = 0; i <= cap; ++i) H2[i + (size_t)j * (nc + 1)] = H[i + (size_t)j * (cap + 1)];
      free(H);
      V = V2; H = H2;
      cs = (double *)realloc(cs, sizeof(double) * (size_t)nc);
      sn = (double *)realloc(sn, sizeof(double) * (size_t)nc);
      gh = (double *)realloc(gh, sizeof(double) * (size_t)(nc + 1));
      cap = nc;
    }
    double *vk = V + (size_t)k * m;
    spmv_t(m, n, S->rp, S->ci, S->a, vk, t);                                /* A^T v_k */
    orc_nrsor(m, n, S->rp, S->ci, S->a, S->perm, t, S->ell, S->omega, w);  /* w = B A^T v_k */
    double *hk = H + (size_t)k * (cap + 1);
    for (int32_t i = 0; i <= k; ++i) {
      double *vi = V + (size_t)i * m;
      hk[i] = dot(m, w, vi);
      axpy(m, -hk[i], vi, w);
    }
    hk[k + 1] = nrm2(m, w);
    double hnext = hk[k + 1];
    for (int32_t i = 0; i < k; ++i) {
      double a = hk[i], b = hk[i + 1];
      hk[i] = cs[i] * a + sn[i] * b;
      hk[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double rr = hypot(hk[k], hk[k + 1]);
    if (!(rr > 0.0) || !isfinite(rr)) { rc = EXIT_BREAKDOWN; break; }
    cs[k] = hk[k] / rr;
    sn[k] = hk[k + 1] / rr;
    hk[k] = rr;
    hk[k + 1] = 0.0;
    gh[k + 1] = -sn[k] * gh[k];
    gh[k] = cs[k] * gh[k];
    res = fabs(gh[k + 1]);
    ++k;
    if (hnext == 0.0) { rc = EXIT_CONVERGED; break; }
    double *vn = V + (size_t)k * m;
    for (int32_t i = 0; i < m; ++i) vn[i] = w[i] / hnext;
  }
  if (k > 0) {
    double *pk = dalloc(k);
    for (int32_t i = k - 1; i >= 0; --i) {
      double sacc = gh[i];
      for (int32_t j = i + 1; j < k; ++j) sacc -= H[i + (size_t)j * (cap + 1)] * pk[j];
      pk[i] = sacc / H[i + (size_t)i * (cap + 1)];
    }
    for (int32_t j = 0; j < k; ++j) axpy(m, pk[j], V + (size_t)j * m, y);   /* y += V_k p_k */
    free(pk);
  }
done:
  *iters = k;
  free(V); free(H); free(cs); free(sn); free(gh); free(w); free(t);
  return rc;
}

int32_t orc_ls_krylov(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                      const double *a, const int32_t *perm, const double *r, int32_t ell,
                      double omega, double tol, int32_t maxit, double *dw, double *dy,
                      orc_krylov_info *info) {
  sys_t S = {m, n, row_ptr, col_idx, a, perm, ell, omega};
  double *f = dalloc(m), *c = dalloc(n), *g = dalloc(m);
  /* the equivalent normal equations A A^T dy = A r: f = A r, and the explicit
     residual ||f - A dw|| with dw = A^T dy, as for the other solvers */
  spmv(m, row_ptr, col_idx, a, r, f);
  double res0 = nrm2(m, f), target = tol * res0;
  memset(info, 0, sizeof(*info));
  info->res0 = res0;
  for (int32_t i = 0; i < m; ++i) dy[i] = 0.0;
  for (int32_t j = 0; j < n; ++j) dw[j] = 0.0;
  double res = res0;
  int32_t used = 0;
  int rc = EXIT_CONVERGED;
  /* reading (as for the other solvers): the recurrence ends the iteration, the
     explicit residual decides convergence, at most ORC_MAX_RESTARTS restarts
     from the current iterate.  The preconditioned residual must shrink by the
     factor the explicit residual still has to shrink. */
  for (int32_t rs = 0; rs <= ORC_MAX_RESTARTS; ++rs) {
    if (res <= target) { rc = EXIT_CONVERGED; break; }
    if (used >= maxit) { rc = EXIT_MAXIT; break; }
    for (int32_t j = 0; j < n; ++j) c[j] = r[j] - dw[j];      /* residual of the LS problem */
    int32_t it = 0;
    rc = bagmres_core(&S, c, target / res, maxit - used, dy, &it);
    used += it;
    spmv_t(m, n, row_ptr, col_idx, a, dy, dw);                /* dw = A^T dy */
    spmv(m, row_ptr, col_idx, a, dw, g);
    for (int32_t i = 0; i < m; ++i) g[i] = f[i] - g[i];
    res = nrm2(m, g);
    if (rc != EXIT_CONVERGED) break;
    if (res > target && rs < ORC_MAX_RESTARTS) info->restarts++;
  }
  info->iters = used;
  info->res = res;
  info->converged = res <= target;
  info->breakdown = rc == EXIT_BREAKDOWN;
  free(f); free(c); free(g);
  return 0;
}

int32_t orc_ls_solve(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *val, const int32_t *perm, const double *d2, const double *r,
                     int32_t ell, double omega, double tol, int32_t maxit, double *dy, double *dw,
                     orc_krylov_info *info) {
  int64_t nnz = row_ptr[m];
  double *ahat = dalloc(nnz), *rho = dalloc(m), *dyh = dalloc(m);
  orc_scale_rows(m, row_ptr, col_idx, val, d2, ahat, rho);
  /* A D = D_cal A_hat, so (A D)^T dy = A_hat^T (D_cal dy): solve for dy_hat = D_cal dy */
  orc_ls_krylov(m, n, row_ptr, col_idx, ahat, perm, r, ell, omega, tol, maxit, dw, dyh, info);
  for (int32_t i = 0; i < m; ++i) dy[i] = rho[i] > 0.0 ? dyh[i] / rho[i] : 0.0;
  free(ahat); free(rho); free(dyh);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: Mehrotra predictor-corrector with the w-recurrence            */
/* ------------------------------------------------------------------------ */
void orc_default_options(orc_options *o) {
  memset(o, 0, sizeof(*o));
  o->tol = 1e-8;        /* eps_out, Eq. (errorMeasure) */
  o->eta = 0.9995;      /* reading: eta in [0.9, 1) is not fixed by the paper */
  o->phi = 1e-5;        /* centrality bound */
  o->sigma_max = 0.208; /* LIPSOL value quoted by the paper */
  o->eps_in0 = 1e-6;    /* initial Krylov tolerance */
  o->omega = 1.0;
  o->start_tol = 1e-10;
  o->backtrack = 0.95;  /* reading: "gradually reduce" -> common factor 0.95 */
  o->max_ipm = 99;
  o->max_krylov = 0;    /* -> m */
  o->inner_sweeps = 1;
  o->method = ORC_MRNE;
  o->color_seed = 0x5EEDULL;
  o->corrector_ba = 0;
  o->max_correctors = 0;
}

static double step_len(int32_t n, const double *x, const double *dx, double eta) {
  /* Eq. (steplength): min(1, eta * min_{dx_i < 0} -x_i / dx_i) */
  double a = INFINITY;
  for (int32_t i = 0; i < n; ++i)
    if (dx[i] < 0.0) {
      double r = -x[i] / dx[i];
      if (r < a) a = r;
    }
  a = eta * a;
  return a < 1.0 ? a : 1.0;
}

static double clamp_eps(double e) { return e < 1e-14 ? 1e-14 : (e > 1e-4 ? 1e-4 : e); }

/* IPM on a problem without empty rows or columns */
static int32_t ipm_core(int32_t m, int32_t n, const int64_t *rp, const int32_t *ci, const double *val,
                        const double *b, const double *c, const orc_options *opt, double *x,
                        double *y, double *s, orc_info *info, double *trace) {
  int32_t *color = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t *cptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
  info->n_colors = orc_color_rows(m, n, rp, ci, opt->color_seed, color, perm, cptr);
  int32_t maxit = opt->max_krylov > 0 ? opt->max_krylov : m;
  int32_t ell = opt->inner_sweeps, meth = opt->method;
  double om = opt->omega;

  double *d2 = dalloc(n), *d = dalloc(n), *rd = dalloc(n), *rp_ = dalloc(m), *f = dalloc(m);
  double *dwa = dalloc(n), *dya = dalloc(m), *dxa = dalloc(n), *dsa = dalloc(n);
  double *dwc = dalloc(n), *dyc = dalloc(m), *dx = dalloc(n), *ds = dalloc(n), *dy = dalloc(m);
  double *h = dalloc(n), *tmpm = dalloc(m), *tmpn = dalloc(n);
  orc_krylov_info ki;

  /* starting point.  reading: the paper defers to LIPSOL without stating the
     procedure; this uses Mehrotra's rule: x~ = min-norm solution of Ax = b,
     y~ solves A A^T y = A c, s~ = c - A^T y~, then the two shifts. */
  for (int32_t j = 0; j < n; ++j) d2[j] = 1.0;
  orc_ne_solve(m, n, rp, ci, val, perm, d2, b, ell, om, meth, opt->start_tol, maxit, tmpm, x, &ki);
  info->krylov_iters_total += ki.iters;
  spmv(m, rp, ci, val, c, f);
  orc_ne_solve(m, n, rp, ci, val, perm, d2, f, ell, om, meth, opt->start_tol, maxit, y, tmpn, &ki);
  info->krylov_iters_total += ki.iters;
  for (int32_t j = 0; j < n; ++j) s[j] = c[j] - tmpn[j];   /* tmpn = A^T y (w with D = I) */
  {
    double mx = INFINITY, ms = INFINITY;
    for (int32_t j = 0; j < n; ++j) { if (x[j] < mx) mx = x[j]; if (s[j] < ms) ms = s[j]; }
    double sx = fmax(-1.5 * mx, 0.0), ss = fmax(-1.5 * ms, 0.0);
    for (int32_t j = 0; j < n; ++j) { x[j] += sx; s[j] += ss; }
    double xs = dot(n, x, s), sumx = 0.0, sums = 0.0;
    for (int32_t j = 0; j < n; ++j) { sumx += x[j]; sums += s[j]; }
    double hx = sums > 0.0 ? 0.5 * xs / sums : 0.0, hs = sumx > 0.0 ? 0.5 * xs / sumx : 0.0;
    for (int32_t j = 0; j < n; ++j) {
      x[j] += hx; s[j] += hs;
      if (!(x[j] > 0.0)) x[j] = 1.0;
      if (!(s[j] > 0.0)) s[j] = 1.0;
    }
  }

  double nb = fmax(nrm2(m, b), 1.0), nc = fmax(nrm2(n, c), 1.0);
  double eps_in = opt->eps_in0;
  int32_t status = ORC_MAX_IPM_ITER;
  int32_t k;
  int failed_prev = 0;
  for (k = 0; k <= opt->max_ipm; ++k) {
    /* residuals of Eq. (SE1) and Gamma of Eq. (errorMeasureDef) */
    spmv(m, rp, ci, val, x, tmpm);
    for (int32_t i = 0; i < m; ++i) rp_[i] = b[i] - tmpm[i];
    spmv_t(m, n, rp, ci, val, y, tmpn);
    for (int32_t j = 0; j < n; ++j) rd[j] = c[j] - tmpn[j] - s[j];
    double mu = dot(n, x, s) / n;
    double pinf = nrm2(m, rp_) / nb, dinf = nrm2(n, rd) / nc;
    double Gam = fmax(mu, fmax(pinf, dinf));
    double pobj = dot(n, c, x), dobj = dot(m, b, y);
    double gap = fabs(pobj - dobj) / (1.0 + fabs(pobj));
    info->gamma = Gam; info->rel_gap = gap; info->pinf = pinf; info->dinf = dinf; info->mu = mu;
    info->obj_primal = pobj; info->obj_dual = dobj;
    info->ipm_iters = k;
    if (!isfinite(Gam)) { status = ORC_DIVERGED; break; }
    if (Gam <= opt->tol && gap <= opt->tol) { status = ORC_OK; break; }
    if (k == opt->max_ipm) { status = ORC_MAX_IPM_ITER; break; }
    /* eps_in schedule (Sec. 4.2); reading: unchanged while log10 Gamma > 1 */
    if (k > 0) {
      if (failed_prev) eps_in *= 1.5;
      double lg = log10(Gam);
      if (lg <= -3.0) eps_in *= 0.375;
      else if (lg <= 1.0) eps_in *= 0.75;
      eps_in = clamp_eps(eps_in);
    }
    int failed = 0;
    for (int32_t j = 0; j < n; ++j) { d2[j] = x[j] / s[j]; d[j] = sqrt(d2[j]); }

    /* predictor: f_af = b + A S^-1 X r_d, solve for dw_af, then Eqs. (aff2), (aff3) */
    for (int32_t j = 0; j < n; ++j) tmpn[j] = d2[j] * rd[j];
    spmv(m, rp, ci, val, tmpn, f);
    for (int32_t i = 0; i < m; ++i) f[i] += b[i];
    orc_ne_solve(m, n, rp, ci, val, perm, d2, f, ell, om, meth, eps_in, maxit, dya, dwa, &ki);
    info->krylov_iters_total += ki.iters;
    int32_t it_af = ki.iters, it_cc = 0;
    if (!ki.converged) failed = 1;
    for (int32_t j = 0; j < n; ++j) {
      dsa[j] = rd[j] - dwa[j] / d[j];
      dxa[j] = -d2[j] * dsa[j] - x[j];
    }
    double ap = step_len(n, x, dxa, opt->eta), ad = step_len(n, s, dsa, opt->eta);
    const double ap_af = ap, ad_af = ad;
    double sigma = 0.0, muaf_tr = 0.0;
    if (fmin(ap, ad) >= 1.0) {
      memcpy(dx, dxa, sizeof(double) * (size_t)n);
      memcpy(ds, dsa, sizeof(double) * (size_t)n);
      memcpy(dy, dya, sizeof(double) * (size_t)m);
    } else {
      double muaf = 0.0;
      for (int32_t j = 0; j < n; ++j) muaf += (x[j] + ap * dxa[j]) * (s[j] + ad * dsa[j]);
      muaf /= n;
      muaf_tr = muaf;
      /* reading: early phase (Gamma >= 1e-3) sigma = min(0.208, (mu_af/mu)^2),
         late phase sigma = min(0.208, 10 Gamma) */
      if (Gam >= 1e-3) {
        double r = muaf / mu;
        sigma = fmin(opt->sigma_max, r * r);
      } else {
        sigma = fmin(opt->sigma_max, 10.0 * Gam);
      }
      /* corrector: f_cc = A S^-1 (dX_af ds_af - sigma mu e); reading: sigma * mu
         (the mu of this iterate) as in the equations that define f_cc */
      for (int32_t j = 0; j < n; ++j) h[j] = (dxa[j] * dsa[j] - sigma * mu) / s[j];
      if (opt->corrector_ba) {
        /* BA-GMRES on the least-squares form of the corrector (Sec. 3.2):
           min ||(A D)^T dy - r||, r = (XS)^-1/2 (dX_af ds_af - sigma mu e) = h / d */
        for (int32_t j = 0; j < n; ++j) tmpn[j] = h[j] / d[j];
        orc_ls_solve(m, n, rp, ci, val, perm, d2, tmpn, ell, om, eps_in, maxit, dyc, dwc, &ki);
      } else {
        spmv(m, rp, ci, val, h, f);
        orc_ne_solve(m, n, rp, ci, val, perm, d2, f, ell, om, meth, eps_in, maxit, dyc, dwc, &ki);
      }
      info->krylov_iters_total += ki.iters;
      it_cc = ki.iters;
      if (!ki.converged) failed = 1;
      for (int32_t j = 0; j < n; ++j) {
        double dsc = -dwc[j] / d[j];                 /* Eq. (cc2) */
        double dxc = -d2[j] * dsc - h[j];            /* Eq. (cc3) */
        dx[j] = dxa[j] + dxc;
        ds[j] = dsa[j] + dsc;
      }
      for (int32_t i = 0; i < m; ++i) dy[i] = dya[i] + dyc[i];
    }
    /* trial steps of the combined direction */
    ap = step_len(n, x, dx, opt->eta);
    ad = step_len(n, s, ds, opt->eta);
    /* multiple centrality correctors (Gondzio): aim at step lengths larger by
       GZ_DELTA, move the complementarity products of that trial point that
       fall outside [GZ_BMIN, GZ_BMAX] * sigma mu back to the box, solve the
       Newton system for that change of the third block (r_p = r_d = 0) and
       keep the corrected direction while it lengthens the shorter step by at
       least GZ_GAMMA * GZ_DELTA.  reading: the parameter values are the ones
       of the published method; sigma mu is this iteration's centring target;
       a corrector whose Krylov solve does not converge is not used. */
    if (opt->max_correctors > 0 && sigma > 0.0) {
      const double GZ_DELTA = 0.1, GZ_BMIN = 0.1, GZ_BMAX = 10.0, GZ_GAMMA = 0.1;
      double *hg = dalloc(n), *dwg = dalloc(n), *dyg = dalloc(m), *dx2 = dalloc(n), *ds2 = dalloc(n);
      for (int32_t kc = 0; kc < opt->max_correctors; ++kc) {
        double amin = fmin(ap, ad);
        if (amin >= 1.0) break;
        double apt = fmin(1.0, ap + GZ_DELTA), adt = fmin(1.0, ad + GZ_DELTA);
        double lo = GZ_BMIN * sigma * mu, hi = GZ_BMAX * sigma * mu;
        for (int32_t j = 0; j < n; ++j) {
          double v = (x[j] + apt * dx[j]) * (s[j] + adt * ds[j]), t = 0.0;
          if (v < lo) t = lo - v;
          else if (v > hi) t = fmax(hi - v, -hi);
          hg[j] = -t / s[j];                       /* the third block S dx + X ds = t */
        }
        spmv(m, rp, ci, val, hg, f);
        orc_ne_solve(m, n, rp, ci, val, perm, d2, f, ell, om, meth, eps_in, maxit, dyg, dwg, &ki);
        info->krylov_iters_total += ki.iters;
        if (!ki.converged) break;
        for (int32_t j = 0; j < n; ++j) {
          double dsc = -dwg[j] / d[j];
          double dxc = -d2[j] * dsc - hg[j];
          dx2[j] = dx[j] + dxc;
          ds2[j] = ds[j] + dsc;
        }
        double ap2 = step_len(n, x, dx2, opt->eta), ad2 = step_len(n, s, ds2, opt->eta);
        if (!(fmin(ap2, ad2) >= amin + GZ_GAMMA * GZ_DELTA)) break;
        memcpy(dx, dx2, sizeof(double) * (size_t)n);
        memcpy(ds, ds2, sizeof(double) * (size_t)n);
        for (int32_t i = 0; i < m; ++i) dy[i] += dyg[i];
        ap = ap2;
        ad = ad2;
        info->correctors++;
      }
      free(hg); free(dwg); free(dyg); free(dx2); free(ds2);
    }
    /* centrality backtracking */
    double tau = 1.0;
    for (int32_t tr = 0; tr < 60; ++tr) {
      double a1 = tau * ap, a2 = tau * ad, mn = INFINITY, sm = 0.0;
      for (int32_t j = 0; j < n; ++j) {
        double pr = (x[j] + a1 * dx[j]) * (s[j] + a2 * ds[j]);
        if (pr < mn) mn = pr;
        sm += pr;
      }
      if (mn >= opt->phi * sm / n) break;
      if (tr == 59) break;           /* reading: after 60 trials the last one is kept */
      tau *= opt->backtrack;
    }
    ap *= tau; ad *= tau;
    for (int32_t j = 0; j < n; ++j) { x[j] += ap * dx[j]; s[j] += ad * ds[j]; }
    for (int32_t i = 0; i < m; ++i) y[i] += ad * dy[i];
    if (failed) info->krylov_failures++;
    failed_prev = failed;
    if (trace && k < opt->max_ipm) {
      double *tr = trace + (size_t)k * ORC_TRACE_COLS;
      tr[0] = Gam; tr[1] = mu; tr[2] = pinf; tr[3] = dinf; tr[4] = eps_in;
      tr[5] = it_af; tr[6] = it_cc; tr[7] = ap; tr[8] = ad; tr[9] = sigma; tr[10] = muaf_tr;
      tr[11] = ap_af; tr[12] = ad_af; tr[13] = tau; tr[14] = failed; tr[15] = gap;
    }
    if (opt->verbose)
      fprintf(stderr, "orc k=%2d Gam=%.3e mu=%.3e pinf=%.2e dinf=%.2e gap=%.2e eps=%.1e it=%d/%d "
                      "ap=%.3f ad=%.3f sig=%.3e\n",
              k, Gam, mu, pinf, dinf, gap, eps_in, it_af, it_cc, ap, ad, sigma);
  }
  info->status = status;
  free(color); free(perm); free(cptr);
  free(d2); free(d); free(rd); free(rp_); free(f); free(dwa); free(dya); free(dxa); free(dsa);
  free(dwc); free(dyc); free(dx); free(ds); free(dy); free(h); free(tmpm); free(tmpn);
  return status;
}

int32_t orc_lp_solve(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *val, const double *b, const double *c, const orc_options *opt,
                     double *x, double *y, double *s, orc_info *info, double *trace) {
  memset(info, 0, sizeof(*info));
  /* removal of zero rows and columns, the only preprocessing of Sec. 4.2 */
  int32_t *rmap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t *cmap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t *ccount = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  int32_t mr = 0, nr = 0;
  for (int64_t k = 0; k < row_ptr[m]; ++k) ccount[col_idx[k]]++;
  for (int32_t i = 0; i < m; ++i) {
    if (row_ptr[i + 1] == row_ptr[i]) {
      rmap[i] = -1;
      if (b[i] != 0.0) { info->status = ORC_EMPTY_ROW_INCONSISTENT; goto out; }
    } else {
      rmap[i] = mr++;
    }
  }
  for (int32_t j = 0; j < n; ++j) {
    if (ccount[j] == 0) {
      cmap[j] = -1;
      if (c[j] < 0.0) { info->status = ORC_EMPTY_COL_UNBOUNDED; goto out; }
    } else {
      cmap[j] = nr++;
    }
  }
  {
    int64_t *rp2 = (int64_t *)calloc((size_t)mr + 1, sizeof(int64_t));
    int32_t *ci2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(row_ptr[m] > 0 ? row_ptr[m] : 1));
    double *v2 = dalloc(row_ptr[m]), *b2 = dalloc(mr), *c2 = dalloc(nr);
    double *x2 = dalloc(nr), *y2 = dalloc(mr), *s2 = dalloc(nr);
    int64_t nz = 0;
    for (int32_t i = 0; i < m; ++i) {
      if (rmap[i] < 0) continue;
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        ci2[nz] = cmap[col_idx[k]];
        v2[nz++] = val[k];
      }
      rp2[rmap[i] + 1] = nz;
      b2[rmap[i]] = b[i];
    }
    for (int32_t j = 0; j < n; ++j) if (cmap[j] >= 0) c2[cmap[j]] = c[j];
    ipm_core(mr, nr, rp2, ci2, v2, b2, c2, opt, x2, y2, s2, info, trace);
    for (int32_t i = 0; i < m; ++i) y[i] = rmap[i] >= 0 ? y2[rmap[i]] : 0.0;
    for (int32_t j = 0; j < n; ++j) {
      x[j] = cmap[j] >= 0 ? x2[cmap[j]] : 0.0;
      s[j] = cmap[j] >= 0 ? s2[cmap[j]] : c[j];
    }
    free(rp2); free(ci2); free(v2); free(b2); free(c2); free(x2); free(y2); free(s2);
  }
out:
  free(rmap); free(cmap); free(ccount);
  return info->status;
}
