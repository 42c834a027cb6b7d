// ipm.cu -- search-direction solve (Sec. 2.2, 3.5) and the interior-point
// driver (Algorithm 1).  Host code only decides scalars (step lengths, sigma,
// tolerances) from reductions computed on the device; every vector operation
// runs in the kernels below or in the persistent Krylov kernel.
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "ipm.cuh"
#include "ipm_kernels.cuh"

namespace {

constexpr int TPB = RED_THREADS;

// fh = f / rho (rows with rho = 0 are empty and carry 0)
__global__ void k_div(int m, const double *f, const double *rho, double *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = rho[i] > 0.0 ? f[i] / rho[i] : 0.0;
}
__global__ void k_fill(int len, double v, double *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = v;
}

// r_p = b - Ax, r_d = c - A^T y - s; sums ||r_p||^2, ||r_d||^2, x^T s, c^T x, b^T y
__global__ void k_resid(int m, int n, const double *b, const double *Ax, const double *y, double *rp,
                        const double *c, const double *ATy, const double *x, const double *s, double *rd,
                        RedArgs R) {
  double v[5] = {0, 0, 0, 0, 0};
  double mn[1] = {INFINITY};
  const int NT = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += NT) {
    double r = b[i] - Ax[i];
    rp[i] = r;
    v[0] += r * r;
    v[4] += b[i] * y[i];
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT) {
    double r = c[j] - ATy[j] - s[j];
    rd[j] = r;
    v[1] += r * r;
    v[2] += x[j] * s[j];
    v[3] += c[j] * x[j];
  }
  grid_reduce<5, 1>(v, mn, R);
}

// sums ||a||^2 over m and ||b||^2 over n
__global__ void k_norms(int m, int n, const double *a, const double *bb, RedArgs R) {
  double v[2] = {0, 0};
  double mn[1] = {INFINITY};
  const int NT = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += NT) v[0] += a[i] * a[i];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT) v[1] += bb[j] * bb[j];
  grid_reduce<2, 1>(v, mn, R);
}

// d2 = x / s, d = sqrt(d2), hv = d2 * r_d
__global__ void k_d2(int n, const double *x, const double *s, const double *rd, double *d2, double *d,
                     double *hv) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double q = x[j] / s[j];
  d2[j] = q;
  d[j] = sqrt(q);
  hv[j] = q * rd[j];
}

// predictor direction, Eqs. (aff2)-(aff3): ds = r_d - dw / d, dx = -d2 ds - x;
// minima of -x/dx over dx < 0 and of -s/ds over ds < 0 (Eq. steplength)
__global__ void k_dir_pred(int n, const double *rd, const double *dw, const double *d, const double *d2,
                           const double *x, const double *s, double *dxa, double *dsa, RedArgs R) {
  double v[1] = {0};
  double mn[2] = {INFINITY, INFINITY};
  const int NT = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT) {
    double ds = rd[j] - dw[j] / d[j];
    double dx = -d2[j] * ds - x[j];
    dsa[j] = ds;
    dxa[j] = dx;
    if (dx < 0.0) mn[0] = fmin(mn[0], -x[j] / dx);
    if (ds < 0.0) mn[1] = fmin(mn[1], -s[j] / ds);
  }
  grid_reduce<1, 2>(v, mn, R);
}

// mu_af * n = (x + ap dxa)^T (s + ad dsa)
__global__ void k_muaf(int n, const double *x, const double *s, const double *dxa, const double *dsa,
                       double ap, double ad, RedArgs R) {
  double v[1] = {0};
  double mn[1] = {INFINITY};
  const int NT = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT)
    v[0] += (x[j] + ap * dxa[j]) * (s[j] + ad * dsa[j]);
  grid_reduce<1, 1>(v, mn, R);
}

// centrality corrector: v = (x + apt dx)(s + adt ds) moved back to [lo, hi]
// (t = target - v, at least -hi), as the third block S dx + X ds = t: h = -t / s
__global__ void k_gz_rhs(int n, const double *x, const double *s, const double *dx, const double *ds, double apt,
                         double adt, double lo, double hi, double *h) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    const double v = (x[j] + apt * dx[j]) * (s[j] + adt * ds[j]);
    double t = 0.0;
    if (v < lo) t = lo - v;
    else if (v > hi) t = fmax(hi - v, -hi);
    h[j] = -t / s[j];
  }
}

// h = S^-1 (dX_af ds_af - sigma mu e)
__global__ void k_h(int n, const double *dxa, const double *dsa, const double *s, double smu, double *h) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) h[j] = (dxa[j] * dsa[j] - smu) / s[j];
}

// corrector recovery, Eqs. (cc2)-(cc3), summed with the predictor direction;
// dy = dya + dyc; ratio minima of the combined direction
__global__ void k_dir_corr(int m, int n, const double *dxa, const double *dsa, const double *dwc,
                           const double *d, const double *d2, const double *h, const double *x,
                           const double *s, double *dx, double *ds, const double *dya, const double *dyc,
                           double *dy, RedArgs R) {
  double v[1] = {0};
  double mn[2] = {INFINITY, INFINITY};
  const int NT = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT) {
    double dsc = -dwc[j] / d[j];
    double dxc = -d2[j] * dsc - h[j];
    double X = dxa[j] + dxc, S = dsa[j] + dsc;
    dx[j] = X;
    ds[j] = S;
    if (X < 0.0) mn[0] = fmin(mn[0], -x[j] / X);
    if (S < 0.0) mn[1] = fmin(mn[1], -s[j] / S);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += NT) dy[i] = dya[i] + dyc[i];
  grid_reduce<1, 2>(v, mn, R);
}

constexpr int NTRIAL = 8;
// centrality test for NTRIAL common shrink factors tau_t = tau0 * bt^t:
// min_j (x + a_p dx)_j (s + a_d ds)_j and the sum, per trial
__global__ void k_backtrack(int n, const double *x, const double *s, const double *dx, const double *ds,
                            double ap, double ad, double tau0, double bt, RedArgs R) {
  double v[NTRIAL];
  double mn[NTRIAL];
#pragma unroll
  for (int t = 0; t < NTRIAL; ++t) { v[t] = 0.0; mn[t] = INFINITY; }
  double tau[NTRIAL];
  tau[0] = tau0;
  for (int t = 1; t < NTRIAL; ++t) tau[t] = tau[t - 1] * bt;
  const int NT = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT) {
    const double X = x[j], S = s[j], DX = dx[j], DS = ds[j];
#pragma unroll
    for (int t = 0; t < NTRIAL; ++t) {
      double pr = (X + tau[t] * ap * DX) * (S + tau[t] * ad * DS);
      v[t] += pr;
      mn[t] = fmin(mn[t], pr);
    }
  }
  grid_reduce<NTRIAL, NTRIAL>(v, mn, R);
}

__global__ void k_update(int m, int n, double *x, double *s, double *y, const double *dx, const double *ds,
                         const double *dy, double ap, double ad) {
  const int NT = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT) {
    x[j] += ap * dx[j];
    s[j] += ad * ds[j];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += NT) y[i] += ad * dy[i];
}

// starting point helpers
__global__ void k_start_min(int n, const double *x, double *s, const double *c, const double *w, RedArgs R) {
  double v[1] = {0};
  double mn[2] = {INFINITY, INFINITY};
  const int NT = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT) {
    double sj = c[j] - w[j];  // s~ = c - A^T y~ (w = A^T y~ from the w-form solve)
    s[j] = sj;
    mn[0] = fmin(mn[0], x[j]);
    mn[1] = fmin(mn[1], sj);
  }
  grid_reduce<1, 2>(v, mn, R);
}
__global__ void k_start_shift(int n, double *x, double *s, double sx, double ss, RedArgs R) {
  double v[3] = {0, 0, 0};
  double mn[1] = {INFINITY};
  const int NT = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += NT) {
    double X = x[j] + sx, S = s[j] + ss;
    x[j] = X;
    s[j] = S;
    v[0] += X * S;
    v[1] += X;
    v[2] += S;
  }
  grid_reduce<3, 1>(v, mn, R);
}
__global__ void k_start_final(int n, double *x, double *s, double hx, double hs) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double X = x[j] + hx, S = s[j] + hs;
  x[j] = X > 0.0 ? X : 1.0;
  s[j] = S > 0.0 ? S : 1.0;
}

// empty row / column checks (removed rows must have b_i = 0, removed columns c_j >= 0)
__global__ void k_check_empty(int m_in, int n_in, const int *pos_of_in_row, const int *col_of_in,
                              const double *b, const double *c, int *flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m_in && pos_of_in_row[i] < 0 && b[i] != 0.0) atomicOr(&flags[0], 1);
  if (i < n_in && col_of_in[i] < 0 && c[i] < 0.0) atomicOr(&flags[0], 2);
  if (i < m_in && !isfinite(b[i])) atomicOr(&flags[0], 4);
  if (i < n_in && !isfinite(c[i])) atomicOr(&flags[0], 4);
}
__global__ void k_scatter_fill_s(int n_in, const int *col_of_in, const double *c, double *s_in) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n_in && col_of_in[j] < 0) s_in[j] = c[j];
}

inline int eb(long long n) { return (int)((n + TPB - 1) / TPB); }

}  // namespace

// ---------------------------------------------------------------------------
// search-direction solve on the current scaling (scale_rows already applied)
// ---------------------------------------------------------------------------
lpk_status ne_solve_scaled(lpk_ctx *ctx, DevProblem &P, const double *f, int ell, double omega, int solver,
                           int precision, double tol, int maxit, double *dy, double *dw, double *tmp_m,
                           KrylovResult *kr) {
  cudaStream_t st = ctx->stream;
  if (P.m > 0) LPK_LAUNCH(ctx, k_div, eb(P.m), TPB, 0, st, P.m, f, P.rho, tmp_m);  // f_hat = D_cal^-1 f
  lpk_status rc = krylov_solve(ctx, P, solver, precision, ell, omega, tmp_m, tol, maxit, dw, dy, kr, nullptr);
  if (rc != LPK_OK) return rc;
  if (ctx->verbose >= 2)
    fprintf(stderr, "  krylov: it=%d (fp32 %d, escalations %d) restarts=%d conv=%d brk=%d res/res0=%.3e (tol %.1e)\n",
            kr->iters, kr->iters32, kr->escalations, kr->restarts, kr->converged, kr->breakdown,
            kr->res0 > 0 ? kr->res / kr->res0 : 0.0, tol);
  // A_hat^T dy_hat = A^T D D_cal^-1 dy_hat, so dy = D_cal^-1 dy_hat
  if (P.m > 0) LPK_LAUNCH(ctx, k_div, eb(P.m), TPB, 0, st, P.m, dy, P.rho, dy);
  return LPK_OK;
}

// The corrector stage in least-squares form (Sec. 3.2): min ||A_hat^T dy_hat - r||
// by BA-GMRES with NR-SOR; f = A D r is its m-space image (f_hat = D_cal^-1 f
// gives the explicit residual ||f_hat - A_hat dw|| used for convergence)
lpk_status ls_solve_scaled(lpk_ctx *ctx, DevProblem &P, const double *r, const double *f, int ell, double omega,
                           int precision, double tol, int maxit, double *dy, double *dw, double *tmp_m,
                           KrylovResult *kr) {
  cudaStream_t st = ctx->stream;
  if (P.m > 0) LPK_LAUNCH(ctx, k_div, eb(P.m), TPB, 0, st, P.m, f, P.rho, tmp_m);
  lpk_status rc = krylov_solve_ls(ctx, P, precision, ell, omega, r, tmp_m, tol, maxit, dw, dy, kr);
  if (rc != LPK_OK) return rc;
  if (ctx->verbose >= 2)
    fprintf(stderr, "  ba-gmres: it=%d restarts=%d conv=%d brk=%d res/res0=%.3e (tol %.1e)\n", kr->iters,
            kr->restarts, kr->converged, kr->breakdown, kr->res0 > 0 ? kr->res / kr->res0 : 0.0, tol);
  if (P.m > 0) LPK_LAUNCH(ctx, k_div, eb(P.m), TPB, 0, st, P.m, dy, P.rho, dy);
  return LPK_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 1
// ---------------------------------------------------------------------------
namespace {
double clamp_eps(double e) { return e < 1e-14 ? 1e-14 : (e > 1e-4 ? 1e-4 : e); }
}  // namespace

lpk_status lp_solve_dev(lpk_ctx *ctx, DevProblem &P, const double *b_in, const double *c_in,
                        const lpk_options &o, double *x_in, double *y_in, double *s_in, lpk_info &info) {
  cudaStream_t st = ctx->stream;
  lpk_status rc;
  if ((rc = ensure_reduce(ctx)) != LPK_OK) return rc;
  const int m = P.m, n = P.n;
  const RedArgs R = red_args(ctx);
  const int RG = red_grid(ctx);
  double *h = ctx->h_red;
  ctx->verbose = o.verbose;
  info = lpk_info{};
  info.n_colors = P.n_colors;

  // workspace (kept with the problem): 12 m-vectors, 21 n-vectors, flags
  const size_t mm = m > 0 ? m : 1, nn = n > 0 ? n : 1;
  const size_t need = sizeof(double) * (12 * mm + 21 * nn + 4);
  if (P.ipm_bytes < need) {
    dev_free(st, P.ipm_buf);
    P.ipm_buf = nullptr;
    P.ipm_bytes = 0;
    LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.ipm_buf, need / sizeof(double)));
    P.ipm_bytes = need;
  }
  double *buf = P.ipm_buf;

  // checks on b and c (input numbering)
  {
    int *flags = (int *)(buf + 12 * mm + 21 * nn);
    LPK_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, sizeof(int), st));
    int len = std::max(P.m_in, P.n_in);
    if (len > 0)
      LPK_LAUNCH(ctx, k_check_empty, eb(len), TPB, 0, st, P.m_in, P.n_in, P.pos_of_in_row, P.col_of_in, b_in, c_in, flags);
    int hf = 0;
    cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    ctx_sync(ctx);
    if (hf & 4) {
      ctx->err = "b or c has a non-finite entry";
      info.status = LPK_INVALID_ARG;
      return LPK_INVALID_ARG;
    }
    if (hf & 1) {
      ctx->err = "empty row of A with nonzero right-hand side";
      info.status = LPK_EMPTY_ROW_INCONSISTENT;
      return LPK_EMPTY_ROW_INCONSISTENT;
    }
    if (hf & 2) {
      ctx->err = "empty column of A with negative cost";
      info.status = LPK_EMPTY_COL_UNBOUNDED;
      return LPK_EMPTY_COL_UNBOUNDED;
    }
  }

  double *q = buf;
  auto take_m = [&]() { double *r = q; q += mm; return r; };
  auto take_n = [&]() { double *r = q; q += nn; return r; };
  double *b = take_m(), *y = take_m(), *rp = take_m(), *f = take_m(), *dya = take_m(), *dyc = take_m(),
         *dy = take_m(), *tm = take_m(), *tm2 = take_m(), *tm3 = take_m(), *dyg = take_m(), *dy2 = take_m();
  double *c = take_n(), *x = take_n(), *s = take_n(), *rd = take_n(), *d2 = take_n(), *d = take_n(),
         *hv = take_n(), *dwa = take_n(), *dxa = take_n(), *dsa = take_n(), *dwc = take_n(), *dx = take_n(),
         *ds = take_n(), *hh = take_n(), *tn = take_n(), *tn2 = take_n(), *tn3 = take_n(), *hg = take_n(),
         *dwg = take_n(), *dx2 = take_n(), *ds2 = take_n();
  (void)tm3; (void)tn3; (void)tn2;
  gather_m(ctx, P, b_in, b);
  gather_n(ctx, P, c_in, c);

  const int maxit = o.max_krylov > 0 ? o.max_krylov : m;
  const int ell = o.inner_sweeps;
  const double om = o.omega;
  const int solver = o.solver, prec = o.precision;
  KrylovResult kr;

  // ---- starting point.  The paper defers to LIPSOL without stating it; this
  // uses Mehrotra's rule: x~ = min-norm solution of A x = b, y~ solves
  // A A^T y = A c, s~ = c - A^T y~, then the two shifts.
  if (n > 0) LPK_LAUNCH(ctx, k_fill, eb(n), TPB, 0, st, n, 1.0, d2);
  scale_rows(ctx, P, d2);
  if ((rc = ne_solve_scaled(ctx, P, b, ell, om, solver, prec, o.start_tol, maxit, tm, x, tm2, &kr)) != LPK_OK)
    return rc;
  info.krylov_iters_total += kr.iters;
  spmv_csr(ctx, P, c, f, nullptr, 1.0);
  if ((rc = ne_solve_scaled(ctx, P, f, ell, om, solver, prec, o.start_tol, maxit, y, tn, tm2, &kr)) != LPK_OK)
    return rc;
  info.krylov_iters_total += kr.iters;
  LPK_LAUNCH(ctx, k_start_min, RG, TPB, 0, st, n, x, s, c, tn, R);
  if ((rc = red_fetch(ctx, 3)) != LPK_OK) return rc;
  {
    const double sx = std::max(-1.5 * h[1], 0.0), ss = std::max(-1.5 * h[2], 0.0);
    LPK_LAUNCH(ctx, k_start_shift, RG, TPB, 0, st, n, x, s, sx, ss, R);
    if ((rc = red_fetch(ctx, 3)) != LPK_OK) return rc;
    const double xs = h[0], sumx = h[1], sums = h[2];
    const double hx = sums > 0.0 ? 0.5 * xs / sums : 0.0, hs = sumx > 0.0 ? 0.5 * xs / sumx : 0.0;
    if (n > 0) LPK_LAUNCH(ctx, k_start_final, eb(n), TPB, 0, st, n, x, s, hx, hs);
  }
  LPK_LAUNCH(ctx, k_norms, RG, TPB, 0, st, m, n, b, c, R);
  if ((rc = red_fetch(ctx, 2)) != LPK_OK) return rc;
  const double nb = std::max(sqrt(h[0]), 1.0), ncn = std::max(sqrt(h[1]), 1.0);

  double eps_in = o.eps_in0;
  int status = LPK_MAX_IPM_ITER;
  bool failed_prev = false;
  for (int k = 0; k <= o.max_ipm; ++k) {
    // residuals (Eq. SE1) and Gamma (Eq. errorMeasureDef)
    spmv_csr(ctx, P, x, tm, nullptr, 1.0);
    spmv_csc(ctx, P, y, tn);
    LPK_LAUNCH(ctx, k_resid, RG, TPB, 0, st, m, n, b, tm, y, rp, c, tn, x, s, rd, R);
    if ((rc = red_fetch(ctx, 5)) != LPK_OK) return rc;
    const double mu = n > 0 ? h[2] / n : 0.0;
    const double pinf = sqrt(h[0]) / nb, dinf = sqrt(h[1]) / ncn;
    const double Gam = std::max(mu, std::max(pinf, dinf));
    const double pobj = h[3], dobj = h[4];
    const double gap = fabs(pobj - dobj) / (1.0 + fabs(pobj));
    info.gamma = Gam; info.rel_gap = gap; info.pinf = pinf; info.dinf = dinf; info.mu = mu;
    info.obj_primal = pobj; info.obj_dual = dobj; info.ipm_iters = k;
    if (!std::isfinite(Gam)) { status = LPK_DIVERGED; break; }
    if (Gam <= o.tol && gap <= o.tol) { status = LPK_OK; break; }
    if (k == o.max_ipm) { status = LPK_MAX_IPM_ITER; break; }
    // eps_in schedule of Sec. 4.2 (unchanged while log10 Gamma > 1)
    if (k > 0) {
      if (failed_prev) eps_in *= 1.5;
      const double lg = log10(Gam);
      if (lg <= -3.0) eps_in *= 0.375;
      else if (lg <= 1.0) eps_in *= 0.75;
      eps_in = clamp_eps(eps_in);
    }
    bool failed = false;
    if (n > 0) LPK_LAUNCH(ctx, k_d2, eb(n), TPB, 0, st, n, x, s, rd, d2, d, hv);
    scale_rows(ctx, P, d2);  // once per IPM iteration, shared by both stages
    // predictor: f_af = b + A S^-1 X r_d
    spmv_csr(ctx, P, hv, f, b, 1.0);
    if ((rc = ne_solve_scaled(ctx, P, f, ell, om, solver, prec, eps_in, maxit, dya, dwa, tm2, &kr)) != LPK_OK)
      return rc;
    info.krylov_iters_total += kr.iters;
    const int it_af = kr.iters;
    int it_cc = 0;
    if (!kr.converged) failed = true;
    LPK_LAUNCH(ctx, k_dir_pred, RG, TPB, 0, st, n, rd, dwa, d, d2, x, s, dxa, dsa, R);
    if ((rc = red_fetch(ctx, 3)) != LPK_OK) return rc;
    double ap = std::min(1.0, o.eta * h[1]), ad = std::min(1.0, o.eta * h[2]);
    double sigma = 0.0;
    double *DX = dxa, *DS = dsa, *DY = dya;
    if (!(std::min(ap, ad) >= 1.0)) {
      LPK_LAUNCH(ctx, k_muaf, RG, TPB, 0, st, n, x, s, dxa, dsa, ap, ad, R);
      if ((rc = red_fetch(ctx, 1)) != LPK_OK) return rc;
      const double muaf = h[0] / n;
      if (Gam >= 1e-3) {
        const double r = muaf / mu;
        sigma = std::min(o.sigma_max, r * r);
      } else {
        sigma = std::min(o.sigma_max, 10.0 * Gam);
      }
      if (n > 0) LPK_LAUNCH(ctx, k_h, eb(n), TPB, 0, st, n, dxa, dsa, s, sigma * mu, hh);
      spmv_csr(ctx, P, hh, f, nullptr, 1.0);  // f_cc = A h
      if (o.corrector == 1) {
        // least-squares form solved by BA-GMRES (Sec. 3.2): r = (XS)^-1/2 (dX ds - sigma mu e) = h / d
        if (n > 0) LPK_LAUNCH(ctx, k_div, eb(n), TPB, 0, st, n, hh, d, tn3);
        if ((rc = ls_solve_scaled(ctx, P, tn3, f, ell, om, prec, eps_in, maxit, dyc, dwc, tm2, &kr)) != LPK_OK)
          return rc;
      } else if ((rc = ne_solve_scaled(ctx, P, f, ell, om, solver, prec, eps_in, maxit, dyc, dwc, tm2, &kr)) !=
                 LPK_OK) {
        return rc;
      }
      info.krylov_iters_total += kr.iters;
      it_cc = kr.iters;
      if (!kr.converged) failed = true;
      LPK_LAUNCH(ctx, k_dir_corr, RG, TPB, 0, st, m, n, dxa, dsa, dwc, d, d2, hh, x, s, dx, ds, dya, dyc, dy, R);
      if ((rc = red_fetch(ctx, 3)) != LPK_OK) return rc;
      DX = dx; DS = ds; DY = dy;
    }
    // trial steps of the combined direction, then centrality backtracking
    double ap0 = std::min(1.0, o.eta * h[1]), ad0 = std::min(1.0, o.eta * h[2]);
    if (DX == dxa) { ap0 = ap; ad0 = ad; }
    // multiple centrality correctors (Gondzio): aim at step lengths larger by
    // GZ_DELTA, move the complementarity products of that trial point that fall
    // outside [GZ_BMIN, GZ_BMAX] sigma mu back to the box, solve the Newton
    // system for that change of its third block (r_p = r_d = 0) and keep the
    // corrected direction while it lengthens the shorter step by at least
    // GZ_GAMMA GZ_DELTA; a corrector whose Krylov solve fails is not used
    if (o.max_correctors > 0 && DX != dxa && sigma > 0.0) {
      constexpr double GZ_DELTA = 0.1, GZ_BMIN = 0.1, GZ_BMAX = 10.0, GZ_GAMMA = 0.1;
      double *DX2 = DX == dx ? dx2 : dx, *DS2 = DS == ds ? ds2 : ds, *DY2 = DY == dy ? dy2 : dy;
      for (int kc = 0; kc < o.max_correctors; ++kc) {
        const double amin = std::min(ap0, ad0);
        if (amin >= 1.0) break;
        const double apt = std::min(1.0, ap0 + GZ_DELTA), adt = std::min(1.0, ad0 + GZ_DELTA);
        if (n > 0)
          LPK_LAUNCH(ctx, k_gz_rhs, eb(n), TPB, 0, st, n, x, s, DX, DS, apt, adt, GZ_BMIN * sigma * mu,
                     GZ_BMAX * sigma * mu, hg);
        spmv_csr(ctx, P, hg, f, nullptr, 1.0);
        if (o.corrector == 1) {
          if (n > 0) LPK_LAUNCH(ctx, k_div, eb(n), TPB, 0, st, n, hg, d, tn3);
          if ((rc = ls_solve_scaled(ctx, P, tn3, f, ell, om, prec, eps_in, maxit, dyg, dwg, tm2, &kr)) != LPK_OK)
            return rc;
        } else if ((rc = ne_solve_scaled(ctx, P, f, ell, om, solver, prec, eps_in, maxit, dyg, dwg, tm2, &kr)) !=
                   LPK_OK) {
          return rc;
        }
        info.krylov_iters_total += kr.iters;
        if (!kr.converged) break;
        LPK_LAUNCH(ctx, k_dir_corr, RG, TPB, 0, st, m, n, DX, DS, dwg, d, d2, hg, x, s, DX2, DS2, DY, dyg, DY2, R);
        if ((rc = red_fetch(ctx, 3)) != LPK_OK) return rc;
        const double ap1 = std::min(1.0, o.eta * h[1]), ad1 = std::min(1.0, o.eta * h[2]);
        if (!(std::min(ap1, ad1) >= amin + GZ_GAMMA * GZ_DELTA)) break;
        std::swap(DX, DX2);
        std::swap(DS, DS2);
        std::swap(DY, DY2);
        ap0 = ap1;
        ad0 = ad1;
        info.correctors++;
      }
    }
    double tau = 1.0;
    bool accepted = false;
    for (int base = 0; base < 60 && !accepted; base += NTRIAL) {
      LPK_LAUNCH(ctx, k_backtrack, RG, TPB, 0, st, n, x, s, DX, DS, ap0, ad0, tau, o.backtrack, R);
      if ((rc = red_fetch(ctx, 2 * NTRIAL)) != LPK_OK) return rc;
      for (int t = 0; t < NTRIAL && base + t < 60; ++t) {
        if (h[NTRIAL + t] >= o.phi * h[t] / n) { accepted = true; break; }
        tau *= o.backtrack;
      }
    }
    if (!accepted) tau /= o.backtrack;  // the last trial is kept
    const double apf = tau * ap0, adf = tau * ad0;
    LPK_LAUNCH(ctx, k_update, RG, TPB, 0, st, m, n, x, s, y, DX, DS, DY, apf, adf);
    if (failed) info.krylov_failures++;
    failed_prev = failed;
    if (o.verbose)
      fprintf(stderr, "lpk k=%2d Gam=%.3e mu=%.3e pinf=%.2e dinf=%.2e gap=%.2e eps=%.1e it=%d/%d ap=%.3f ad=%.3f "
                      "sig=%.3e\n", k, Gam, mu, pinf, dinf, gap, eps_in, it_af, it_cc, apf, adf, sigma);
  }
  info.status = status;
  // back to the input numbering: removed rows get y = 0, removed columns x = 0, s = c
  scatter_m(ctx, P, y, y_in);
  scatter_n(ctx, P, x, x_in, nullptr);
  scatter_n(ctx, P, s, s_in, nullptr);
  if (P.n_in > P.n) LPK_LAUNCH(ctx, k_scatter_fill_s, eb(P.n_in), TPB, 0, st, P.n_in, P.col_of_in, c_in, s_in);
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  return (lpk_status)status;
}
