// capi.cu -- the extern "C" entry points declared in include/lpk.h.
#include <math.h>

#include <cstring>
#include <new>
#include <vector>

#include "ipm.cuh"
#include "ipm_kernels.cuh"

namespace {

// Host or device vector argument: device pointers are used in place, host
// arrays are staged through a temporary device buffer.
struct Vec {
  lpk_ctx *ctx;
  double *dev = nullptr;
  void *user;
  size_t len;
  bool owned = false;
  bool out;
  Vec(lpk_ctx *c, const double *p, size_t l, int on_device, bool is_out)
      : ctx(c), user((void *)p), len(l), out(is_out) {
    if (on_device || p == nullptr) {
      dev = (double *)p;
    } else {
      owned = true;
    }
  }
  lpk_status init() {
    if (!owned) return LPK_OK;
    LPK_CUDA_TRY(ctx, dev_alloc(ctx, &dev, len));
    if (!out && len)
      LPK_CUDA_TRY(ctx, cudaMemcpyAsync(dev, user, sizeof(double) * len, cudaMemcpyHostToDevice, ctx->stream));
    return LPK_OK;
  }
  lpk_status finish() {
    if (owned && out && len)
      LPK_CUDA_TRY(ctx, cudaMemcpyAsync(user, dev, sizeof(double) * len, cudaMemcpyDeviceToHost, ctx->stream));
    return LPK_OK;
  }
  ~Vec() {
    if (owned && dev) {
      dev_free(ctx->stream, dev);
      ctx_sync(ctx);  // outputs are in the caller's host buffer on return
    }
  }
};

struct DevBuf {  // temporary device vector of one call (stream-ordered free)
  lpk_ctx *ctx;
  double *p = nullptr;
  explicit DevBuf(lpk_ctx *c) : ctx(c) {}
  ~DevBuf() { dev_free(ctx->stream, p); }
};

__global__ void k_ahat_to_input(long long nnz, const long long *src, const double *ah, double *out) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < nnz) out[src[k]] = ah[k];
}
__global__ void k_d2_check(int n, const double *d2, int *bad) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && !(d2[j] > 0.0 && isfinite(d2[j]))) atomicOr(bad, 1);
}

#define CHECK_CTX(ctx)                           \
  do {                                           \
    if (!(ctx)) return LPK_INVALID_ARG;          \
    cudaSetDevice((ctx)->device);                \
  } while (0)
#define CHECK_P(ctx, P)                          \
  do {                                           \
    if (!(P) || !(P)->ctx || (P)->ctx != (ctx)) {   \
      (ctx)->err = "problem does not belong to this context"; \
      return LPK_INVALID_ARG;                    \
    }                                            \
  } while (0)
#define TRY(expr)                                \
  do {                                           \
    lpk_status s__ = (expr);                     \
    if (s__ != LPK_OK) return s__;               \
  } while (0)

lpk_status check_d2(lpk_ctx *ctx, const DevProblem &P, const double *d2_int) {
  int *bad;
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &bad, 1));
  cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream);
  if (P.n > 0) LPK_LAUNCH(ctx, k_d2_check, (P.n + 255) / 256, 256, 0, ctx->stream, P.n, d2_int, bad);
  int h = 0;
  cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  dev_free(ctx->stream, bad);
  ctx_sync(ctx);
  if (h) {
    ctx->err = "d2 must be positive and finite";
    return LPK_INVALID_ARG;
  }
  return LPK_OK;
}

}  // namespace

LPK_API lpk_status lpk_create(lpk_ctx **out, int32_t device, void *cuda_stream) {
  if (!out) return LPK_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LPK_CUDA_ERROR;
  if (cudaSetDevice(device) != cudaSuccess) return LPK_CUDA_ERROR;
  lpk_ctx *ctx = new (std::nothrow) lpk_ctx();
  if (!ctx) return LPK_OOM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete ctx;
    return LPK_CUDA_ERROR;
  }
  const lpk_status st = noalloc_setup(ctx);  // scratch of lpk_ne_solve_noalloc on this device
  if (st != LPK_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return LPK_OK;
}

LPK_API void lpk_destroy(lpk_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (lpk_problem *p : ctx->problems) {  // problems still alive die with their context
    free_problem(p->d);
    p->ctx = nullptr;
  }
  ctx->problems.clear();
  dev_free(ctx->stream, ctx->red_part);
  dev_free(ctx->stream, ctx->red_count);
  dev_free(ctx->stream, ctx->red_out);
  dev_free(ctx->stream, ctx->kctl);
  dev_free(ctx->stream, ctx->kpart);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ev_block) cudaEventDestroy(ctx->ev_block);
  if (ctx->h_red) cudaFreeHost(ctx->h_red);
  if (ctx->h_kctl) cudaFreeHost(ctx->h_kctl);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  delete ctx;
}

LPK_API lpk_status lpk_get_stats(const lpk_ctx *ctx, lpk_stats *out) {
  if (!ctx || !out) return LPK_INVALID_ARG;
  *out = ctx->stats;
  out->last_cluster_size = ctx->last_cluster;
  out->last_resident = ctx->last_resident;
  out->last_u_global = ctx->last_u_global;
  return LPK_OK;
}

LPK_API lpk_status lpk_set_exec(lpk_ctx *ctx, int32_t exec, int32_t cluster_size) {
  if (!ctx) return LPK_INVALID_ARG;
  const int no_res = (exec & LPK_EXEC_NO_RESIDENT) != 0;
  const int ush = (exec & LPK_EXEC_U_SHARED) != 0, ugl = (exec & LPK_EXEC_U_GLOBAL) != 0;
  exec &= ~(LPK_EXEC_NO_RESIDENT | LPK_EXEC_U_SHARED | LPK_EXEC_U_GLOBAL);
  if (exec < LPK_EXEC_AUTO || exec > LPK_EXEC_BATCH || (ush && ugl) ||
      !(cluster_size == 0 || cluster_size == 2 || cluster_size == 4 || cluster_size == 8 || cluster_size == 16)) {
    ctx->err = "lpk_set_exec: exec must be 0..3 (with at most one of U_SHARED, U_GLOBAL) and cluster_size 0, 2, 4, 8 "
               "or 16";
    return LPK_INVALID_ARG;
  }
  ctx->cluster_mode = exec;
  ctx->cluster_size_override = cluster_size;
  ctx->resident_mode = no_res;
  ctx->u_place = ush ? 1 : ugl ? 2 : 0;
  return LPK_OK;
}

LPK_API lpk_status lpk_set_wait_limit(lpk_ctx *ctx, double seconds, int64_t test_stall_barrier) {
  if (!ctx) return LPK_INVALID_ARG;
  if (!(seconds > 0.0 && seconds < 1e6) || test_stall_barrier < 0) {
    ctx->err = "lpk_set_wait_limit: seconds must be in (0, 1e6) and test_stall_barrier >= 0";
    return LPK_INVALID_ARG;
  }
  ctx->wait_limit_ns = (unsigned long long)(seconds * 1e9);
  ctx->stall_barrier = test_stall_barrier;
  return LPK_OK;
}

LPK_API lpk_status lpk_set_phase_timing(lpk_ctx *ctx, int32_t on) {
  if (!ctx) return LPK_INVALID_ARG;
  ctx->phase_timing = on ? 1 : 0;
  return LPK_OK;
}

LPK_API lpk_status lpk_reset_stats(lpk_ctx *ctx) {
  if (!ctx) return LPK_INVALID_ARG;
  ctx->stats = lpk_stats{};
  return LPK_OK;
}

LPK_API const char *lpk_last_error(const lpk_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

LPK_API void lpk_default_options(lpk_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->eta = 0.9995;
  o->phi = 1e-5;
  o->sigma_max = 0.208;
  o->eps_in0 = 1e-6;
  o->omega = 1.0;
  o->start_tol = 1e-10;
  o->backtrack = 0.95;
  o->max_ipm = 99;
  o->max_krylov = 0;
  o->inner_sweeps = 1;
  o->solver = LPK_MRNE;
  o->precision = LPK_FP64;
  o->verbose = 0;
  o->color_seed = 0x5EEDull;
}

LPK_API lpk_status lpk_prepare(lpk_ctx *ctx, const lpk_matrix *A, uint64_t color_seed, lpk_problem **P) {
  CHECK_CTX(ctx);
  if (!A || !P || A->m < 0 || A->n < 0 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val))) {
    ctx->err = "lpk_prepare: invalid arguments";
    return LPK_INVALID_ARG;
  }
  if (A->nnz >= (1ll << 31) - 1) {
    ctx->err = "lpk_prepare: nnz must be below 2^31";
    return LPK_INVALID_ARG;
  }
  *P = nullptr;
  lpk_problem *p = new (std::nothrow) lpk_problem();
  if (!p) return LPK_OOM;
  p->ctx = ctx;
  lpk_status st = prep_problem(ctx, A, color_seed, p->d);
  if (st != LPK_OK) {
    free_problem(p->d);
    delete p;
    return st;
  }
  ctx->problems.push_back(p);
  *P = p;
  return LPK_OK;
}

LPK_API void lpk_problem_free(lpk_problem *P) {
  if (!P) return;
  if (P->ctx) {  // null once its context was destroyed (device memory already released)
    lpk_ctx *ctx = P->ctx;
    cudaSetDevice(ctx->device);
    ctx_sync(ctx);
    free_problem(P->d);
    for (size_t i = 0; i < ctx->problems.size(); ++i)
      if (ctx->problems[i] == P) {
        ctx->problems.erase(ctx->problems.begin() + i);
        break;
      }
  }
  delete P;
}

LPK_API lpk_status lpk_problem_dims(const lpk_problem *P, int32_t *m, int32_t *n, int64_t *nnz,
                                    int32_t *n_colors) {
  if (!P) return LPK_INVALID_ARG;
  if (m) *m = P->d.m_in;
  if (n) *n = P->d.n_in;
  if (nnz) *nnz = P->d.nnz;
  if (n_colors) *n_colors = P->d.n_colors;
  return LPK_OK;
}

LPK_API lpk_status lpk_problem_coloring(lpk_ctx *ctx, const lpk_problem *P, int32_t *color, int32_t *perm,
                                        int32_t *color_ptr) {
  CHECK_CTX(ctx);
  CHECK_P(ctx, P);
  const DevProblem &d = P->d;
  if (color && d.m_in)
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(color, d.color_in, sizeof(int) * d.m_in, cudaMemcpyDeviceToHost, ctx->stream));
  if (perm && d.m)
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(perm, d.in_row_of_pos, sizeof(int) * d.m, cudaMemcpyDeviceToHost, ctx->stream));
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  if (color_ptr) std::memcpy(color_ptr, d.color_ptr_h.data(), sizeof(int) * d.color_ptr_h.size());
  return LPK_OK;
}

LPK_API lpk_status lpk_scale_rows(lpk_ctx *ctx, lpk_problem *P, const double *d2, double *rho, double *ahat,
                                  int32_t on_device) {
  CHECK_CTX(ctx);
  CHECK_P(ctx, P);
  DevProblem &d = P->d;
  if (!d2 || !rho) return LPK_INVALID_ARG;
  Vec vd2(ctx, d2, d.n_in, on_device, false), vrho(ctx, rho, d.m_in, on_device, true),
      vah(ctx, ahat, d.nnz, on_device, true);
  TRY(vd2.init());
  TRY(vrho.init());
  TRY(vah.init());
  DevBuf t(ctx);
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &t.p, d.n + 1));
  gather_n(ctx, d, vd2.dev, t.p);
  TRY(check_d2(ctx, d, t.p));
  scale_rows(ctx, d, t.p);
  scatter_m(ctx, d, d.rho, vrho.dev);
  if (ahat && d.nnz)
    LPK_LAUNCH(ctx, k_ahat_to_input, (int)((d.nnz + 255) / 256), 256, 0, ctx->stream, d.nnz, d.src, d.ah64, vah.dev);
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  TRY(vrho.finish());
  TRY(vah.finish());
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  return LPK_OK;
}

LPK_API lpk_status lpk_spmv(lpk_ctx *ctx, lpk_problem *P, int32_t transpose, const double *x, double *y,
                            int32_t on_device) {
  CHECK_CTX(ctx);
  CHECK_P(ctx, P);
  DevProblem &d = P->d;
  if (!x || !y) return LPK_INVALID_ARG;
  const size_t lx = transpose ? d.m_in : d.n_in, ly = transpose ? d.n_in : d.m_in;
  Vec vx(ctx, x, lx, on_device, false), vy(ctx, y, ly, on_device, true);
  TRY(vx.init());
  TRY(vy.init());
  DevBuf a(ctx), b(ctx);
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &a.p, d.m + d.n + 2));
  b.p = nullptr;
  double *tm = a.p, *tn = a.p + d.m + 1;
  if (!ctx->ev0) {
    LPK_CUDA_TRY(ctx, cudaEventCreate(&ctx->ev0));
    LPK_CUDA_TRY(ctx, cudaEventCreate(&ctx->ev1));
  }
  // the product kernel is timed alone (events on the context stream)
  if (transpose) {
    gather_m(ctx, d, vx.dev, tm);
    LPK_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
    spmv_csc(ctx, d, tm, tn);
    LPK_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    scatter_n(ctx, d, tn, vy.dev, nullptr);
  } else {
    gather_n(ctx, d, vx.dev, tn);
    LPK_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
    spmv_csr(ctx, d, tn, tm, nullptr, 1.0);
    LPK_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    scatter_m(ctx, d, tm, vy.dev);
  }
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  TRY(vy.finish());
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  float ms = 0.f;
  LPK_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  ctx->stats.spmv_launches++;
  ctx->stats.spmv_ms += ms;
  return LPK_OK;
}

LPK_API lpk_status lpk_sweep(lpk_ctx *ctx, lpk_problem *P, const double *d2, const double *g, int32_t kind,
                             int32_t inner_sweeps, double omega, int32_t precision, double *z, double *u,
                             int32_t on_device) {
  CHECK_CTX(ctx);
  CHECK_P(ctx, P);
  DevProblem &d = P->d;
  if (!d2 || !g || !z || !u || inner_sweeps < 1 || !(omega > 0.0 && omega < 2.0) ||
      (kind != LPK_NE_SSOR && kind != LPK_NE_SOR) || (precision != LPK_FP64 && precision != LPK_MIXED)) {
    ctx->err = "lpk_sweep: invalid arguments";
    return LPK_INVALID_ARG;
  }
  Vec vd2(ctx, d2, d.n_in, on_device, false), vg(ctx, g, d.m_in, on_device, false),
      vz(ctx, z, d.m_in, on_device, true), vu(ctx, u, d.n_in, on_device, true);
  TRY(vd2.init());
  TRY(vg.init());
  TRY(vz.init());
  TRY(vu.init());
  DevBuf t(ctx);
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &t.p, 2 * d.m + 2 * d.n + 4));
  double *td2 = t.p, *tg = td2 + d.n + 1, *tz = tg + d.m + 1, *tu = tz + d.m + 1;
  gather_n(ctx, d, vd2.dev, td2);
  TRY(check_d2(ctx, d, td2));
  scale_rows(ctx, d, td2);
  gather_m(ctx, d, vg.dev, tg);
  TRY(sweep_only(ctx, d, kind, precision, inner_sweeps, omega, tg, tz, tu));
  scatter_m(ctx, d, tz, vz.dev);
  scatter_n(ctx, d, tu, vu.dev, nullptr);
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  TRY(vz.finish());
  TRY(vu.finish());
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  return LPK_OK;
}

LPK_API lpk_status lpk_ne_solve(lpk_ctx *ctx, lpk_problem *P, const double *d2, const double *f,
                                int32_t inner_sweeps, double omega, int32_t solver, int32_t precision, double tol,
                                int32_t max_iter, double *dy, double *dw, lpk_krylov_info *kinfo,
                                int32_t on_device) {
  CHECK_CTX(ctx);
  CHECK_P(ctx, P);
  DevProblem &d = P->d;
  if (!d2 || !f || !dy || inner_sweeps < 1 || !(omega > 0.0 && omega < 2.0) || !(tol >= 0.0) ||
      max_iter < 0 || (solver != LPK_MRNE && solver != LPK_CGNE && solver != LPK_ABGMRES) ||
      (precision != LPK_FP64 && precision != LPK_MIXED)) {
    ctx->err = "lpk_ne_solve: invalid arguments";
    return LPK_INVALID_ARG;
  }
  Vec vd2(ctx, d2, d.n_in, on_device, false), vf(ctx, f, d.m_in, on_device, false),
      vdy(ctx, dy, d.m_in, on_device, true), vdw(ctx, dw, d.n_in, on_device, true);
  TRY(vd2.init());
  TRY(vf.init());
  TRY(vdy.init());
  TRY(vdw.init());
  DevBuf t(ctx);
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &t.p, 3 * d.m + 2 * d.n + 5));
  double *td2 = t.p, *tf = td2 + d.n + 1, *tdy = tf + d.m + 1, *tdw = tdy + d.m + 1, *tmp = tdw + d.n + 1;
  gather_n(ctx, d, vd2.dev, td2);
  TRY(check_d2(ctx, d, td2));
  gather_m(ctx, d, vf.dev, tf);
  scale_rows(ctx, d, td2);
  KrylovResult kr;
  const int maxit = max_iter > 0 ? max_iter : d.m;
  TRY(ne_solve_scaled(ctx, d, tf, inner_sweeps, omega, solver, precision, tol, maxit, tdy, tdw, tmp, &kr));
  scatter_m(ctx, d, tdy, vdy.dev);
  if (dw) scatter_n(ctx, d, tdw, vdw.dev, nullptr);
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  TRY(vdy.finish());
  TRY(vdw.finish());
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  if (kinfo) {
    kinfo->iters = kr.iters;
    kinfo->converged = kr.converged;
    kinfo->restarts = kr.restarts;
    kinfo->breakdown = kr.breakdown;
    kinfo->res0 = kr.res0;
    kinfo->res = kr.res;
  }
  return LPK_OK;
}

namespace {
__global__ void k_sqrt_mul(int n, const double *d2, const double *r, double *out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = sqrt(d2[j]) * r[j];
}
}  // namespace

LPK_API lpk_status lpk_ls_solve(lpk_ctx *ctx, lpk_problem *P, const double *d2, const double *r,
                                int32_t inner_sweeps, double omega, int32_t precision, double tol,
                                int32_t max_iter, double *dy, double *dw, lpk_krylov_info *kinfo,
                                int32_t on_device) {
  CHECK_CTX(ctx);
  CHECK_P(ctx, P);
  DevProblem &d = P->d;
  if (!d2 || !r || !dy || inner_sweeps < 1 || !(omega > 0.0 && omega < 2.0) || !(tol >= 0.0) ||
      max_iter < 0 || (precision != LPK_FP64 && precision != LPK_MIXED)) {
    ctx->err = "lpk_ls_solve: invalid arguments";
    return LPK_INVALID_ARG;
  }
  Vec vd2(ctx, d2, d.n_in, on_device, false), vr(ctx, r, d.n_in, on_device, false),
      vdy(ctx, dy, d.m_in, on_device, true), vdw(ctx, dw, d.n_in, on_device, true);
  TRY(vd2.init());
  TRY(vr.init());
  TRY(vdy.init());
  TRY(vdw.init());
  DevBuf t(ctx);
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &t.p, 3 * d.m + 4 * d.n + 7));
  double *td2 = t.p, *tr = td2 + d.n + 1, *tt = tr + d.n + 1, *tf = tt + d.n + 1, *tdy = tf + d.m + 1,
         *tdw = tdy + d.m + 1, *tmp = tdw + d.n + 1;
  gather_n(ctx, d, vd2.dev, td2);
  TRY(check_d2(ctx, d, td2));
  gather_n(ctx, d, vr.dev, tr);
  scale_rows(ctx, d, td2);
  // f = A D r, the right-hand side of the equivalent normal equations
  if (d.n > 0) LPK_LAUNCH(ctx, k_sqrt_mul, (d.n + 255) / 256, 256, 0, ctx->stream, d.n, td2, tr, tt);
  spmv_csr(ctx, d, tt, tf, nullptr, 1.0);
  KrylovResult kr;
  const int maxit = max_iter > 0 ? max_iter : d.m;
  TRY(ls_solve_scaled(ctx, d, tr, tf, inner_sweeps, omega, precision, tol, maxit, tdy, tdw, tmp, &kr));
  scatter_m(ctx, d, tdy, vdy.dev);
  if (dw) scatter_n(ctx, d, tdw, vdw.dev, nullptr);
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  TRY(vdy.finish());
  TRY(vdw.finish());
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  if (kinfo) {
    kinfo->iters = kr.iters;
    kinfo->converged = kr.converged;
    kinfo->restarts = kr.restarts;
    kinfo->breakdown = kr.breakdown;
    kinfo->res0 = kr.res0;
    kinfo->res = kr.res;
  }
  return LPK_OK;
}

LPK_API lpk_status lpk_lp_solve(lpk_ctx *ctx, lpk_problem *P, const double *b, const double *c,
                                const lpk_options *opt, double *x, double *y, double *s, lpk_info *info,
                                int32_t on_device) {
  CHECK_CTX(ctx);
  CHECK_P(ctx, P);
  DevProblem &d = P->d;
  lpk_options o;
  if (opt) o = *opt;
  else lpk_default_options(&o);
  if (!b || !c || !x || !y || !s || o.inner_sweeps < 1 || !(o.omega > 0.0 && o.omega < 2.0) ||
      !(o.eta > 0.0 && o.eta < 1.0) || o.max_ipm < 0 || o.max_krylov < 0 ||
      (o.solver != LPK_MRNE && o.solver != LPK_CGNE && o.solver != LPK_ABGMRES) ||
      (o.corrector != 0 && o.corrector != 1) || o.max_correctors < 0 || o.max_correctors > 10 ||
      (o.precision != LPK_FP64 && o.precision != LPK_MIXED)) {
    ctx->err = "lpk_lp_solve: invalid arguments";
    return LPK_INVALID_ARG;
  }
  Vec vb(ctx, b, d.m_in, on_device, false), vc(ctx, c, d.n_in, on_device, false),
      vx(ctx, x, d.n_in, on_device, true), vy(ctx, y, d.m_in, on_device, true), vs(ctx, s, d.n_in, on_device, true);
  TRY(vb.init());
  TRY(vc.init());
  TRY(vx.init());
  TRY(vy.init());
  TRY(vs.init());
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, ctx->stream);
  lpk_info inf;
  lpk_status st = lp_solve_dev(ctx, d, vb.dev, vc.dev, o, vx.dev, vy.dev, vs.dev, inf);
  cudaEventRecord(e1, ctx->stream);
  ctx_sync(ctx);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  inf.solve_ms = ms;
  if (info) *info = inf;
  if (st == LPK_OK || st == LPK_MAX_IPM_ITER || st == LPK_DIVERGED) {
    TRY(vx.finish());
    TRY(vy.finish());
    TRY(vs.finish());
    LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  }
  return st;
}
