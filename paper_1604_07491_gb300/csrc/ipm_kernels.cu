// ipm_kernels.cu -- sparse products, row scaling and the fused elementwise
// kernels of the interior-point step.  All m-space vectors are in sweep
// (color-permuted) order, all n-space vectors in kept-column order.
#include "ipm_kernels.cuh"

namespace {

constexpr int TPB = 256;
inline int wblk(long long rows, int tpb = TPB) { return (int)((rows * 32 + tpb - 1) / tpb); }
inline int tblk(long long n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

// ---- Sec. 3.5 row scaling --------------------------------------------------
// d_j = sqrt(d2_j), rho_i = ||(A D)_i||_2, ahat = a_ij d_j / rho_i (FP64 and FP32)
__global__ void k_scale(int m, const int *__restrict__ rp, const int *__restrict__ ci,
                        const double *__restrict__ a, const double *__restrict__ d2,
                        double *__restrict__ ah64, float *__restrict__ ah32, double *__restrict__ rho) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= m) return;
  const int k0 = rp[r], k1 = rp[r + 1];
  double s = 0.0;
  for (int k = k0 + lane; k < k1; k += 32) {
    double e = a[k] * sqrt(d2[ci[k]]);
    s += e * e;
  }
  s = warp_sum(s);
  const double nr = sqrt(s);
  for (int k = k0 + lane; k < k1; k += 32) {
    double e = a[k] * sqrt(d2[ci[k]]);
    double v = nr > 0.0 ? e / nr : 0.0;
    ah64[k] = v;
    ah32[k] = (float)v;
  }
  if (lane == 0) rho[r] = nr;
}

// the same scaled entries in CSC order: identical expression, so bitwise equal
__global__ void k_scale_csc(int n, const int *__restrict__ cp, const int *__restrict__ ri,
                            const double *__restrict__ at, const double *__restrict__ d2,
                            const double *__restrict__ rho, double *__restrict__ aht) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double dj = sqrt(d2[j]);
  for (int q = cp[j]; q < cp[j + 1]; ++q) {
    const double e = at[q] * dj;
    const double nr = rho[ri[q]];
    aht[q] = nr > 0.0 ? e / nr : 0.0;
  }
}

// y = sign * A x + add  (warp per row)
__global__ void k_spmv_csr(int m, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ a, const double *__restrict__ x,
                           double *__restrict__ y, const double *__restrict__ add, double sign) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= m) return;
  double s = 0.0;
  for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) s += a[k] * x[ci[k]];
  s = warp_sum(s);
  if (lane == 0) y[r] = sign * s + (add ? add[r] : 0.0);
}

// y = A^T x through the CSC (warp per column)
__global__ void k_spmv_csc(int n, const int *__restrict__ cp, const int *__restrict__ ri,
                           const double *__restrict__ at, const double *__restrict__ x,
                           double *__restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  double s = 0.0;
  for (int q = cp[j] + lane; q < cp[j + 1]; q += 32) s += at[q] * x[ri[q]];
  s = warp_sum(s);
  if (lane == 0) y[j] = s;
}

__global__ void k_gather(int len, const int *__restrict__ idx, const double *__restrict__ in,
                         double *__restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = in[idx[i]];
}
__global__ void k_scatter(int len, const int *__restrict__ idx, const double *__restrict__ in,
                          double *__restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[idx[i]] = in[i];
}
// out[j] = fill[j] for every input column j (used before scattering kept columns)
__global__ void k_copy(int len, const double *__restrict__ in, double *__restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = in[i];
}
__global__ void k_fill(int len, double v, double *__restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = v;
}

}  // namespace

// ---------------------------------------------------------------------------
void scale_rows(lpk_ctx *ctx, DevProblem &P, const double *d2) {
  if (P.m > 0) LPK_LAUNCH(ctx, k_scale, wblk(P.m), TPB, 0, ctx->stream, P.m, P.rp, P.ci, P.a, d2, P.ah64, P.ah32, P.rho);
  if (P.n > 0) LPK_LAUNCH(ctx, k_scale_csc, tblk(P.n), TPB, 0, ctx->stream, P.n, P.cp, P.ri, P.at, d2, P.rho, P.aht);
}
void spmv_csr(lpk_ctx *ctx, const DevProblem &P, const double *x, double *y, const double *add, double sign) {
  if (P.m > 0) LPK_LAUNCH(ctx, k_spmv_csr, wblk(P.m), TPB, 0, ctx->stream, P.m, P.rp, P.ci, P.a, x, y, add, sign);
}
void spmv_csc(lpk_ctx *ctx, const DevProblem &P, const double *x, double *y) {
  if (P.n > 0) LPK_LAUNCH(ctx, k_spmv_csc, wblk(P.n), TPB, 0, ctx->stream, P.n, P.cp, P.ri, P.at, x, y);
}
void gather_m(lpk_ctx *ctx, const DevProblem &P, const double *in, double *out) {
  if (P.m > 0) LPK_LAUNCH(ctx, k_gather, tblk(P.m), TPB, 0, ctx->stream, P.m, P.in_row_of_pos, in, out);
}
void scatter_m(lpk_ctx *ctx, const DevProblem &P, const double *in, double *out) {
  if (P.m_in > P.m) LPK_LAUNCH(ctx, k_fill, tblk(P.m_in), TPB, 0, ctx->stream, P.m_in, 0.0, out);
  if (P.m > 0) LPK_LAUNCH(ctx, k_scatter, tblk(P.m), TPB, 0, ctx->stream, P.m, P.in_row_of_pos, in, out);
}
void gather_n(lpk_ctx *ctx, const DevProblem &P, const double *in, double *out) {
  if (P.n > 0) LPK_LAUNCH(ctx, k_gather, tblk(P.n), TPB, 0, ctx->stream, P.n, P.in_col_of, in, out);
}
void scatter_n(lpk_ctx *ctx, const DevProblem &P, const double *in, double *out, const double *fill) {
  if (P.n_in > P.n) {
    if (fill)
      LPK_LAUNCH(ctx, k_copy, tblk(P.n_in), TPB, 0, ctx->stream, P.n_in, fill, out);
    else
      LPK_LAUNCH(ctx, k_fill, tblk(P.n_in), TPB, 0, ctx->stream, P.n_in, 0.0, out);
  }
  if (P.n > 0) LPK_LAUNCH(ctx, k_scatter, tblk(P.n), TPB, 0, ctx->stream, P.n, P.in_col_of, in, out);
}

// ---------------------------------------------------------------------------
// deterministic two-stage reductions
// ---------------------------------------------------------------------------
lpk_status ensure_reduce(lpk_ctx *ctx) {
  if (ctx->red_part) return LPK_OK;
  ctx->red_blocks = 2 * ctx->num_sms;
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &ctx->red_part, (size_t)RED_MAX_SLOTS * ctx->red_blocks));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &ctx->red_count, 1));
  LPK_CUDA_TRY(ctx, cudaMemsetAsync(ctx->red_count, 0, sizeof(unsigned), ctx->stream));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &ctx->red_out, RED_MAX_SLOTS));
  LPK_CUDA_TRY(ctx, cudaMallocHost(&ctx->h_red, sizeof(double) * RED_MAX_SLOTS));
  return LPK_OK;
}

lpk_status red_fetch(lpk_ctx *ctx, int nslots) {
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_red, ctx->red_out, sizeof(double) * nslots, cudaMemcpyDeviceToHost,
                                    ctx->stream));
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  return LPK_OK;
}

RedArgs red_args(lpk_ctx *ctx) { return RedArgs{ctx->red_part, ctx->red_count, ctx->red_out}; }
int red_grid(lpk_ctx *ctx) { return ctx->red_blocks; }
