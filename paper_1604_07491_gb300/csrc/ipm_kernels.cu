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

// Sparse products with LPR lanes per row (or column): short rows leave most
// of a warp idle with one row per warp, so a warp takes 32 / LPR rows at once
// (more independent loads in flight per warp); the partial sums of a row are
// combined by shuffles inside its LPR-lane group, in a fixed order.
template <int LPR>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, LPR);
  return v;
}

// y = sign * A x + add
template <int LPR>
__global__ void k_spmv_csr(int m, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ a, const double *__restrict__ x,
                           double *__restrict__ y, const double *__restrict__ add, double sign) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = (int)(t / LPR), sub = (int)(t % LPR);
  double s = 0.0;
  if (r < m)
    for (int k = __ldg(rp + r) + sub, k1 = __ldg(rp + r + 1); k < k1; k += LPR) s += __ldg(a + k) * __ldg(x + __ldg(ci + k));
  s = group_sum<LPR>(s);  // every lane of the warp takes part
  if (r < m && sub == 0) y[r] = sign * s + (add ? add[r] : 0.0);
}

// y = A^T x through the CSC
template <int LPR>
__global__ void k_spmv_csc(int n, const int *__restrict__ cp, const int *__restrict__ ri,
                           const double *__restrict__ at, const double *__restrict__ x,
                           double *__restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = (int)(t / LPR), sub = (int)(t % LPR);
  double s = 0.0;
  if (j < n)
    for (int q = __ldg(cp + j) + sub, q1 = __ldg(cp + j + 1); q < q1; q += LPR) s += __ldg(at + q) * __ldg(x + __ldg(ri + q));
  s = group_sum<LPR>(s);
  if (j < n && sub == 0) y[j] = s;
}

// lanes per row from the mean row length
inline int lanes_for(long long nnz, long long rows) {
  const long long avg = rows > 0 ? (nnz + rows - 1) / rows : 0;
  return avg <= 8 ? 4 : avg <= 24 ? 8 : avg <= 64 ? 16 : 32;
}
inline int gblk(long long rows, int lpr, int tpb = TPB) { return (int)((rows * lpr + tpb - 1) / tpb); }

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
  if (P.m <= 0) return;
  cudaStream_t s = ctx->stream;
  switch (lanes_for(P.nnz, P.m)) {
    case 4: LPK_LAUNCH(ctx, k_spmv_csr<4>, gblk(P.m, 4), TPB, 0, s, P.m, P.rp, P.ci, P.a, x, y, add, sign); break;
    case 8: LPK_LAUNCH(ctx, k_spmv_csr<8>, gblk(P.m, 8), TPB, 0, s, P.m, P.rp, P.ci, P.a, x, y, add, sign); break;
    case 16: LPK_LAUNCH(ctx, k_spmv_csr<16>, gblk(P.m, 16), TPB, 0, s, P.m, P.rp, P.ci, P.a, x, y, add, sign); break;
    default: LPK_LAUNCH(ctx, k_spmv_csr<32>, gblk(P.m, 32), TPB, 0, s, P.m, P.rp, P.ci, P.a, x, y, add, sign); break;
  }
}
void spmv_csc(lpk_ctx *ctx, const DevProblem &P, const double *x, double *y) {
  if (P.n <= 0) return;
  cudaStream_t s = ctx->stream;
  switch (lanes_for(P.nnz, P.n)) {
    case 4: LPK_LAUNCH(ctx, k_spmv_csc<4>, gblk(P.n, 4), TPB, 0, s, P.n, P.cp, P.ri, P.at, x, y); break;
    case 8: LPK_LAUNCH(ctx, k_spmv_csc<8>, gblk(P.n, 8), TPB, 0, s, P.n, P.cp, P.ri, P.at, x, y); break;
    case 16: LPK_LAUNCH(ctx, k_spmv_csc<16>, gblk(P.n, 16), TPB, 0, s, P.n, P.cp, P.ri, P.at, x, y); break;
    default: LPK_LAUNCH(ctx, k_spmv_csc<32>, gblk(P.n, 32), TPB, 0, s, P.n, P.cp, P.ri, P.at, x, y); break;
  }
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
