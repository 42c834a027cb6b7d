// ipm_kernels.cu -- sparse products, row scaling and the fused elementwise
// kernels of the interior-point step.  All m-space vectors are in sweep
// (color-permuted) order, all n-space vectors in kept-column order.
#include "ipm_kernels.cuh"

namespace {

constexpr int TPB = 256;
inline int wblk(long long rows, int tpb = TPB) { return (int)((rows * 32 + tpb - 1) / tpb); }
inline int tblk(long long n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

template <int LPR>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, LPR);
  return v;
}

// ---- Sec. 3.5 row scaling --------------------------------------------------
// d_j = sqrt(d2_j), rho_i = ||(A D)_i||_2, ahat = a_ij d_j / rho_i (FP64 and FP32).
// Square roots and divisions are multi-instruction FP64 sequences, and FP64
// is scarce on this GPU: d is taken once per column (k_sqrt), 1 / rho once per
// row, and every entry is (a_ij d_j) * (1 / rho_i) -- within an ulp or two of
// the quotient.  The CSC copy is a gather of the CSR entries.
__global__ void k_sqrt(int n, const double *__restrict__ d2, double *__restrict__ d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) d[j] = sqrt(d2[j]);
}

template <int LPR>
__global__ void k_scale(int m, const int *__restrict__ rp, const int *__restrict__ ci,
                        const double *__restrict__ a, const double *__restrict__ d,
                        double *__restrict__ ah64, float *__restrict__ ah32, double *__restrict__ rho) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = (int)(t / LPR), sub = (int)(t % LPR);
  int k0 = 0, k1 = 0;
  double s = 0.0;
  if (r < m) {
    k0 = __ldg(rp + r);
    k1 = __ldg(rp + r + 1);
    for (int k = k0 + sub; k < k1; k += LPR) {
      const double e = __ldg(a + k) * __ldg(d + __ldg(ci + k));
      s += e * e;
    }
  }
  s = group_sum<LPR>(s);  // every lane of the warp takes part
  if (r >= m) return;
  const double nr = sqrt(s);
  const double ri = nr > 0.0 ? 1.0 / nr : 0.0;
  for (int k = k0 + sub; k < k1; k += LPR) {
    const double v = (__ldg(a + k) * __ldg(d + __ldg(ci + k))) * ri;
    ah64[k] = v;
    ah32[k] = (float)v;
  }
  if (sub == 0) rho[r] = nr;
}

// the same scaled entries in CSC order, copied from their CSR positions (so
// bitwise equal); a thread per entry, whatever the column lengths
__global__ void k_scale_csc(long long nnz, const int *__restrict__ cpos, const double *__restrict__ ah64,
                            double *__restrict__ aht) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nnz) aht[q] = ah64[__ldg(cpos + q)];
}

// Sparse products with LPR lanes per row (or column): short rows leave most
// of a warp idle with one row per warp, so a warp takes 32 / LPR rows at once
// (more independent loads in flight per warp); the partial sums of a row are
// combined by shuffles inside its LPR-lane group, in a fixed order.

// y = sign * A x + add.  A group of LPR lanes per row; each lane walks the
// row's entries lane, lane + LPR, ... four at a time: the four (index, value)
// loads and then the four gathers of x are issued before the first
// multiply-add, so a lane has several independent loads in flight instead of
// one dependent chain per entry.  The multiply-adds stay in entry order, so
// the sums are those of the one-entry-at-a-time loop.
template <int LPR>
__global__ void k_spmv_csr(int m, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ a, const double *__restrict__ x,
                           double *__restrict__ y, const double *__restrict__ add, double sign) {
  constexpr int U = 4;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = (int)(t / LPR), sub = (int)(t % LPR);
  double s = 0.0;
  if (r < m) {
    const int k1 = __ldg(rp + r + 1);
    for (int k = __ldg(rp + r) + sub; k < k1; k += U * LPR) {
      int c[U];
      double av[U], xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = k + u * LPR;
        c[u] = kk < k1 ? __ldg(ci + kk) : 0;
        av[u] = kk < k1 ? __ldcs(a + kk) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = k + u * LPR < k1 ? __ldg(x + c[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k + u * LPR < k1) s += av[u] * xv[u];
    }
  }
  s = group_sum<LPR>(s);  // every lane of the warp takes part
  if (r < m && sub == 0) y[r] = add ? sign * s + add[r] : (sign == 1.0 ? s : sign * s);
}

// y = A^T x through the CSC, organised as k_spmv_csr
template <int LPR>
__global__ void k_spmv_csc(int n, const int *__restrict__ cp, const int *__restrict__ ri,
                           const double *__restrict__ at, const double *__restrict__ x,
                           double *__restrict__ y) {
  constexpr int U = 4;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = (int)(t / LPR), sub = (int)(t % LPR);
  double s = 0.0;
  if (j < n) {
    const int q1 = __ldg(cp + j + 1);
    for (int q = __ldg(cp + j) + sub; q < q1; q += U * LPR) {
      int c[U];
      double av[U], xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int qq = q + u * LPR;
        c[u] = qq < q1 ? __ldg(ri + qq) : 0;
        av[u] = qq < q1 ? __ldcs(at + qq) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = q + u * LPR < q1 ? __ldg(x + c[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (q + u * LPR < q1) s += av[u] * xv[u];
    }
  }
  s = group_sum<LPR>(s);
  if (j < n && sub == 0) y[j] = s;
}

// Lanes per row from the mean row length.  Each level of the group's shuffle
// reduction is one FP64 add per row, and an FP64 warp instruction occupies a
// sub-partition's FP64 pipe for tens of cycles on this GPU, so the group is
// kept narrow (about four entries per lane) rather than one entry per lane.
inline int lanes_for(long long nnz, long long rows) {
  const long long avg = rows > 0 ? (nnz + rows - 1) / rows : 0;
  return avg <= 8 ? 2 : avg <= 32 ? 4 : avg <= 64 ? 8 : avg <= 128 ? 16 : 32;
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
  cudaStream_t s = ctx->stream;
  if (P.n > 0) LPK_LAUNCH(ctx, k_sqrt, tblk(P.n), TPB, 0, s, P.n, d2, P.dcol);
  if (P.m > 0) {
    switch (lanes_for(P.nnz, P.m)) {
      case 2: LPK_LAUNCH(ctx, k_scale<2>, gblk(P.m, 2), TPB, 0, s, P.m, P.rp, P.ci, P.a, P.dcol, P.ah64, P.ah32, P.rho); break;
      case 4: LPK_LAUNCH(ctx, k_scale<4>, gblk(P.m, 4), TPB, 0, s, P.m, P.rp, P.ci, P.a, P.dcol, P.ah64, P.ah32, P.rho); break;
      case 8: LPK_LAUNCH(ctx, k_scale<8>, gblk(P.m, 8), TPB, 0, s, P.m, P.rp, P.ci, P.a, P.dcol, P.ah64, P.ah32, P.rho); break;
      case 16: LPK_LAUNCH(ctx, k_scale<16>, gblk(P.m, 16), TPB, 0, s, P.m, P.rp, P.ci, P.a, P.dcol, P.ah64, P.ah32, P.rho); break;
      default: LPK_LAUNCH(ctx, k_scale<32>, gblk(P.m, 32), TPB, 0, s, P.m, P.rp, P.ci, P.a, P.dcol, P.ah64, P.ah32, P.rho); break;
    }
  }
  if (P.nnz > 0) LPK_LAUNCH(ctx, k_scale_csc, tblk(P.nnz), TPB, 0, s, P.nnz, P.cpos, P.ah64, P.aht);
}
void spmv_csr(lpk_ctx *ctx, const DevProblem &P, const double *x, double *y, const double *add, double sign) {
  if (P.m <= 0) return;
  cudaStream_t s = ctx->stream;
  switch (lanes_for(P.nnz, P.m)) {
    case 2: LPK_LAUNCH(ctx, k_spmv_csr<2>, gblk(P.m, 2), TPB, 0, s, P.m, P.rp, P.ci, P.a, x, y, add, sign); break;
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
    case 2: LPK_LAUNCH(ctx, k_spmv_csc<2>, gblk(P.n, 2), TPB, 0, s, P.n, P.cp, P.ri, P.at, x, y); break;
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
