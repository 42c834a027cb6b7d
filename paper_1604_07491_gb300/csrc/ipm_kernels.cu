// ipm_kernels.cu -- sparse products, row scaling and the fused elementwise
// kernels of the interior-point step.  All m-space vectors are in sweep
// (color-permuted) order, all n-space vectors in kept-column order.
#include "ipm_kernels.cuh"

namespace {

constexpr int TPB = 256;
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

// Lanes per row for the row scaling, from the mean row length.  Each level
// of the group's shuffle reduction is one FP64 add per row, and an FP64 warp
// instruction occupies a sub-partition's FP64 pipe for tens of cycles on this
// GPU, so the group is kept narrow (about four entries per lane).
inline int lanes_for(long long nnz, long long rows) {
  const long long avg = rows > 0 ? (nnz + rows - 1) / rows : 0;
  return avg <= 8 ? 2 : avg <= 32 ? 4 : avg <= 64 ? 8 : avg <= 128 ? 16 : 32;
}
inline int gblk(long long rows, int lpr, int tpb = TPB) { return (int)((rows * lpr + tpb - 1) / tpb); }

// ---- sparse products y = sign * A x + add and y = A^T x ---------------------
// Balanced over entries, not rows: warp w takes the SEG_CH = 32 SEG_K entries
// [w SEG_CH, (w + 1) SEG_CH) of the compressed arrays and lane l the SEG_K
// consecutive entries from w SEG_CH + l SEG_K.  FP64 issue, not DRAM, bounds
// these products on this GPU (an FP64 warp instruction holds a
// sub-partition's FP64 pipe for tens of cycles whatever its active lanes), and
// with a lane group per row short and ragged rows leave most lanes of every
// multiply-add idle.  Here every multiply-add instruction has all its lanes
// busy.  A lane's multiply-adds run in entry order and restart at each row
// start; a row that crosses lanes is combined by a segmented shuffle scan
// keyed by row (lanes in order), a row that crosses warps by k_seg_fix
// (chunks in order).  The result does not depend on scheduling.
//
// seg_first[w] is the first row (or column) that starts at or after entry
// w SEG_CH, seg_first[nw] = rows; it is built once per problem (k_seg_first).
constexpr int SEG_WPB = TPB / 32;

__global__ void k_seg_first(int rows, const int *__restrict__ rp, int nw, int *__restrict__ first) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w > nw) return;
  if (w == nw) {
    first[w] = rows;
    return;
  }
  const long long e = (long long)w * SEG_CH;
  int lo = 0, hi = rows;  // first r in [0, rows) with rp[r] >= e, else rows
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (rp[mid] < e) lo = mid + 1;
    else hi = mid;
  }
  first[w] = lo;
}

__device__ __forceinline__ double seg_out(double v, const double *add, int r, double sign) {
  return add ? sign * v + add[r] : (sign == 1.0 ? v : sign * v);
}

// a matrix without entries: every row is empty
__global__ void k_seg_empty(int rows, double *__restrict__ y, const double *__restrict__ add, double sign) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) y[r] = seg_out(0.0, add, r, sign);
}

// VEC: the value and index arrays are 16-byte aligned (vector loads)
template <bool VEC>
__global__ void __launch_bounds__(TPB) k_seg_spmv(int rows, long long nnz, const int *__restrict__ rp,
                                                  const int *__restrict__ ci, const double *__restrict__ a,
                                                  const int *__restrict__ first, int nw,
                                                  const double *__restrict__ x, double *__restrict__ y,
                                                  const double *__restrict__ add, double sign,
                                                  double *__restrict__ carry) {
  constexpr int K = SEG_K, CH = SEG_CH;
  constexpr unsigned FULL = 0xffffffffu;
  // per warp, entry q of the chunk at [(q % K) * 32 + q / K] (lane-major, no
  // bank conflicts): the row starting at q (-1: none), and each lane's list
  // of finished rows
  __shared__ int s_start[SEG_WPB][CH];
  __shared__ int s_row[SEG_WPB][CH];
  __shared__ double s_val[SEG_WPB][CH];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.x * SEG_WPB + wib;
  if (w >= nw) return;  // whole warps
  int *st = s_start[wib], *lr = s_row[wib];
  double *lv = s_val[wib];
  const long long e0 = (long long)w * CH;
  const int len = (int)(nnz - e0 < CH ? nnz - e0 : CH);
  const int q0 = lane * K;
  const int nv = len - q0 < 0 ? 0 : (len - q0 < K ? len - q0 : K);  // entries of this lane
  // the loads are issued in dependency order so that their round trips
  // overlap: chunk index, entries (index, value), row pointers, then the
  // gathers of x
  const int ra = __ldg(first + w), rb = __ldg(first + w + 1);
  int cv[K];
  double av[K], xv[K];
  const long long p0 = e0 + q0;
  if (VEC && nv == K) {
#pragma unroll
    for (int j = 0; j < K; j += 4) {
      const int4 c4 = __ldg(reinterpret_cast<const int4 *>(ci + p0 + j));
      cv[j] = c4.x;
      cv[j + 1] = c4.y;
      cv[j + 2] = c4.z;
      cv[j + 3] = c4.w;
    }
#pragma unroll
    for (int j = 0; j < K; j += 2) {
      const double2 a2 = __ldg(reinterpret_cast<const double2 *>(a + p0 + j));
      av[j] = a2.x;
      av[j + 1] = a2.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      cv[j] = j < nv ? __ldg(ci + p0 + j) : 0;
      av[j] = j < nv ? __ldg(a + p0 + j) : 0.0;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) xv[j] = j < nv ? __ldg(x + cv[j]) : 0.0;
#pragma unroll
  for (int j = 0; j < K; ++j) st[j * 32 + lane] = -1;
  __syncwarp();
  // rows starting in this chunk: mark their first entries
  for (int r = ra + lane; r < rb; r += 32) {
    const int p = __ldg(rp + r);
    if (__ldg(rp + r + 1) > p) {
      const int q = (int)(p - e0);
      st[(q % K) * 32 + q / K] = r;
    } else {
      y[r] = seg_out(0.0, add, r, sign);  // empty row
    }
  }
  // the row holding entry e0 began in an earlier chunk
  const bool cont = ra >= rows || __ldg(rp + ra) > e0;
  const int head_row = cont ? ra - 1 : -1;
  __syncwarp();

  int mark[K];
  int last = -1;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    mark[j] = st[j * 32 + lane];
    last = max(last, mark[j]);
  }
  // the lane's incoming row: the latest start before its first entry
  // (rows grow with the entry index, so a max-scan over the lanes)
  int inc = last;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc = max(inc, v);
  }
  int incoming = __shfl_up_sync(FULL, inc, 1);
  if (lane == 0 || incoming < 0) incoming = head_row;

  // the lane's entries in order: a start ends the current row's run
  int cur = incoming, nst = 0, cnt = 0;
  double s = 0.0, head_part = 0.0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (mark[j] >= 0) {
      if (nst == 0) {
        head_part = s;  // the incoming row's entries in this lane
      } else {
        lr[cnt * 32 + lane] = cur;  // a row wholly inside this lane
        lv[cnt * 32 + lane] = s;
        ++cnt;
      }
      ++nst;
      cur = mark[j];
      s = 0.0;
    }
    if (j < nv) s = fma(av[j], xv[j], s);
  }

  // segmented inclusive scan of the lanes' last runs, keyed by row
  const int key = nv > 0 ? cur : -2;
  double S = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double v = __shfl_up_sync(FULL, S, o);
    const int k = __shfl_up_sync(FULL, key, o);
    if (lane >= o && k == key) S += v;
  }
  const double S_prev = __shfl_up_sync(FULL, S, 1);
  const int key_prev = __shfl_up_sync(FULL, key, 1);
  const bool next_starts = __shfl_down_sync(FULL, mark[0] >= 0, 1);
  if (nv > 0 && nst > 0 && mark[0] < 0 && incoming >= 0) {
    // the lane ends its incoming row: the earlier lanes' sum plus its own run
    // (a row that ends at a lane boundary is ended by the lane before)
    const double tot = (lane > 0 && key_prev == incoming ? S_prev : 0.0) + head_part;
    if (cont && incoming == head_row) {
      carry[w] = tot;  // the rest of a row begun in an earlier chunk
    } else {
      lr[cnt * 32 + lane] = incoming;
      lv[cnt * 32 + lane] = tot;
      ++cnt;
    }
  }
  const bool last_lane = q0 + K >= len;
  if (nv > 0 && (last_lane || next_starts)) {
    // the lane's last row ends here (or at the chunk's end): its sum over
    // the chunk so far is S
    const bool more = last_lane && e0 + len < nnz && (rb >= rows || __ldg(rp + rb) > e0 + len);
    if (cont && cur == head_row) {
      carry[w] = S;  // no row starts in this chunk before this point
    } else if (more) {
      y[cur] = S;  // continues in the next chunk: k_seg_fix adds the rest
    } else {
      lr[cnt * 32 + lane] = cur;
      lv[cnt * 32 + lane] = S;
      ++cnt;
    }
  }
  if (add == nullptr && sign == 1.0) {
    for (int c = 0; c < cnt; ++c) y[lr[c * 32 + lane]] = lv[c * 32 + lane];
  } else {
    for (int c = 0; c < cnt; ++c) {
      const int r = lr[c * 32 + lane];
      y[r] = seg_out(lv[c * 32 + lane], add, r, sign);
    }
  }
}

// rows that cross chunks: the chunk that starts the row left its partial sum
// in y[r]; the first chunk continuing it adds the carries of every chunk that
// continues it, in chunk order
__global__ void k_seg_fix(int rows, const int *__restrict__ rp, const int *__restrict__ first, int nw,
                          const double *__restrict__ carry, double *__restrict__ y,
                          const double *__restrict__ add, double sign) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w <= 0 || w >= nw) return;
  const int ra = first[w];
  if (first[w - 1] == ra) return;  // no row starts in chunk w - 1: not the first continuation
  if (ra < rows && rp[ra] <= (long long)w * SEG_CH) return;  // a row starts at the chunk
  const int r = ra - 1;
  double v = y[r] + carry[w];
  for (int u = w + 1; u < nw && first[u] == ra && (ra >= rows || rp[ra] > (long long)u * SEG_CH); ++u) v += carry[u];
  y[r] = seg_out(v, add, r, sign);
}

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

void seg_spmv(lpk_ctx *ctx, int rows, long long nnz, const int *rp, const int *ci, const double *a,
              const int *first, double *carry, const double *x, double *y, const double *add, double sign) {
  cudaStream_t s = ctx->stream;
  const int nw = seg_chunks(nnz);
  if (nw == 0) {
    if (rows > 0) LPK_LAUNCH(ctx, k_seg_empty, tblk(rows), TPB, 0, s, rows, y, add, sign);
    return;
  }
  const int grid = (nw + SEG_WPB - 1) / SEG_WPB;
  if (aligned16(ci) && aligned16(a))
    LPK_LAUNCH(ctx, k_seg_spmv<true>, grid, TPB, 0, s, rows, nnz, rp, ci, a, first, nw, x, y, add, sign, carry);
  else
    LPK_LAUNCH(ctx, k_seg_spmv<false>, grid, TPB, 0, s, rows, nnz, rp, ci, a, first, nw, x, y, add, sign, carry);
  if (nw > 1) LPK_LAUNCH(ctx, k_seg_fix, tblk(nw), TPB, 0, s, rows, rp, first, nw, carry, y, add, sign);
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
namespace {
__global__ void k_start_bits(int rows, const int *__restrict__ rp, unsigned *__restrict__ bits) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int q = rp[r];
  if (rp[r + 1] > q) atomicOr(bits + (q >> 5), 1u << (q & 31));
}
}  // namespace

void start_bits(lpk_ctx *ctx, int rows, const int *rp, unsigned *bits) {
  if (rows > 0) LPK_LAUNCH(ctx, k_start_bits, tblk(rows), TPB, 0, ctx->stream, rows, rp, bits);
}

void seg_index(lpk_ctx *ctx, int rows, const int *rp, long long nnz, int *first) {
  const int nw = seg_chunks(nnz);
  LPK_LAUNCH(ctx, k_seg_first, tblk(nw + 1), TPB, 0, ctx->stream, rows, rp, nw, first);
}
void spmv_csr(lpk_ctx *ctx, const DevProblem &P, const double *x, double *y, const double *add, double sign) {
  if (P.m > 0) seg_spmv(ctx, P.m, P.nnz, P.rp, P.ci, P.a, P.seg_r, P.seg_carry, x, y, add, sign);
}
void spmv_csc(lpk_ctx *ctx, const DevProblem &P, const double *x, double *y) {
  if (P.n > 0) seg_spmv(ctx, P.n, P.nnz, P.cp, P.ri, P.at, P.seg_c, P.seg_carry, x, y, nullptr, 1.0);
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
