// prep.cu -- lpk_prepare on the device: validation, removal of empty rows and
// columns (Sec. 4.2), multicolor row ordering, permuted CSR and CSC.
//
// Coloring.  The paper sweeps rows in natural order (Algorithms 5-6).  To make
// a sweep data-parallel the rows are partitioned into colors whose rows share
// no column: within a color the updates u += d_i alpha_i touch disjoint
// entries of u, so the rows of a color can run concurrently and the sweep is
// exactly the sequential sweep over the permuted row order.  The coloring is
// greedy first fit over rows in decreasing priority pi(i) = splitmix64(seed ^
// i) (ties by lower i), computed Jones-Plassmann style: in each round every
// uncolored row whose higher-priority neighbours are all colored takes the
// smallest color none of them uses.  Rows colored in one round are never
// neighbours, so the result equals the sequential greedy order exactly.
#include <algorithm>
#include <cstdio>

#include "lpk_internal.cuh"

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  // SplitMix64 finaliser (published constants of Steele, Lea and Flood's generator)
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// ---- validation -----------------------------------------------------------
// err codes: 1 row_ptr decreasing, 2 column out of range, 3 non-finite value,
// 4 columns not strictly increasing within a row
__global__ void k_validate(int m, int n, const long long *rp, const int *ci, const double *v,
                           int *err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  long long k0 = rp[i], k1 = rp[i + 1];
  if (k1 < k0) { atomicMax(err, 1); return; }
  int prev = -1;
  for (long long k = k0; k < k1; ++k) {
    int c = ci[k];
    if (c < 0 || c >= n) { atomicMax(err, 2); return; }
    if (!isfinite(v[k])) { atomicMax(err, 3); return; }
    if (c <= prev) { atomicMax(err, 4); return; }
    prev = c;
  }
}

__global__ void k_counts(int m, const long long *rp, const int *ci, int *rowcnt, int *colcnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  rowcnt[i] = (int)(rp[i + 1] - rp[i]);
  for (long long k = rp[i]; k < rp[i + 1]; ++k) atomicAdd(&colcnt[ci[k]], 1);
}

__global__ void k_flags(int len, const int *cnt, int *flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) flag[i] = cnt[i] > 0 ? 1 : 0;
}

// exclusive scan in one block (chunked); out has len+1 entries
template <typename T>
__global__ void k_scan(int len, const int *in, T *out) {
  __shared__ T s[1024];
  __shared__ T carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < len; base += 1024) {
    int i = base + threadIdx.x;
    T v = i < len ? (T)in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      T t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < len) out[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[len] = carry;
}

// kept index maps: map_in[i] = new index or -1; inv[new] = i
__global__ void k_keepmap(int len, const int *cnt, const int *scan, int *map_in, int *inv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  if (cnt[i] > 0) {
    map_in[i] = scan[i];
    inv[scan[i]] = i;
  } else {
    map_in[i] = -1;
  }
}

// reduced (natural-order) CSR pattern: row lengths of kept rows
__global__ void k_red_rowlen(int mr, const int *in_row_of_red, const int *rowcnt, int *len) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < mr) len[r] = rowcnt[in_row_of_red[r]];
}
__global__ void k_red_fill(int mr, const int *in_row_of_red, const long long *rp_in, const int *ci_in,
                           const int *col_map, const long long *rp_red, int *ci_red) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mr) return;
  long long k0 = rp_in[in_row_of_red[r]], k1 = rp_in[in_row_of_red[r] + 1], o = rp_red[r];
  for (long long k = k0; k < k1; ++k) ci_red[o + (k - k0)] = col_map[ci_in[k]];
}

// CSC pattern by atomic fill (order within a column is irrelevant to coloring)
__global__ void k_csc_fill_pattern(int mr, const long long *rp, const int *ci, int *cursor, int *ri) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mr) return;
  for (long long k = rp[r]; k < rp[r + 1]; ++k) ri[atomicAdd(&cursor[ci[k]], 1)] = r;
}

__global__ void k_prio(int mr, uint64_t seed, unsigned long long *prio, int *round_of) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mr) return;
  prio[r] = splitmix64(seed ^ (uint64_t)(uint32_t)r);
  round_of[r] = -1;
}

__device__ __forceinline__ bool precedes(unsigned long long pk, int k, unsigned long long pi, int i) {
  return pk > pi || (pk == pi && k < i);
}

// one Jones-Plassmann first-fit round, one warp per row
__global__ void k_color_round(int mr, const long long *rp, const int *ci, const int *cp, const int *ri,
                              const unsigned long long *prio, int *color, int *round_of, int round,
                              int *remaining) {
  __shared__ unsigned mask[TPB / 32][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= mr) return;
  if (round_of[i] >= 0) return;  // warp-uniform
  const unsigned long long pi = prio[i];
  const long long k0 = rp[i], k1 = rp[i + 1];
  bool ready = true;
  for (long long k = k0 + lane; k < k1 && ready; k += 32) {
    int j = ci[k];
    for (int q = cp[j]; q < cp[j + 1]; ++q) {
      int nb = ri[q];
      if (nb == i) continue;
      if (precedes(prio[nb], nb, pi, i)) {
        int ro = round_of[nb];
        if (ro < 0 || ro >= round) { ready = false; break; }
      }
    }
  }
  ready = __all_sync(0xffffffffu, ready);
  if (!ready) {
    if (lane == 0) atomicAdd(remaining, 1);
    return;
  }
  // first fit: smallest color absent among higher-priority neighbours
  for (int base = 0;; base += 1024) {
    mask[w][lane] = 0u;
    __syncwarp();
    for (long long k = k0 + lane; k < k1; k += 32) {
      int j = ci[k];
      for (int q = cp[j]; q < cp[j + 1]; ++q) {
        int nb = ri[q];
        if (nb == i || !precedes(prio[nb], nb, pi, i)) continue;
        int c = color[nb] - base;
        if (c >= 0 && c < 1024) atomicOr(&mask[w][c >> 5], 1u << (c & 31));
      }
    }
    __syncwarp();
    unsigned freebits = ~mask[w][lane];
    unsigned any = __ballot_sync(0xffffffffu, freebits != 0u);
    if (any) {
      int l = __ffs(any) - 1;
      unsigned fb = __shfl_sync(0xffffffffu, freebits, l);
      if (lane == 0) {
        color[i] = base + l * 32 + (__ffs(fb) - 1);
        round_of[i] = round;
      }
      return;
    }
    __syncwarp();
  }
}

__global__ void k_max(int len, const int *v, int *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) atomicMax(out, v[i]);
}

// stable counting sort of rows by color: per block of 1024 rows a histogram,
// a global scan over (color, block), then an in-block serial placement
constexpr int SORT_CHUNK = 1024;
__global__ void k_color_hist(int mr, int nc, int nb, const int *color, int *cnt /*[nc*nb]*/) {
  int b = blockIdx.x;
  for (int t = threadIdx.x; t < SORT_CHUNK; t += blockDim.x) {
    int r = b * SORT_CHUNK + t;
    if (r < mr) atomicAdd(&cnt[color[r] * nb + b], 1);
  }
}
__global__ void k_color_place(int mr, int nb, const int *color, int *cur /*[nc*nb], scan copy*/,
                              int *perm, int *pos_of_red) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  // serial walk over the rows of chunk b in ascending order; the (color, chunk)
  // cursor is touched by this thread only, so the placement is stable
  for (int t = 0; t < SORT_CHUNK; ++t) {
    int r = b * SORT_CHUNK + t;
    if (r >= mr) break;
    int p = cur[color[r] * nb + b]++;
    perm[p] = r;
    pos_of_red[r] = p;
  }
}

// permuted CSR: row lengths in sweep order, then fill
__global__ void k_perm_rowlen(int mr, const int *perm, const long long *rp_red, int *len) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < mr) len[p] = (int)(rp_red[perm[p] + 1] - rp_red[perm[p]]);
}
__global__ void k_perm_fill(int mr, const int *perm, const int *in_row_of_red, const long long *rp_in,
                            const double *val_in, const int *ci_red, const long long *rp_red,
                            const int *rp_p, int *ci_p, double *a_p, long long *src) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= mr) return;
  int r = perm[p];
  long long kin = rp_in[in_row_of_red[r]], kred = rp_red[r];
  int o = rp_p[p], len = rp_p[p + 1] - o;
  for (int t = 0; t < len; ++t) {
    ci_p[o + t] = ci_red[kred + t];
    a_p[o + t] = val_in[kin + t];
    src[o + t] = kin + t;
  }
}

// CSC of the permuted matrix: atomic fill, then sort every column by row
// CSC entry q of the permuted matrix: row ri[q], value at[q], and cpos[q] the
// position of the same entry in the CSR arrays
__global__ void k_csc_fill(int mr, const int *rp, const int *ci, const double *a, int *cursor, int *ri,
                           double *at, int *cpos) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= mr) return;
  for (int k = rp[p]; k < rp[p + 1]; ++k) {
    int q = atomicAdd(&cursor[ci[k]], 1);
    ri[q] = p;
    at[q] = a[k];
    cpos[q] = k;
  }
}
__global__ void k_csc_sort(int nr, const int *cp, int *ri, double *at, int *cpos) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nr) return;
  for (int q = cp[j] + 1; q < cp[j + 1]; ++q) {  // insertion sort (columns are short)
    int r = ri[q];
    double v = at[q];
    int k = cpos[q];
    int t = q - 1;
    while (t >= cp[j] && ri[t] > r) {
      ri[t + 1] = ri[t];
      at[t + 1] = at[t];
      cpos[t + 1] = cpos[t];
      --t;
    }
    ri[t + 1] = r;
    at[t + 1] = v;
    cpos[t + 1] = k;
  }
}

__global__ void k_compose(int m_in, const int *row_map, const int *pos_of_red, const int *color_red,
                          int *pos_of_in_row, int *color_in) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m_in) return;
  int r = row_map[i];
  pos_of_in_row[i] = r >= 0 ? pos_of_red[r] : -1;
  color_in[i] = r >= 0 ? color_red[r] : -1;
}
__global__ void k_inrow_of_pos(int mr, const int *perm, const int *in_row_of_red, int *in_row_of_pos) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < mr) in_row_of_pos[p] = in_row_of_red[perm[p]];
}

inline int nblk(long long n, int t = TPB) { return (int)((n + t - 1) / t); }

struct Scratch {  // device temporaries of prepare, freed (stream-ordered) at its end
  lpk_ctx *ctx;
  std::vector<void *> ptrs;
  explicit Scratch(lpk_ctx *c) : ctx(c) {}
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    cudaError_t e = dev_alloc(ctx, p, count);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~Scratch() {
    for (void *p : ptrs) dev_free(ctx->stream, p);
  }
};

}  // namespace

void free_problem(DevProblem &P) {
  void *ptrs[] = {P.pos_of_in_row, P.in_row_of_pos, P.col_of_in, P.in_col_of, P.color_in, P.rp,
                  P.ci,            P.a,             P.src,       P.ah64,      P.ah32,     P.rho,
                  P.cp,            P.ri,            P.at,        P.aht,       P.color_ptr, P.ws,
                  P.gm_V,          P.ipm_buf,       P.dcol,      P.cpos,      P.seg_r,     P.seg_c,
                  P.seg_carry,     P.cbits,         P.seg_cstart, P.seg_ccont};
  for (void *p : ptrs) dev_free(P.stream, p);
  P = DevProblem();
}

lpk_status prep_problem(lpk_ctx *ctx, const lpk_matrix *A, uint64_t seed, DevProblem &P) {
  cudaStream_t st = ctx->stream;
  const int m = A->m, n = A->n;
  const long long nnz = A->nnz;
  P.stream = st;
  P.m_in = m;
  P.n_in = n;
  Scratch S(ctx);
  long long *rp_in;
  int *ci_in;
  double *val_in;
  // ---- input on the device ------------------------------------------------
  if (A->on_device) {
    rp_in = (long long *)A->row_ptr;
    ci_in = (int *)A->col_idx;
    val_in = (double *)A->val;
    long long ends[2];
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(&ends[0], rp_in, sizeof(long long), cudaMemcpyDeviceToHost, st));
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(&ends[1], rp_in + m, sizeof(long long), cudaMemcpyDeviceToHost, st));
    LPK_CUDA_TRY(ctx, ctx_sync(ctx));
    if (ends[0] != 0 || ends[1] != nnz) {
      ctx->err = "row_ptr[0] must be 0 and row_ptr[m] must equal nnz";
      return LPK_INVALID_ARG;
    }
  } else {
    if (A->row_ptr[0] != 0 || A->row_ptr[m] != nnz) {
      ctx->err = "row_ptr[0] must be 0 and row_ptr[m] must equal nnz";
      return LPK_INVALID_ARG;
    }
    LPK_CUDA_TRY(ctx, S.get(&rp_in, m + 1));
    LPK_CUDA_TRY(ctx, S.get(&ci_in, nnz));
    LPK_CUDA_TRY(ctx, S.get(&val_in, nnz));
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(rp_in, A->row_ptr, sizeof(long long) * (m + 1), cudaMemcpyHostToDevice, st));
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(ci_in, A->col_idx, sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(val_in, A->val, sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
  }
  int *err, *rowcnt, *colcnt, *rflag, *cflag, *rscan, *cscan, *row_map, *red_row, *col_map_tmp;
  LPK_CUDA_TRY(ctx, S.get(&err, 4));
  LPK_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 4 * sizeof(int), st));
  if (m > 0) LPK_LAUNCH(ctx, k_validate, nblk(m), TPB, 0, st, m, n, rp_in, ci_in, val_in, err);
  int herr = 0;
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  if (herr) {
    const char *msg[] = {"", "row_ptr decreases", "column index out of range", "non-finite value",
                         "column indices not strictly increasing within a row"};
    ctx->err = std::string("invalid matrix: ") + msg[herr];
    return LPK_INVALID_ARG;
  }
  // ---- empty rows / columns -----------------------------------------------
  LPK_CUDA_TRY(ctx, S.get(&rowcnt, m));
  LPK_CUDA_TRY(ctx, S.get(&colcnt, n));
  LPK_CUDA_TRY(ctx, S.get(&rflag, m));
  LPK_CUDA_TRY(ctx, S.get(&cflag, n));
  LPK_CUDA_TRY(ctx, S.get(&rscan, m + 1));
  LPK_CUDA_TRY(ctx, S.get(&cscan, n + 1));
  LPK_CUDA_TRY(ctx, S.get(&row_map, m));
  LPK_CUDA_TRY(ctx, S.get(&red_row, m));
  LPK_CUDA_TRY(ctx, cudaMemsetAsync(colcnt, 0, sizeof(int) * (n > 0 ? n : 1), st));
  if (m > 0) LPK_LAUNCH(ctx, k_counts, nblk(m), TPB, 0, st, m, rp_in, ci_in, rowcnt, colcnt);
  if (m > 0) LPK_LAUNCH(ctx, k_flags, nblk(m), TPB, 0, st, m, rowcnt, rflag);
  if (n > 0) LPK_LAUNCH(ctx, k_flags, nblk(n), TPB, 0, st, n, colcnt, cflag);
  LPK_LAUNCH(ctx, k_scan<int>, 1, 1024, 0, st, m, rflag, rscan);
  LPK_LAUNCH(ctx, k_scan<int>, 1, 1024, 0, st, n, cflag, cscan);
  int mr = 0, nr = 0;
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(&mr, rscan + m, sizeof(int), cudaMemcpyDeviceToHost, st));
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(&nr, cscan + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  P.m = mr;
  P.n = nr;
  P.nnz = nnz;
  P.has_empty_rows = mr < m;
  P.has_empty_cols = nr < n;
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.col_of_in, n));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.in_col_of, nr));
  if (m > 0) LPK_LAUNCH(ctx, k_keepmap, nblk(m), TPB, 0, st, m, rowcnt, rscan, row_map, red_row);
  if (n > 0) LPK_LAUNCH(ctx, k_keepmap, nblk(n), TPB, 0, st, n, colcnt, cscan, P.col_of_in, P.in_col_of);
  (void)col_map_tmp;
  // reduced natural-order CSR pattern
  int *rlen, *ci_red;
  long long *rp_red;
  LPK_CUDA_TRY(ctx, S.get(&rlen, mr));
  LPK_CUDA_TRY(ctx, S.get(&rp_red, mr + 1));
  LPK_CUDA_TRY(ctx, S.get(&ci_red, nnz));
  if (mr > 0) LPK_LAUNCH(ctx, k_red_rowlen, nblk(mr), TPB, 0, st, mr, red_row, rowcnt, rlen);
  LPK_LAUNCH(ctx, k_scan<long long>, 1, 1024, 0, st, mr, rlen, rp_red);
  if (mr > 0) LPK_LAUNCH(ctx, k_red_fill, nblk(mr), TPB, 0, st, mr, red_row, rp_in, ci_in, P.col_of_in, rp_red, ci_red);
  // column pattern (reduced numbering)
  int *ccnt_red, *cp_red, *cursor, *ri_red;
  LPK_CUDA_TRY(ctx, S.get(&ccnt_red, nr));
  LPK_CUDA_TRY(ctx, S.get(&cp_red, nr + 1));
  LPK_CUDA_TRY(ctx, S.get(&cursor, nr));
  LPK_CUDA_TRY(ctx, S.get(&ri_red, nnz));
  {
    // column counts of kept columns are the input counts
    LPK_CUDA_TRY(ctx, cudaMemsetAsync(ccnt_red, 0, sizeof(int) * (nr > 0 ? nr : 1), st));
  }
  // recount in reduced numbering (cheap and avoids another gather kernel)
  if (mr > 0) {
    LPK_LAUNCH(ctx, k_counts, nblk(mr), TPB, 0, st, mr, rp_red, ci_red, rlen, ccnt_red);
  }
  LPK_LAUNCH(ctx, k_scan<int>, 1, 1024, 0, st, nr, ccnt_red, cp_red);
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(cursor, cp_red, sizeof(int) * (nr > 0 ? nr : 1), cudaMemcpyDeviceToDevice, st));
  if (mr > 0) LPK_LAUNCH(ctx, k_csc_fill_pattern, nblk(mr), TPB, 0, st, mr, rp_red, ci_red, cursor, ri_red);
  // ---- coloring rounds ------------------------------------------------------
  unsigned long long *prio;
  int *color, *round_of, *remaining;
  LPK_CUDA_TRY(ctx, S.get(&prio, mr));
  LPK_CUDA_TRY(ctx, S.get(&color, mr));
  LPK_CUDA_TRY(ctx, S.get(&round_of, mr));
  LPK_CUDA_TRY(ctx, S.get(&remaining, 8));
  if (mr > 0) LPK_LAUNCH(ctx, k_prio, nblk(mr), TPB, 0, st, mr, seed, prio, round_of);
  int round = 0;
  const int wblocks = nblk((long long)mr * 32);
  while (mr > 0) {
    const int burst = 4;  // rounds between host checks
    LPK_CUDA_TRY(ctx, cudaMemsetAsync(remaining, 0, sizeof(int) * burst, st));
    for (int b = 0; b < burst; ++b)
      LPK_LAUNCH(ctx, k_color_round, wblocks, TPB, 0, st, mr, rp_red, ci_red, cp_red, ri_red, prio, color, round_of,
                                              round + b, remaining + b);
    int rem[burst];
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(rem, remaining, sizeof(int) * burst, cudaMemcpyDeviceToHost, st));
    LPK_CUDA_TRY(ctx, ctx_sync(ctx));
    round += burst;
    if (rem[burst - 1] == 0) break;
    if (round > mr + 8) {
      ctx->err = "coloring did not terminate";
      return LPK_CUDA_ERROR;
    }
  }
  int *cmax;
  LPK_CUDA_TRY(ctx, S.get(&cmax, 1));
  LPK_CUDA_TRY(ctx, cudaMemsetAsync(cmax, 0xff, sizeof(int), st));  // -1
  if (mr > 0) LPK_LAUNCH(ctx, k_max, nblk(mr), TPB, 0, st, mr, color, cmax);
  int hmax = -1;
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(&hmax, cmax, sizeof(int), cudaMemcpyDeviceToHost, st));
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  const int nc = hmax + 1;
  P.n_colors = nc;
  // ---- rows sorted by (color, row) ------------------------------------------
  const int nb = (mr + SORT_CHUNK - 1) / SORT_CHUNK;
  int *hist, *hscan, *perm, *pos_of_red;
  LPK_CUDA_TRY(ctx, S.get(&hist, (size_t)nc * nb));
  LPK_CUDA_TRY(ctx, S.get(&hscan, (size_t)nc * nb + 1));
  LPK_CUDA_TRY(ctx, S.get(&perm, mr));
  LPK_CUDA_TRY(ctx, S.get(&pos_of_red, mr));
  if (mr > 0) {
    LPK_CUDA_TRY(ctx, cudaMemsetAsync(hist, 0, sizeof(int) * (size_t)nc * nb, st));
    LPK_LAUNCH(ctx, k_color_hist, nb, TPB, 0, st, mr, nc, nb, color, hist);
    LPK_LAUNCH(ctx, k_scan<int>, 1, 1024, 0, st, nc * nb, hist, hscan);
    LPK_CUDA_TRY(ctx, cudaMemcpyAsync(hist, hscan, sizeof(int) * (size_t)nc * nb, cudaMemcpyDeviceToDevice, st));
    LPK_LAUNCH(ctx, k_color_place, nblk(nb, 64), 64, 0, st, mr, nb, color, hist, perm, pos_of_red);
  }
  P.color_ptr_h.assign(nc + 1, 0);
  {
    std::vector<int> hs((size_t)nc * nb + 1);
    if (mr > 0)
      LPK_CUDA_TRY(ctx, cudaMemcpyAsync(hs.data(), hscan, sizeof(int) * hs.size(), cudaMemcpyDeviceToHost, st));
    LPK_CUDA_TRY(ctx, ctx_sync(ctx));
    for (int c = 0; c < nc; ++c) P.color_ptr_h[c] = hs[(size_t)c * nb];
    P.color_ptr_h[nc] = mr;
  }
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.color_ptr, nc + 1));
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(P.color_ptr, P.color_ptr_h.data(), sizeof(int) * (nc + 1), cudaMemcpyHostToDevice, st));
  // ---- permuted CSR ---------------------------------------------------------
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.rp, mr + 1));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.ci, nnz));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.a, nnz));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.src, nnz));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.ah64, nnz));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.ah32, nnz));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.rho, mr));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.dcol, nr));
  if (mr > 0) LPK_LAUNCH(ctx, k_perm_rowlen, nblk(mr), TPB, 0, st, mr, perm, rp_red, rlen);
  LPK_LAUNCH(ctx, k_scan<int>, 1, 1024, 0, st, mr, rlen, P.rp);
  if (mr > 0)
    LPK_LAUNCH(ctx, k_perm_fill, nblk(mr), TPB, 0, st, mr, perm, red_row, rp_in, val_in, ci_red, rp_red, P.rp, P.ci, P.a,
                                           P.src);
  // ---- CSC of the permuted matrix -------------------------------------------
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.cp, nr + 1));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.ri, nnz));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.at, nnz));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.aht, nnz));
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(P.cp, cp_red, sizeof(int) * (nr + 1), cudaMemcpyDeviceToDevice, st));
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(cursor, cp_red, sizeof(int) * (nr > 0 ? nr : 1), cudaMemcpyDeviceToDevice, st));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.cpos, nnz));
  if (mr > 0) LPK_LAUNCH(ctx, k_csc_fill, nblk(mr), TPB, 0, st, mr, P.rp, P.ci, P.a, cursor, P.ri, P.at, P.cpos);
  if (nr > 0) LPK_LAUNCH(ctx, k_csc_sort, nblk(nr), TPB, 0, st, nr, P.cp, P.ri, P.at, P.cpos);
  // ---- chunk index of the entry-balanced products ----------------------------
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.seg_r, seg_chunks(nnz) + 1));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.seg_c, seg_chunks(nnz) + 1));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.seg_carry, seg_chunks(nnz)));
  seg_index(ctx, mr, P.rp, nnz, P.seg_r);
  seg_index(ctx, nr, P.cp, nnz, P.seg_c);
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.cbits, nnz / 32 + 1));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.seg_cstart, seg_chunks(nnz)));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.seg_ccont, seg_chunks(nnz)));
  LPK_CUDA_TRY(ctx, cudaMemsetAsync(P.cbits, 0, sizeof(unsigned) * (nnz / 32 + 1), st));
  start_bits(ctx, nr, P.cp, P.cbits);
  // ---- maps to the input numbering ------------------------------------------
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.pos_of_in_row, m));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.color_in, m));
  LPK_CUDA_TRY(ctx, dev_alloc(ctx, &P.in_row_of_pos, mr));
  if (m > 0) LPK_LAUNCH(ctx, k_compose, nblk(m), TPB, 0, st, m, row_map, pos_of_red, color, P.pos_of_in_row, P.color_in);
  if (mr > 0) LPK_LAUNCH(ctx, k_inrow_of_pos, nblk(mr), TPB, 0, st, mr, perm, red_row, P.in_row_of_pos);
  P.rp_h.assign(mr + 1, 0);
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(P.rp_h.data(), P.rp, sizeof(int) * (mr + 1), cudaMemcpyDeviceToHost, st));
  std::vector<int> cp_h(nr + 1, 0);
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(cp_h.data(), P.cp, sizeof(int) * (nr + 1), cudaMemcpyDeviceToHost, st));
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  LPK_CUDA_TRY(ctx, ctx_sync(ctx));
  int max_col = 0;
  for (int j = 0; j < nr; ++j) max_col = std::max(max_col, cp_h[j + 1] - cp_h[j]);
  P.ragged_cols = nr > 0 && max_col >= 32 && (double)max_col > 4.0 * (double)nnz / nr;
  return LPK_OK;
}
