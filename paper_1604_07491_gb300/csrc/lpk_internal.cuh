// lpk_internal.cuh -- internal data structures and device helpers of the
// sm_103a library behind include/lpk.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lpk.h"

#define LPK_WARP 32

// ---------------------------------------------------------------------------
// Problem resident in HBM.  Rows are stored in sweep order: the multicolor
// permutation puts the rows of color c at positions [color_ptr[c],
// color_ptr[c+1]), so a color is one contiguous, coalesced CSR range and the
// m-space vectors of the Krylov solvers live in that order.
// ---------------------------------------------------------------------------
struct DevProblem {
  int m_in = 0, n_in = 0;     // input sizes
  int m = 0, n = 0;           // after removal of empty rows / columns
  long long nnz = 0;
  int n_colors = 0;
  bool has_empty_rows = false, has_empty_cols = false;

  // index maps (device)
  int *pos_of_in_row = nullptr;  // [m_in] input row -> sweep position (-1: removed)
  int *in_row_of_pos = nullptr;  // [m]    sweep position -> input row
  int *col_of_in = nullptr;      // [n_in] input column -> kept column (-1: removed)
  int *in_col_of = nullptr;      // [n]    kept column -> input column
  int *color_in = nullptr;       // [m_in] color of every input row (-1: removed)

  // permuted CSR (positions are sweep order), kept-column numbering
  int *rp = nullptr;             // [m+1]
  int *ci = nullptr;             // [nnz]
  double *a = nullptr;           // [nnz] A
  long long *src = nullptr;      // [nnz] input nonzero index of each entry
  double *ah64 = nullptr;        // [nnz] A_hat = D_cal^-1 A D, FP64
  float *ah32 = nullptr;         // [nnz] A_hat, FP32 copy for the mixed inner sweeps
  double *rho = nullptr;         // [m]   row norms of A D
  double *dcol = nullptr;        // [n]   d = sqrt(d2) of the last scaling

  // CSC of the permuted matrix (row indices are sweep positions, sorted)
  int *cp = nullptr;             // [n+1]
  int *ri = nullptr;             // [nnz]
  double *at = nullptr;          // [nnz]
  double *aht = nullptr;         // [nnz] A_hat in CSC order (bitwise equal to ah64)
  int *cpos = nullptr;           // [nnz] CSR position of each CSC entry

  // entry-balanced sparse products: chunks of SEG_CH entries; the first row
  // (column) starting at or after each chunk, and one partial sum per chunk
  int *seg_r = nullptr;          // [seg_chunks(nnz) + 1]
  int *seg_c = nullptr;          // [seg_chunks(nnz) + 1]
  double *seg_carry = nullptr;   // [seg_chunks(nnz)]
  // the persistent kernel's CSC product (same chunks): bit q of cbits is set
  // when a column starts at CSC entry q; per chunk, the partial sum of the
  // column that starts in it and goes on, and of the column it continues
  unsigned *cbits = nullptr;     // [nnz / 32 + 1]
  int ragged_cols = 0;           // longest column >= 32 entries and > 4 x the mean: entry-balanced CSC
  double *seg_cstart = nullptr, *seg_ccont = nullptr;  // [seg_chunks(nnz)]

  int *color_ptr = nullptr;      // [n_colors+1] device copy
  std::vector<int> color_ptr_h;  // host copy
  std::vector<int> rp_h;         // host copy of rp (sizes the shared-memory row cache)

  // execution path chosen by the autotuner (first solve on this problem)
  int tuned = 0, tuned_mode = 0, tuned_cs = 0, tuned_ug = 0;
  // time per Krylov iteration of the grid and of clusters of 16, 8, 4 CTAs
  // with u in shared / global memory (autotune)
  double tuned_us[7] = {0, 0, 0, 0, 0, 0, 0};

  cudaStream_t stream = nullptr;  // the owning context's stream (frees are ordered on it)

  // interior-point workspace (allocated on the first lp_solve)
  size_t ipm_bytes = 0;
  double *ipm_buf = nullptr;

  // Krylov workspace (allocated on first use)
  size_t ws_bytes = 0;
  void *ws = nullptr;
  // AB-GMRES storage (allocated on first use): one block for the basis, R,
  // rotations and partial dots, sized for gm_kmax basis vectors of gm_m rows
  size_t gm_bytes = 0, gm_kmax = 0, gm_m = 0;
  double *gm_V = nullptr;
};

struct lpk_problem {
  lpk_ctx *ctx = nullptr;
  DevProblem d;
};

struct lpk_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::string err;
  int verbose = 0;               // from lpk_options.verbose of the running solve
  lpk_stats stats{};             // see lpk_get_stats
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ev_block = nullptr;  // blocking-sync event of ctx_sync

  // reductions of the elementwise kernels: per-block partials + completion
  // counter, the last block reduces in fixed order (deterministic)
  double *red_part = nullptr;    // [RED_MAX_BLOCKS * RED_MAX_SLOTS]
  unsigned *red_count = nullptr;
  double *red_out = nullptr;     // [RED_MAX_SLOTS]
  double *h_red = nullptr;       // pinned host copy of red_out
  int red_blocks = 0;

  // execution path of the persistent Krylov kernel (lpk_set_exec)
  int cluster_mode = 0;          // 0 auto, 1 grid, 2 cluster, 3 batch
  int cluster_size_override = 0; // 0: chosen from nnz
  int last_cluster = 0;          // cluster size of the last launch (0: grid)
  int resident_mode = 0;         // 0: rows cached in shared memory when they fit, 1: never
  int last_resident = 0;         // the last launch cached the rows
  int u_place = 0;               // cluster path: 0 by the problem, 1 u in shared memory, 2 in global memory
  int last_u_global = 0;         // the last cluster launch kept u in global memory
  unsigned long long wait_limit_ns = 5000000000ull;  // bound of every grid-barrier wait
  long long stall_barrier = 0;   // testing: grid barrier CTA 0 does not arrive at (0: none)
  int phase_timing = 0;          // persistent kernel: time its barrier intervals by phase kind

  // problems prepared on this context (freed with it)
  std::vector<lpk_problem *> problems;

  // persistent Krylov kernel
  void *kctl = nullptr;          // KrylovCtl (device)
  void *h_kctl = nullptr;        // pinned host copy
  double *kpart = nullptr;       // per-CTA partials of the persistent kernels
  int kgrid_cache[8] = {0};      // cooperative grid sizes per kernel variant
};

// Device memory (devmem.cu): stream-ordered allocation on the context's
// stream from the library's pool; dev_free is ordered on the given stream.
cudaError_t dev_alloc_bytes(lpk_ctx *ctx, void **p, size_t bytes);
// Wait for the context's stream (blocking, not spinning, on the batch path).
cudaError_t ctx_sync(lpk_ctx *ctx);
void dev_free(cudaStream_t s, void *p);
template <typename T>
inline cudaError_t dev_alloc(lpk_ctx *ctx, T **p, size_t count) {
  return dev_alloc_bytes(ctx, (void **)p, sizeof(T) * (count > 0 ? count : 1));
}

constexpr int RED_MAX_SLOTS = 24;
constexpr int RED_THREADS = 256;

// every kernel launch site counts itself (lpk_get_stats)
#define LPK_COUNT(ctx) ((ctx)->stats.launches++)
#define LPK_LAUNCH(ctx, kernel, grid, block, smem, stream, ...) \
  do {                                                           \
    LPK_COUNT(ctx);                                              \
    kernel<<<grid, block, smem, stream>>>(__VA_ARGS__);          \
  } while (0)

// status helper for host code
#define LPK_CUDA_TRY(ctx, expr)                                                     \
  do {                                                                             \
    cudaError_t e__ = (expr);                                                      \
    if (e__ != cudaSuccess) {                                                      \
      (ctx)->err = std::string(#expr) + ": " + cudaGetErrorString(e__);            \
      return e__ == cudaErrorMemoryAllocation ? LPK_OOM : LPK_CUDA_ERROR;          \
    }                                                                              \
  } while (0)

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// L2-coherent loads/stores for data that other CTAs write during a launch
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }

// Block-wide sums of K values in a fixed order; result valid in every thread.
// sbuf must hold K * (blockDim.x / 32) doubles.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *sbuf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sbuf[k * nw + wid] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sbuf[k * nw + w];
    v[k] = s;
  }
  __syncthreads();
}

// host-side helpers implemented in the .cu files
lpk_status prep_problem(lpk_ctx *ctx, const lpk_matrix *A, uint64_t seed, DevProblem &P);
void free_problem(DevProblem &P);
lpk_status ensure_reduce(lpk_ctx *ctx);

// elementwise / sparse kernels (ipm_kernels.cu)
constexpr int SEG_K = 8;              // entries per lane of the sparse products
constexpr int SEG_CH = 32 * SEG_K;    // entries per warp (chunk)
inline int seg_chunks(long long nnz) { return (int)((nnz + SEG_CH - 1) / SEG_CH); }
// first[w] = first of the `rows` compressed rows starting at or after entry
// w SEG_CH (w < seg_chunks(nnz)), first[seg_chunks(nnz)] = rows
void seg_index(lpk_ctx *ctx, int rows, const int *rp, long long nnz, int *first);
// bits[q / 32] bit q % 32 set when one of the `rows` compressed rows starts at
// entry q (bits zeroed by the caller)
void start_bits(lpk_ctx *ctx, int rows, const int *rp, unsigned *bits);
void scale_rows(lpk_ctx *ctx, DevProblem &P, const double *d2);
void spmv_csr(lpk_ctx *ctx, const DevProblem &P, const double *x, double *y, const double *add,
              double sign);
void spmv_csc(lpk_ctx *ctx, const DevProblem &P, const double *x, double *y);
void gather_m(lpk_ctx *ctx, const DevProblem &P, const double *in, double *out);   // input -> sweep
void scatter_m(lpk_ctx *ctx, const DevProblem &P, const double *in, double *out);  // sweep -> input
void gather_n(lpk_ctx *ctx, const DevProblem &P, const double *in, double *out);
void scatter_n(lpk_ctx *ctx, const DevProblem &P, const double *in, double *out, const double *fill);

// persistent Krylov (krylov.cu).  f_hat in sweep order; dw[n], dy_hat[m] (sweep order)
struct KrylovResult {
  int iters = 0, converged = 0, restarts = 0, breakdown = 0, timeout = 0;
  int iters32 = 0, escalations = 0;  // mixed precision: FP32-sweep iterations, FP64 escalations
  double res0 = 0, res = 0;
};
lpk_status krylov_solve(lpk_ctx *ctx, DevProblem &P, int method, int precision, int ell, double omega,
                        const double *f_hat, double tol, int maxit, double *dw, double *dy_hat,
                        KrylovResult *out, double *hist);
lpk_status sweep_only(lpk_ctx *ctx, DevProblem &P, int kind, int precision, int ell, double omega,
                      const double *g_hat, double *z, double *u);
// address of the no-allocation scratch on ctx->device (lpk_create, once per device)
lpk_status noalloc_setup(lpk_ctx *ctx);
// persistent Krylov solve on caller-supplied device memory (no allocation)
size_t krylov_scratch_doubles(const DevProblem &P);
// BA-GMRES with NR-SOR on min ||A_hat^T dy_hat - r|| (r_n: n-space, kept
// columns; f_hat = A_hat r: m-space, for the explicit residual); dw = A_hat^T dy_hat
lpk_status krylov_solve_ls(lpk_ctx *ctx, DevProblem &P, int precision, int ell, double omega, const double *r_n,
                           const double *f_hat, double tol, int maxit, double *dw, double *dy_hat,
                           KrylovResult *out);
lpk_status krylov_solve_scratch(lpk_ctx *ctx, DevProblem &P, int method, int precision, int ell, double omega,
                                const double *f_hat, double tol, int maxit, double *dw, double *dy_hat,
                                KrylovResult *out, double *ws);
