// noalloc.cu -- lpk_ne_solve_noalloc: the search-direction solve without any
// device allocation.
//
// Some callers cannot call cudaMalloc while they solve: applications whose
// device memory is owned by their own allocator (a caching allocator or a
// fixed arena that must not lose memory to the driver behind its back), and
// long-running services that must not fail with an out-of-memory error in the
// middle of a solve.  For them every temporary of this solve (the internal
// copies of d2, f, dy, dw, the Krylov workspace, the persistent kernel's
// control block and its reduction partials) lives in one file-scope device
// array of fixed size.  Its address is looked up when the first context on a
// device is created (lpk_create), which also loads this module on that device
// under lazy module loading, so the array is reserved then and held by that
// GPU until the process exits.
#include <cstdio>
#include <mutex>
#include <string>

#include "lpk_internal.cuh"

namespace {

constexpr size_t NOALLOC_BYTES = size_t(32) << 20;  // 32 MiB
constexpr size_t NOALLOC_DOUBLES = NOALLOC_BYTES / sizeof(double);
constexpr int MAX_DEVICES = 64;

}  // namespace

// The scratch.  In host code this name is only a host-side stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

namespace {

double *g_scratch_dev[MAX_DEVICES] = {nullptr};  // device address per device, set once
std::mutex g_scratch_mu;

}  // namespace

// Set-up, once per device, with that device current: lpk_create calls it
// right after cudaSetDevice(device).  cudaGetSymbolAddress gives the device
// address of the array (the name itself is only a host-side stand-in) and
// loads the module, reserving the array, if that has not happened yet.
lpk_status noalloc_setup(lpk_ctx *ctx) {
  const int dev = ctx->device;
  if (dev < 0 || dev >= MAX_DEVICES) return LPK_OK;  // no scratch on such a device: the entry point says so
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (g_scratch_dev[dev]) return LPK_OK;
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    ctx->err = std::string("cudaGetSymbolAddress of the no-allocation scratch failed: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LPK_OOM : LPK_CUDA_ERROR;
  }
  g_scratch_dev[dev] = (double *)p;
  return LPK_OK;
}

namespace {

lpk_status scratch_address(lpk_ctx *ctx, double **out) {
  const int dev = ctx->device;
  double *p = nullptr;
  if (dev >= 0 && dev < MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    p = g_scratch_dev[dev];
  }
  if (!p) {
    ctx->err = "lpk_ne_solve_noalloc: no scratch array on this device (device index beyond 63?)";
    return LPK_INVALID_ARG;
  }
  *out = p;
  return LPK_OK;
}

__global__ void k_div_na(int m, const double *f, const double *rho, double *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = rho[i] > 0.0 ? f[i] / rho[i] : 0.0;
}
__global__ void k_d2_flag(int n, const double *d2, double *flag) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && !(d2[j] > 0.0 && isfinite(d2[j]))) flag[0] = 1.0;
}

// device memory of the context's GPU, or managed memory
bool is_device_ptr(const void *p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

size_t round4(size_t x) { return (x + 3) & ~size_t(3); }  // keep 32-byte alignment of each block

}  // namespace

LPK_API lpk_status lpk_ne_solve_noalloc(lpk_ctx *ctx, lpk_problem *P, const double *d2, const double *f,
                                        int32_t inner_sweeps, double omega, int32_t solver, int32_t precision,
                                        double tol, int32_t max_iter, double *dy, double *dw,
                                        lpk_krylov_info *kinfo) {
  if (!ctx) return LPK_INVALID_ARG;
  cudaSetDevice(ctx->device);
  if (!P || !P->ctx || P->ctx != ctx) {
    ctx->err = "problem does not belong to this context";
    return LPK_INVALID_ARG;
  }
  DevProblem &d = P->d;
  if (!d2 || !f || !dy || inner_sweeps < 1 || !(omega > 0.0 && omega < 2.0) || !(tol >= 0.0) || max_iter < 0 ||
      (solver != LPK_MRNE && solver != LPK_CGNE) || (precision != LPK_FP64 && precision != LPK_MIXED)) {
    ctx->err = "lpk_ne_solve_noalloc: invalid arguments (solver must be MRNE or CGNE)";
    return LPK_INVALID_ARG;
  }
  const int dv = ctx->device;
  if (!is_device_ptr(d2, dv) || !is_device_ptr(f, dv) || !is_device_ptr(dy, dv) || (dw && !is_device_ptr(dw, dv))) {
    ctx->err = "lpk_ne_solve_noalloc: d2, f, dy and dw must be device (or managed) memory of the context's GPU";
    return LPK_INVALID_ARG;
  }
  const size_t m = d.m, n = d.n;
  const size_t need = round4(n + 1) + 3 * round4(m + 1) + round4(n + 1) + 4 + krylov_scratch_doubles(d);
  if (need > NOALLOC_DOUBLES) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "lpk_ne_solve_noalloc: this problem needs %.1f MiB of scratch, more than the %zu MiB the "
             "library reserves (use lpk_ne_solve)",
             need * 8.0 / (1 << 20), NOALLOC_BYTES >> 20);
    ctx->err = msg;
    return LPK_INVALID_ARG;
  }
  double *base = nullptr;
  lpk_status st = scratch_address(ctx, &base);
  if (st != LPK_OK) return st;
  double *td2 = base;
  double *tf = td2 + round4(n + 1);
  double *tfh = tf + round4(m + 1);
  double *tdy = tfh + round4(m + 1);
  double *tdw = tdy + round4(m + 1);
  double *flag = tdw + round4(n + 1);
  double *ws = flag + 4;  // 32-byte aligned: every block above is a multiple of 4 doubles
  cudaStream_t s = ctx->stream;
  // the flag must start at zero (the array keeps the previous call's contents)
  LPK_CUDA_TRY(ctx, cudaMemsetAsync(flag, 0, sizeof(double), s));
  gather_n(ctx, d, d2, td2);
  if (n > 0) LPK_LAUNCH(ctx, k_d2_flag, (int)((n + 255) / 256), 256, 0, s, (int)n, td2, flag);
  double hflag = 0.0;
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(&hflag, flag, sizeof(double), cudaMemcpyDeviceToHost, s));
  LPK_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (hflag != 0.0) {
    ctx->err = "d2 must be positive and finite";
    return LPK_INVALID_ARG;
  }
  gather_m(ctx, d, f, tf);
  scale_rows(ctx, d, td2);
  if (m > 0) LPK_LAUNCH(ctx, k_div_na, (int)((m + 255) / 256), 256, 0, s, (int)m, tf, d.rho, tfh);
  KrylovResult kr;
  const int maxit = max_iter > 0 ? max_iter : d.m;
  st = krylov_solve_scratch(ctx, d, solver, precision, inner_sweeps, omega, tfh, tol, maxit, tdw, tdy, &kr, ws);
  if (st != LPK_OK) return st;
  // A_hat^T dy_hat = A^T D D_cal^-1 dy_hat, so dy = D_cal^-1 dy_hat
  if (m > 0) LPK_LAUNCH(ctx, k_div_na, (int)((m + 255) / 256), 256, 0, s, (int)m, tdy, d.rho, tdy);
  scatter_m(ctx, d, tdy, dy);
  if (dw) scatter_n(ctx, d, tdw, dw, nullptr);
  LPK_CUDA_TRY(ctx, cudaGetLastError());
  LPK_CUDA_TRY(ctx, cudaStreamSynchronize(s));
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
