// ipm_kernels.cuh -- deterministic grid reductions for the elementwise kernels.
#pragma once
#include <math.h>

#include "lpk_internal.cuh"

struct RedArgs {
  double *part;      // [gridDim.x * RED_MAX_SLOTS]
  unsigned *count;   // completion counter (returns to 0 after each use)
  double *out;       // [RED_MAX_SLOTS]
};

lpk_status red_fetch(lpk_ctx *ctx, int nslots);
RedArgs red_args(lpk_ctx *ctx);
int red_grid(lpk_ctx *ctx);

// Sums in slots [0, NS), minima in slots [NS, NS+NM).  Every block writes its
// partials; the last block to finish reduces all partials in block order, so
// the result does not depend on scheduling.  Call from every thread.
template <int NS, int NM>
__device__ __forceinline__ void grid_reduce(double (&s)[NS], double (&mn)[NM], const RedArgs &R) {
  constexpr int K = NS + NM;
  __shared__ double sb[K > 0 ? K * (RED_THREADS / 32) : 1];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k) s[k] = warp_sum(s[k]);
#pragma unroll
  for (int k = 0; k < NM; ++k) mn[k] = warp_min(mn[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) sb[k * nw + wid] = s[k];
#pragma unroll
    for (int k = 0; k < NM; ++k) sb[(NS + k) * nw + wid] = mn[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < K; ++k) {
      double v = k < NS ? 0.0 : INFINITY;
      for (int w = 0; w < nw; ++w) v = k < NS ? v + sb[k * nw + w] : fmin(v, sb[k * nw + w]);
      R.part[(size_t)blockIdx.x * RED_MAX_SLOTS + k] = v;
    }
    __threadfence();
    unsigned t = atomicAdd(R.count, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // last block: thread k reduces slot k over blocks 0..gridDim.x-1 in order
  if (threadIdx.x < K) {
    const int k = threadIdx.x;
    double v = k < NS ? 0.0 : INFINITY;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      double p = __ldcg(&R.part[(size_t)b * RED_MAX_SLOTS + k]);
      v = k < NS ? v + p : fmin(v, p);
    }
    R.out[k] = v;
  }
  if (threadIdx.x == 0) *R.count = 0u;
}
