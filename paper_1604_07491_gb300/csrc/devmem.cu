// devmem.cu -- device memory of the library: stream-ordered allocations from
// one memory pool per device that keeps freed memory for reuse.
//
// Several contexts (one per host thread, each with its own stream) solve LPs
// side by side on one GPU in the batched and serving modes.  A plain
// cudaFree waits for the whole device, so one context finishing a solve would
// stall behind the others' persistent kernels; cudaFreeAsync on the owning
// stream does not.  The pool's release threshold is set to the maximum so
// memory freed by one solve is reused by the next without returning it to
// the driver at every synchronisation.
#include <cstdint>
#include <mutex>

#include "lpk_internal.cuh"

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[MAX_DEVICES] = {};

cudaError_t pool_for(int dev, cudaMemPool_t *out) {
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    cudaError_t e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    g_pool[dev] = p;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

}  // namespace

cudaError_t dev_alloc_bytes(lpk_ctx *ctx, void **p, size_t bytes) {
  cudaMemPool_t pool;
  cudaError_t e = pool_for(ctx->device, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 16, pool, ctx->stream);
}

void dev_free(cudaStream_t s, void *p) {
  if (p) cudaFreeAsync(p, s);
}

// Host waits on the context's stream.  Alone, a context spins in the driver
// (lowest wake-up latency).  On the batch path many contexts wait at once,
// one host thread each; spinning threads would then take every host core and
// delay each other's next launch by whole scheduler periods, so those waits
// block on an event created for blocking synchronisation instead.
cudaError_t ctx_sync(lpk_ctx *ctx) {
  if (ctx->cluster_mode != 3) return cudaStreamSynchronize(ctx->stream);
  if (!ctx->ev_block) {
    cudaError_t e = cudaEventCreateWithFlags(&ctx->ev_block, cudaEventBlockingSync | cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaEventRecord(ctx->ev_block, ctx->stream);
  if (e != cudaSuccess) return e;
  return cudaEventSynchronize(ctx->ev_block);
}
