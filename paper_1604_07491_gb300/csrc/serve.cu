// serve.cu -- many LPs on one GPU at once: the batched solve and the
// continuous-batching server.  The paper solves one LP at a time on a CPU; it
// has no counterpart for either.
//
// A solve of a small or medium LP keeps only one thread-block cluster busy
// (its persistent Krylov kernel) and a few elementwise kernels between the
// Krylov solves, so one LP leaves most of the GPU idle.  Here independent LPs
// run side by side, one per "lane": a host thread with its own context and
// CUDA stream.  The lanes' persistent kernels run as separate clusters, each
// with its own hardware cluster barrier, so no lane ever waits on another
// (the grid path, whose barrier spans every SM, is excluded).  Device memory
// comes from the library's stream-ordered pool, so a lane that allocates or
// frees never waits for the others' kernels.
//
// Lanes run the LPK_EXEC_BATCH path: the cluster size depends on the problem
// alone, and all reductions are in a fixed order, so an LP gives bitwise the
// same result alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "lpk_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// batched solve
// ---------------------------------------------------------------------------
struct ModeGuard {  // the batch path for the duration of one solve
  lpk_ctx *ctx;
  int saved;
  explicit ModeGuard(lpk_ctx *c) : ctx(c), saved(c->cluster_mode) {
    if (saved == 0) ctx->cluster_mode = 3;
  }
  ~ModeGuard() { ctx->cluster_mode = saved; }
};

}  // namespace

LPK_API lpk_status lpk_lp_solve_batch(int32_t count, lpk_problem *const *problems, const double *const *b,
                                      const double *const *c, const lpk_options *opt, double *const *x,
                                      double *const *y, double *const *s, lpk_info *info, int32_t on_device) {
  if (count < 0 || (count > 0 && (!problems || !b || !c || !x || !y || !s || !info))) return LPK_INVALID_ARG;
  // every problem on its own context; no context on the grid path
  for (int i = 0; i < count; ++i) {
    if (!problems[i] || !problems[i]->ctx) return LPK_INVALID_ARG;
    lpk_ctx *ci = problems[i]->ctx;
    if (ci->cluster_mode == 1) {
      ci->err = "lpk_lp_solve_batch: a context on the grid path cannot share the GPU";
      return LPK_INVALID_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (problems[j]->ctx == ci) {
        ci->err = "lpk_lp_solve_batch: every problem needs its own context";
        return LPK_INVALID_ARG;
      }
  }
  std::vector<lpk_status> st(count, LPK_OK);
  auto run = [&](int i) {
    lpk_problem *P = problems[i];
    ModeGuard g(P->ctx);
    st[i] = lpk_lp_solve(P->ctx, P, b[i], c[i], opt, x[i], y[i], s[i], &info[i], on_device);
    if (st[i] != LPK_OK) info[i].status = st[i];
  };
  std::vector<std::thread> th;
  th.reserve(count > 0 ? count - 1 : 0);
  try {
    for (int i = 1; i < count; ++i) th.emplace_back(run, i);
  } catch (...) {
    for (auto &t : th) t.join();
    return LPK_OOM;
  }
  if (count > 0) run(0);
  for (auto &t : th) t.join();
  for (int i = 0; i < count; ++i)
    if (st[i] != LPK_OK) return st[i];
  return LPK_OK;
}

// ---------------------------------------------------------------------------
// continuous-batching server
// ---------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  int32_t m = 0, n = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> val, b, c, x, y, s;
  lpk_options opt{};
  int64_t mem = 0;       // device bytes charged at admission
  lpk_request_result res{};
  bool done = false;
};

// Device memory one request holds while it runs: the prepared problem with
// prepare's temporaries (at most 80 B per nonzero), the interior-point and
// Krylov workspaces, and for AB-GMRES (or a BA-GMRES corrector) the basis
// sized to the iteration cap (capped at 16 GiB, as the kernel caps it).
int64_t request_bytes(const Request &r, int num_sms) {
  const int64_t m = r.m, n = r.n, nnz = (int64_t)r.ci.size();
  int64_t bytes = 80 * nnz + 8 * (24 * m + 32 * n) + (1 << 20);
  if (r.opt.solver == LPK_ABGMRES || r.opt.corrector == 1) {  // AB-GMRES or BA-GMRES basis
    const int64_t kmax = r.opt.max_krylov > 0 ? r.opt.max_krylov : m;
    const int64_t ld = (kmax + 4) & ~int64_t(3);
    const int64_t S = num_sms > 16 ? num_sms : 16;
    const int64_t gm = ld * (m + 6 + S) + kmax * (kmax + 1) / 2 + m + 4;
    bytes += 8 * std::min<int64_t>(gm, int64_t(16) << 27);
  }
  return bytes;
}

}  // namespace

struct lpk_server {
  lpk_server_config cfg{};
  int num_sms = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_ticket = 1;
  int64_t mem_in_use = 0, mem_peak = 0, running = 0, completed = 0;
  bool stop = false;
  std::vector<std::thread> lanes;
  std::vector<lpk_ctx *> ctxs;
  std::vector<cudaStream_t> streams;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  // first pending request (in arrival order) whose memory fits the budget;
  // with nothing running, the head is admitted whatever its size
  std::shared_ptr<Request> admit_locked() {
    for (auto it = pending.begin(); it != pending.end(); ++it) {
      if (mem_in_use + (*it)->mem <= cfg.mem_budget || (running == 0 && it == pending.begin())) {
        auto r = *it;
        pending.erase(it);
        mem_in_use += r->mem;
        if (mem_in_use > mem_peak) mem_peak = mem_in_use;
        ++running;
        return r;
      }
    }
    return nullptr;
  }

  void lane_main(int k) {
    lpk_ctx *ctx = ctxs[k];
    cudaSetDevice(cfg.device);
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          if (stop) return true;
          r = admit_locked();
          return r != nullptr;
        });
        if (!r) return;  // stopping
      }
      r->res.t_start = now();
      r->res.lane = k;
      lpk_matrix A{};
      A.m = r->m;
      A.n = r->n;
      A.nnz = (int64_t)r->ci.size();
      A.row_ptr = r->rp.data();
      A.col_idx = r->ci.data();
      A.val = r->val.data();
      A.on_device = 0;
      lpk_problem *P = nullptr;
      lpk_status st = lpk_prepare(ctx, &A, cfg.color_seed, &P);
      if (st == LPK_OK) {
        r->x.assign(r->n, 0.0);
        r->y.assign(r->m, 0.0);
        r->s.assign(r->n, 0.0);
        st = lpk_lp_solve(ctx, P, r->b.data(), r->c.data(), &r->opt, r->x.data(), r->y.data(), r->s.data(),
                          &r->res.info, 0);
      }
      if (P) lpk_problem_free(P);
      r->res.status = st;
      if (st != LPK_OK && r->res.info.status == LPK_OK) r->res.info.status = st;
      if (st != LPK_OK) {
        std::strncpy(r->res.error, lpk_last_error(ctx), sizeof(r->res.error) - 1);
        r->res.error[sizeof(r->res.error) - 1] = '\0';
      }
      r->res.t_end = now();
      {
        std::lock_guard<std::mutex> lk(mu);
        mem_in_use -= r->mem;
        --running;
        ++completed;
        r->done = true;
      }
      cv_done.notify_all();
      cv_work.notify_all();  // memory came back: another lane may admit
    }
  }
};

LPK_API void lpk_server_default_config(lpk_server_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->lanes = 16;
  cfg->mem_budget = 0;
  cfg->color_seed = 0x5EEDull;
}

LPK_API lpk_status lpk_server_create(lpk_server **out, const lpk_server_config *cfg_in) {
  if (!out) return LPK_INVALID_ARG;
  *out = nullptr;
  lpk_server_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else lpk_server_default_config(&cfg);
  if (cfg.lanes < 1 || cfg.lanes > 256 || cfg.mem_budget < 0) return LPK_INVALID_ARG;
  if (cudaSetDevice(cfg.device) != cudaSuccess) return LPK_CUDA_ERROR;
  if (cfg.mem_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return LPK_CUDA_ERROR;
    cfg.mem_budget = (int64_t)(fr / 2);
  }
  lpk_server *S = new (std::nothrow) lpk_server();
  if (!S) return LPK_OOM;
  S->cfg = cfg;
  S->t0 = Clock::now();
  cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, cfg.device);
  for (int k = 0; k < cfg.lanes; ++k) {
    cudaStream_t st = nullptr;
    lpk_ctx *ctx = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        lpk_create(&ctx, cfg.device, st) != LPK_OK) {
      if (st) cudaStreamDestroy(st);
      lpk_server_destroy(S);
      return LPK_CUDA_ERROR;
    }
    lpk_set_exec(ctx, LPK_EXEC_BATCH, 0);
    S->streams.push_back(st);
    S->ctxs.push_back(ctx);
  }
  try {
    for (int k = 0; k < cfg.lanes; ++k) S->lanes.emplace_back([S, k] { S->lane_main(k); });
  } catch (...) {
    lpk_server_destroy(S);
    return LPK_OOM;
  }
  *out = S;
  return LPK_OK;
}

LPK_API void lpk_server_destroy(lpk_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->pending.clear();
  }
  S->cv_work.notify_all();
  for (auto &t : S->lanes) t.join();
  for (lpk_ctx *c : S->ctxs) lpk_destroy(c);
  for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
  delete S;
}

LPK_API double lpk_server_now(const lpk_server *S) { return S ? S->now() : 0.0; }

LPK_API lpk_status lpk_server_submit(lpk_server *S, const lpk_matrix *A, const double *b, const double *c,
                                     const lpk_options *opt, int64_t *ticket) {
  if (!S || !A || !b || !c || !ticket || A->on_device || A->m < 0 || A->n < 0 || A->nnz < 0 ||
      !A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val)))
    return LPK_INVALID_ARG;
  if (A->row_ptr[0] != 0 || A->row_ptr[A->m] != A->nnz) return LPK_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->res.t_submit = S->now();
  r->m = A->m;
  r->n = A->n;
  r->rp.assign(A->row_ptr, A->row_ptr + A->m + 1);
  r->ci.assign(A->col_idx, A->col_idx + A->nnz);
  r->val.assign(A->val, A->val + A->nnz);
  r->b.assign(b, b + A->m);
  r->c.assign(c, c + A->n);
  if (opt) r->opt = *opt;
  else lpk_default_options(&r->opt);
  r->mem = request_bytes(*r, S->num_sms);
  r->res.mem_bytes = r->mem;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return LPK_INVALID_ARG;
    r->ticket = S->next_ticket++;
    S->pending.push_back(r);
    S->all[r->ticket] = r;
  }
  S->cv_work.notify_one();
  *ticket = r->ticket;
  return LPK_OK;
}

LPK_API lpk_status lpk_server_wait(lpk_server *S, int64_t ticket, double timeout_s, double *x, double *y,
                                   double *s, lpk_request_result *res) {
  if (!S) return LPK_INVALID_ARG;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return LPK_INVALID_ARG;
    r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_s < 0) {
      S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
      return LPK_TIMEOUT;
    }
    S->all.erase(ticket);
  }
  if (x && !r->x.empty()) std::memcpy(x, r->x.data(), sizeof(double) * r->x.size());
  if (y && !r->y.empty()) std::memcpy(y, r->y.data(), sizeof(double) * r->y.size());
  if (s && !r->s.empty()) std::memcpy(s, r->s.data(), sizeof(double) * r->s.size());
  if (res) *res = r->res;
  return LPK_OK;
}

LPK_API lpk_status lpk_server_stats(lpk_server *S, lpk_server_stats_t *out) {
  if (!S || !out) return LPK_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  out->pending = (int64_t)S->pending.size();
  out->running = S->running;
  out->completed = S->completed;
  out->mem_in_use = S->mem_in_use;
  out->mem_peak = S->mem_peak;
  out->mem_budget = S->cfg.mem_budget;
  out->lanes = S->cfg.lanes;
  out->reserved = 0;
  return LPK_OK;
}
