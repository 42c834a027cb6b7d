// krylov.cu -- persistent cooperative kernels for the search-direction solve
// (Sec. 3): CGNE (Algorithm 2) and MRNE (Algorithm 3) with NE-SSOR inner
// iterations (Algorithm 5), plus a sweep-only mode for NE-SSOR / NE-SOR
// (Algorithm 6).  One launch runs a whole Krylov solve: no host round trip per
// iteration.
//
// Phases are separated by a software grid barrier (monotonic arrival counter,
// bounded wait on %globaltimer; on expiry the kernel records LPK_TIMEOUT and
// every CTA returns).  Reductions are two-stage and deterministic: each CTA
// writes its partial, and after the barrier every CTA sums all partials in
// CTA order, so all CTAs take identical control decisions.
//
// Inner sweep.  Rows are stored color by color; the rows of one color share
// no column, so a warp per row computes d_i = omega (g_i - (alpha_i, u))
// (unit row norms after the Sec. 3.5 scaling), z_i += d_i and scatters
// u += d_i alpha_i without atomics.  A barrier separates colors.  Forward
// passes take colors 0..C-1, backward passes C-1..0, which is the exact
// reverse of the forward row order, as NE-SSOR requires.
//
// Recurrences (row-space shadows give dy with dw = A_hat^T dy, no extra product):
//  MRNE: t = A_hat p; [vt, v] = SSOR(t); alpha = gamma / (v, p) with
//        (v, p) = (vt, t) accumulated in the last sweep pass; dw += alpha p;
//        dy += alpha pt; g -= alpha t; q -= alpha v; qt -= alpha vt;
//        gamma' = ||q||^2; p = q + beta p; pt = qt + beta pt.
//  CGNE: alpha = gamma / (q, q); dw += alpha q; dy += alpha qt; g -= alpha A_hat q;
//        [z, u] = SSOR(g); gamma' = (g, z) (accumulated in the last pass);
//        q = u + beta q; qt = z + beta qt.
//  The p (MRNE) and q (CGNE) updates are fused into the next product: the
//  product gathers q + beta p_old inline while the new p is written to a
//  second buffer, saving one barrier per iteration.
#include <cstdio>

#include "lpk_internal.cuh"

namespace {

constexpr int KTPB = 512;
constexpr int KWPB = KTPB / 32;
constexpr int RC = 4;                 // row entries per lane kept in registers
constexpr unsigned long long TIMEOUT_NS = 5000000000ull;  // 5 s per barrier wait

enum { M_MRNE = 0, M_CGNE = 1, M_SWEEP = 7, M_SWEEP_SSOR = 8, M_SWEEP_SOR = 9 };
enum { EXIT_CONV = 0, EXIT_MAXIT = 1, EXIT_BREAK = 2, EXIT_STALL = 3 };

struct KrylovCtl {
  unsigned long long bar;
  int status;
  int iters, restarts, converged, breakdown, iters32, escalations;
  double res0, res;
  long long passes, rows, cols, barriers;   // work counters of the launch
};

struct KArgs {
  int m, n, nc;
  const int *rp, *ci, *cptr;
  const double *a64;
  const float *a32;
  const int *cp, *ri;              // CSC of A_hat (rows are sweep positions)
  const double *aht;               // A_hat values in CSC order
  int wy;                          // mixed precision: w-space images by FP64 CSC products
  int f32;                         // inner sweeps start in FP32
  int stall;                       // FP32 phase ends after this many iterations without a new best
  double *uw;                      // n-space workspace of the CGNE wy path
  int ell;
  double omega;
  const double *f;
  double tol;
  int maxit;
  int method;
  double cycle_tol;                // a cycle ends at ||g|| <= cycle_tol * ||g at cycle start||
  int max_restarts;
  double *dw, *dy;                 // outputs (n), (m)
  double *g, *t, *qt, *pt, *by;    // m-space workspace
  double *q, *p0, *p1, *bw;        // n-space workspace
  void *u, *z;                     // sweep state: u (n), z (m), TI
  double *part;                    // [8 * gridDim]
  KrylovCtl *ctl;
  double *hist;
  // sweep-only mode outputs
  double *out_z, *out_u;
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// work counters (every thread keeps identical copies; CTA 0 reports them)
struct Counters {
  long long passes = 0, rows = 0, cols = 0;
};

struct GridBar {
  unsigned long long *cnt;
  int *status;
  unsigned long long epoch;
  unsigned nblk;
  // returns false if the wait timed out or another CTA reported a failure
  // The CTA barrier orders this CTA's writes before thread 0's release-add;
  // the acquire poll orders every later read after all CTAs' writes.
  __device__ __forceinline__ bool sync(int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
      epoch += 1;
      const unsigned long long target = epoch * (unsigned long long)nblk;
      asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(cnt) : "memory");
      int ok = 1;
      unsigned it = 0;
      unsigned long long t0 = 0;
      while (ld_acquire(cnt) < target) {
        if ((++it & 255u) == 0u) {
          if (*(volatile int *)status != 0) { ok = 0; break; }
          unsigned long long now = globaltimer();
          if (t0 == 0) t0 = now;
          else if (now - t0 > TIMEOUT_NS) { atomicCAS(status, 0, (int)LPK_TIMEOUT); ok = 0; break; }
        }
      }
      *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
  }
};

// CTA partial sums -> part[k * G + rank] (thread 0 writes)
template <int K>
__device__ __forceinline__ void put_partials(double (&v)[K], double *part, double *sred) {
  block_sum<K>(v, sred);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[k * gridDim.x + blockIdx.x] = v[k];
  }
}
// after a barrier: every CTA sums the G partials of slots [0, K) in CTA order
template <int K>
__device__ __forceinline__ void get_sums(double (&v)[K], const double *part, double *sred) {
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = threadIdx.x < gridDim.x ? __ldcg(&part[k * gridDim.x + threadIdx.x]) : 0.0;
  block_sum<K>(v, sred);
}

template <typename TI>
__device__ __forceinline__ const TI *ahat(const KArgs &A);
template <>
__device__ __forceinline__ const double *ahat<double>(const KArgs &A) { return A.a64; }
template <>
__device__ __forceinline__ const float *ahat<float>(const KArgs &A) { return A.a32; }

// One row of an inner sweep (warp-cooperative): d = omega (g_r - (a_r, u)),
// z_r += d, u += d a_r.  Matrix values are TV (FP64, or the FP32 copy in mixed
// precision); u, z and all arithmetic are FP64, so the preconditioner is the
// exact SSOR operator of the (rounded) matrix: linear and, for NE-SSOR, SPD.
// Returns the row's z after the update (lane 0 only meaningful).
template <typename TV>
__device__ __forceinline__ double sweep_row(int r, const int *__restrict__ rp, const int *__restrict__ ci,
                                            const TV *__restrict__ a, double *u, double *z, double gr,
                                            double om, bool first) {
  const int lane = threadIdx.x & 31;
  const int k0 = __ldg(rp + r), k1 = __ldg(rp + r + 1);
  const int len = k1 - k0;
  double s = 0.0;
  if (len <= 32 * RC) {
    int cv[RC];
    double av[RC], uv[RC];
#pragma unroll
    for (int e = 0; e < RC; ++e) {
      int k = k0 + lane + 32 * e;
      if (k < k1) {
        cv[e] = __ldg(ci + k);
        av[e] = (double)__ldg(a + k);
        uv[e] = ldcg(u + cv[e]);
        s += av[e] * uv[e];
      }
    }
    s = warp_sum(s);
    const double d = om * (gr - s);
#pragma unroll
    for (int e = 0; e < RC; ++e) {
      int k = k0 + lane + 32 * e;
      if (k < k1) u[cv[e]] = uv[e] + d * av[e];
    }
    double zn = d;
    if (lane == 0) {
      zn = first ? d : ldcg(z + r) + d;
      z[r] = zn;
    }
    return zn;
  } else {
    for (int k = k0 + lane; k < k1; k += 32) s += (double)__ldg(a + k) * ldcg(u + __ldg(ci + k));
    s = warp_sum(s);
    const double d = om * (gr - s);
    for (int k = k0 + lane; k < k1; k += 32) {
      int c = __ldg(ci + k);
      u[c] = ldcg(u + c) + d * (double)__ldg(a + k);
    }
    double zn = d;
    if (lane == 0) {
      zn = first ? d : ldcg(z + r) + d;
      z[r] = zn;
    }
    return zn;
  }
}

// A full application of the inner iterations on input g (m, double):
// SSOR (2 passes per sweep) or SOR (1 pass).  u must be zero on entry.  If
// acc != nullptr, each lane 0 adds z_r * g_r at the row's last visit.
// Ends with a barrier after the last color.  Returns false on barrier failure.
template <typename TV>
__device__ bool inner_sweeps(const KArgs &A, GridBar &G, int *s_ok, const double *g, bool ssor,
                             double *acc, Counters &C) {
  const TV *a = ahat<TV>(A);
  double *u = (double *)A.u;
  double *z = (double *)A.z;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * KWPB + (threadIdx.x >> 5), GW = gridDim.x * KWPB;
  const double om = A.omega;
  const int passes = ssor ? 2 * A.ell : A.ell;
  C.passes += passes;
  for (int ps = 0; ps < passes; ++ps) {
    const bool backward = ssor && (ps & 1);
    const bool lastpass = ps == passes - 1;
    for (int cc = 0; cc < A.nc; ++cc) {
      const int c = backward ? A.nc - 1 - cc : cc;
      const int r0 = __ldg(A.cptr + c), r1 = __ldg(A.cptr + c + 1);
      for (int r = r0 + gw; r < r1; r += GW) {
        const double gd = ldcg(g + r);
        const double zn = sweep_row<TV>(r, A.rp, A.ci, a, u, z, gd, om, ps == 0);
        if (lastpass && acc && lane == 0) *acc += zn * gd;
      }
      if (!(lastpass && cc == A.nc - 1 && acc)) {
        if (!G.sync(s_ok)) return false;
      }
    }
  }
  return true;
}

// t = A_hat x in double, x gathered as xa[c] + beta * xb[c] (xb may be null)
template <typename TU>
__device__ __forceinline__ void spmv_rows(const KArgs &A, const TU *xa, double beta, const double *xb,
                                          double *t, const double *sub /*t = sub - Ax if non-null*/) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * KWPB + (threadIdx.x >> 5), GW = gridDim.x * KWPB;
  for (int r = gw; r < A.m; r += GW) {
    const int k0 = __ldg(A.rp + r), k1 = __ldg(A.rp + r + 1);
    double s = 0.0;
    for (int k = k0 + lane; k < k1; k += 32) {
      const int c = __ldg(A.ci + k);
      double xv = (double)ldcg(xa + c);
      if (xb) xv += beta * ldcg(xb + c);
      s += __ldg(A.a64 + k) * xv;
    }
    s = warp_sum(s);
    if (lane == 0) t[r] = sub ? ldcg(sub + r) - s : s;
  }
}

// out = A_hat^T x in double through the CSC (warp per column); returns this
// thread's share of ||out||^2
template <typename TX>
__device__ __forceinline__ double csc_products(const KArgs &A, const TX *x, double *out) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * KWPB + (threadIdx.x >> 5), GW = gridDim.x * KWPB;
  double acc = 0.0;
  for (int j = gw; j < A.n; j += GW) {
    const int q0 = __ldg(A.cp + j), q1 = __ldg(A.cp + j + 1);
    double s = 0.0;
    for (int q = q0 + lane; q < q1; q += 32) s += __ldg(A.aht + q) * (double)ldcg(x + __ldg(A.ri + q));
    s = warp_sum(s);
    if (lane == 0) {
      out[j] = s;
      acc += s * s;
    }
  }
  return acc;
}

// Sweep state accessors (u, z are FP64 in both precisions; f32 selects the
// FP32 copy of the matrix values inside the sweeps).
struct Inner {
  void *u, *z;
  bool f32;
  __device__ __forceinline__ double zget(int i) const { return ldcg((const double *)z + i); }
  __device__ __forceinline__ double uget(int j) const { return ldcg((const double *)u + j); }
};

__device__ __forceinline__ double csc_z(const KArgs &A, const Inner &I, double *out) {
  return csc_products<double>(A, (const double *)I.z, out);
}

template <int METH, typename TV>
__global__ void __launch_bounds__(KTPB, 1) k_krylov(KArgs A) {
  __shared__ double sred[8 * KWPB];
  __shared__ int s_ok;
  GridBar G{&A.ctl->bar, &A.ctl->status, 0ull, gridDim.x};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, NT = gridDim.x * blockDim.x;
  const int m = A.m, n = A.n;
  Inner I{A.u, A.z, A.f32 != 0};
  Counters Cn;
  double *ud = (double *)A.u;  // zeroing as doubles clears either representation

  // ---- sweep-only mode (lpk_sweep) ----------------------------------------
  if (METH == M_SWEEP) {
    for (int j = tid; j < n; j += NT) ud[j] = 0.0;
    if (!G.sync(&s_ok)) return;
    if (!inner_sweeps<TV>(A, G, &s_ok, A.f, A.method == M_SWEEP_SSOR, nullptr, Cn)) return;
    for (int j = tid; j < n; j += NT) A.out_u[j] = I.uget(j);
    for (int i = tid; i < m; i += NT) A.out_z[i] = I.zget(i);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      A.ctl->passes = Cn.passes;
      A.ctl->barriers = (long long)G.epoch;
    }
    return;
  }

  // ---- start: g = f, dw = 0, dy = 0, u = 0; ||f|| -------------------------
  double res0 = 0.0;
  {
    double v[1] = {0.0};
    for (int i = tid; i < m; i += NT) {
      double fi = A.f[i];
      A.g[i] = fi;
      A.dy[i] = 0.0;
      v[0] += fi * fi;
    }
    for (int j = tid; j < n; j += NT) {
      A.dw[j] = 0.0;
      ud[j] = 0.0;
    }
    if (METH == M_CGNE) {  // the starting iterate is the best one so far
      for (int j = tid; j < n; j += NT) A.bw[j] = 0.0;
      for (int i = tid; i < m; i += NT) A.by[i] = 0.0;
    }
    put_partials<1>(v, A.part, sred);
    if (!G.sync(&s_ok)) return;
    get_sums<1>(v, A.part, sred);
    res0 = sqrt(v[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      A.ctl->res0 = res0;
      if (A.hist) A.hist[0] = res0;
    }
    if (res0 == 0.0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) { A.ctl->converged = 1; A.ctl->res = 0.0; }
      return;
    }
  }
  const double target = A.tol * res0;  // identical in every CTA
  int k = 0, k32 = 0, restarts = 0, escal = 0, reason = EXIT_MAXIT;
  double gnorm = res0;
  double *p_cur = A.p0, *p_nxt = A.p1;
  const bool flex = false;  // fixed linear preconditioner in both precisions: the paper's beta

  for (;;) {  // restart loop
    double gamma = 0.0, beta = 0.0;
    bool first = true;
    reason = EXIT_MAXIT;
    double best = gnorm;
    int best_k = k;
    if (METH == M_MRNE) {
      // q0 = A^T C g0 (w-space), qt0 = C g0
      if (!inner_sweeps<TV>(A, G, &s_ok, A.g, true, nullptr, Cn)) return;
      double v[1] = {0.0};
      if (A.wy) {
        ++Cn.cols;
        v[0] = csc_z(A, I, A.q);  // q0 = A_hat^T z in FP64
      } else {
        for (int j = tid; j < n; j += NT) {
          double qj = I.uget(j);
          A.q[j] = qj;
          v[0] += qj * qj;
        }
      }
      for (int i = tid; i < m; i += NT) A.qt[i] = I.zget(i);
      put_partials<1>(v, A.part, sred);
      if (!G.sync(&s_ok)) return;
      get_sums<1>(v, A.part, sred);
      gamma = v[0];
      while (true) {
        if (gnorm <= target) { reason = EXIT_CONV; break; }
        if (k >= A.maxit) { reason = EXIT_MAXIT; break; }
        if (I.f32 && k - best_k >= A.stall) { reason = EXIT_STALL; break; }
        // P1: p = q + beta p_old (fused), pt = qt + beta pt, t = A_hat p, u = 0
        for (int j = tid; j < n; j += NT) {
          double qj = ldcg(A.q + j);
          p_nxt[j] = first ? qj : qj + beta * ldcg(p_cur + j);
          ud[j] = 0.0;
        }
        for (int i = tid; i < m; i += NT) {
          double qi = ldcg(A.qt + i);
          A.pt[i] = first ? qi : qi + beta * ldcg(A.pt + i);
        }
        ++Cn.rows;
        spmv_rows<double>(A, A.q, first ? 0.0 : beta, first ? nullptr : p_cur, A.t, nullptr);
        { double *tmp = p_cur; p_cur = p_nxt; p_nxt = tmp; }
        first = false;
        if (!G.sync(&s_ok)) return;
        // P2: [vt, v] = SSOR(t), (v, p) = (vt, t)
        double acc[1] = {0.0};
        if (!inner_sweeps<TV>(A, G, &s_ok, A.t, true, &acc[0], Cn)) return;
        put_partials<1>(acc, A.part, sred);
        if (!G.sync(&s_ok)) return;
        get_sums<1>(acc, A.part, sred);
        const double vp = acc[0];
        if (!(vp > 0.0) || !(gamma > 0.0) || !isfinite(vp)) { reason = EXIT_BREAK; break; }
        const double alpha = gamma / vp;
        // P3: updates and norms
        double w[2] = {0.0, 0.0};
        for (int j = tid; j < n; j += NT) {
          double pj = ldcg(p_cur + j);
          A.dw[j] = ldcg(A.dw + j) + alpha * pj;
          if (!A.wy) {
            double qj = ldcg(A.q + j) - alpha * I.uget(j);
            A.q[j] = qj;
            w[0] += qj * qj;
          }
        }
        for (int i = tid; i < m; i += NT) {
          A.dy[i] = ldcg(A.dy + i) + alpha * ldcg(A.pt + i);
          double gi = ldcg(A.g + i) - alpha * ldcg(A.t + i);
          A.g[i] = gi;
          A.qt[i] = ldcg(A.qt + i) - alpha * I.zget(i);
          w[1] += gi * gi;
        }
        put_partials<2>(w, A.part, sred);
        if (!G.sync(&s_ok)) return;
        get_sums<2>(w, A.part, sred);
        double gnew = w[0];
        if (A.wy) {  // P4: q = A_hat^T qt in FP64; gamma' = ||q||^2 and (q_old, q)
          const int lane = threadIdx.x & 31;
          const int gw = blockIdx.x * KWPB + (threadIdx.x >> 5), GW = gridDim.x * KWPB;
          double w2[2] = {0.0, 0.0};
          ++Cn.cols;
          for (int j = gw; j < n; j += GW) {
            const int q0 = __ldg(A.cp + j), q1 = __ldg(A.cp + j + 1);
            double sacc = 0.0;
            for (int q = q0 + lane; q < q1; q += 32) sacc += __ldg(A.aht + q) * ldcg(A.qt + __ldg(A.ri + q));
            sacc = warp_sum(sacc);
            if (lane == 0) {
              const double qo = ldcg(A.q + j);
              A.q[j] = sacc;
              w2[0] += sacc * sacc;
              w2[1] += qo * sacc;
            }
          }
          put_partials<2>(w2, A.part, sred);
          if (!G.sync(&s_ok)) return;
          get_sums<2>(w2, A.part, sred);
          gnew = w2[0];
          beta = flex ? (w2[0] - w2[1]) / gamma : w2[0] / gamma;
        } else {
          beta = gnew / gamma;
        }
        gamma = gnew;
        ++k;
        if (I.f32) ++k32;
        gnorm = sqrt(w[1]);
        if (A.hist && blockIdx.x == 0 && threadIdx.x == 0) A.hist[k] = gnorm;
        if (gnorm < best) { best = gnorm; best_k = k; }
      }
    } else {  // CGNE
      // z0 = C g0, u0 = A^T z0, gamma0 = (g0, z0)
      double acc[1] = {0.0};
      if (!inner_sweeps<TV>(A, G, &s_ok, A.g, true, &acc[0], Cn)) return;
      put_partials<1>(acc, A.part, sred);
      if (!G.sync(&s_ok)) return;
      get_sums<1>(acc, A.part, sred);
      gamma = acc[0];
      if (A.wy) {  // u0 = A_hat^T z0 in FP64
        ++Cn.cols;
        csc_z(A, I, A.uw);
        if (!G.sync(&s_ok)) return;
      }
      bool save_best = false;
      while (true) {
        if (gnorm <= target) { reason = EXIT_CONV; break; }
        if (k >= A.maxit) { reason = EXIT_MAXIT; break; }
        if (I.f32 && k - best_k >= A.stall) { reason = EXIT_STALL; break; }
        // P1: q = u + beta q_old, qt = z + beta qt, t = A_hat q, (q, q)
        double v[1] = {0.0};
        for (int j = tid; j < n; j += NT) {
          double uj = A.wy ? ldcg(A.uw + j) : I.uget(j);
          double qj = first ? uj : uj + beta * ldcg(A.q + j);
          p_nxt[j] = qj;
          v[0] += qj * qj;
        }
        for (int i = tid; i < m; i += NT) {
          double zi = I.zget(i);
          A.qt[i] = first ? zi : zi + beta * ldcg(A.qt + i);
        }
        if (save_best) {  // keep the minimum-residual iterate (Sec. 4.2)
          for (int j = tid; j < n; j += NT) A.bw[j] = ldcg(A.dw + j);
          for (int i = tid; i < m; i += NT) A.by[i] = ldcg(A.dy + i);
        }
        ++Cn.rows;
        if (A.wy)
          spmv_rows<double>(A, A.uw, first ? 0.0 : beta, first ? nullptr : A.q, A.t, nullptr);
        else
          spmv_rows<double>(A, (const double *)A.u, first ? 0.0 : beta, first ? nullptr : A.q, A.t, nullptr);
        put_partials<1>(v, A.part, sred);
        first = false;
        if (!G.sync(&s_ok)) return;
        get_sums<1>(v, A.part, sred);
        const double qq = v[0];
        if (!(qq > 0.0) || !(gamma > 0.0) || !isfinite(gamma)) { reason = EXIT_BREAK; break; }
        const double alpha = gamma / qq;
        // P2: dw += alpha q, dy += alpha qt, g -= alpha t, u = 0, ||g||, (g, z_old)
        double w[2] = {0.0, 0.0};
        for (int j = tid; j < n; j += NT) {
          double qj = ldcg(p_nxt + j);
          A.q[j] = qj;
          A.dw[j] = ldcg(A.dw + j) + alpha * qj;
          ud[j] = 0.0;
        }
        for (int i = tid; i < m; i += NT) {
          A.dy[i] = ldcg(A.dy + i) + alpha * ldcg(A.qt + i);
          double gi = ldcg(A.g + i) - alpha * ldcg(A.t + i);
          A.g[i] = gi;
          w[0] += gi * gi;
          if (flex) w[1] += gi * I.zget(i);
        }
        put_partials<2>(w, A.part, sred);
        if (!G.sync(&s_ok)) return;
        get_sums<2>(w, A.part, sred);
        ++k;
        if (I.f32) ++k32;
        gnorm = sqrt(w[0]);
        if (A.hist && blockIdx.x == 0 && threadIdx.x == 0) A.hist[k] = gnorm;
        save_best = gnorm < best;
        if (save_best) { best = gnorm; best_k = k; }
        if (gnorm <= target) { reason = EXIT_CONV; break; }
        if (k >= A.maxit) { reason = EXIT_MAXIT; break; }
        // P3: [z, u] = SSOR(g), gamma' = (g, z)
        double a2[1] = {0.0};
        if (!inner_sweeps<TV>(A, G, &s_ok, A.g, true, &a2[0], Cn)) return;
        put_partials<1>(a2, A.part, sred);
        if (!G.sync(&s_ok)) return;
        get_sums<1>(a2, A.part, sred);
        beta = flex ? (a2[0] - w[1]) / gamma : a2[0] / gamma;
        gamma = a2[0];
        if (A.wy) {
          ++Cn.cols;
          csc_z(A, I, A.uw);
          if (!G.sync(&s_ok)) return;
        }
      }
      if (reason != EXIT_CONV && best < gnorm) {
        // bw/by hold the minimum-residual iterate (the current one is worse)
        for (int j = tid; j < n; j += NT) A.dw[j] = ldcg(A.bw + j);
        for (int i = tid; i < m; i += NT) A.dy[i] = ldcg(A.by + i);
        if (!G.sync(&s_ok)) return;
      }
    }
    // ---- explicit residual g = f - A_hat dw; restart when it disagrees ------
    if (A.wy) {  // dw = A_hat^T dy in FP64 keeps the two spaces consistent
      ++Cn.cols;
      csc_products<double>(A, A.dy, A.dw);
      if (!G.sync(&s_ok)) return;
    }
    double v[1] = {0.0};
    ++Cn.rows;
    spmv_rows<double>(A, A.dw, 0.0, nullptr, A.g, A.f);
    for (int j = tid; j < n; j += NT) ud[j] = 0.0;
    if (!G.sync(&s_ok)) return;
    for (int i = tid; i < m; i += NT) {
      double gi = ldcg(A.g + i);
      v[0] += gi * gi;
    }
    put_partials<1>(v, A.part, sred);
    if (!G.sync(&s_ok)) return;
    get_sums<1>(v, A.part, sred);
    const double res = sqrt(v[0]);
    gnorm = res;
    if (METH == M_CGNE) {  // a restart starts from the current iterate
      for (int j = tid; j < n; j += NT) A.bw[j] = ldcg(A.dw + j);
      for (int i = tid; i < m; i += NT) A.by[i] = ldcg(A.dy + i);
    }
    // mixed precision: a stalled FP32 phase, or an FP32 recurrence the explicit
    // residual does not confirm, continues with FP64 inner sweeps
    const bool escalate = res > target && I.f32 && k < A.maxit &&
                          (reason == EXIT_STALL || reason == EXIT_CONV);
    if (escalate) {
      I.f32 = false;
      ++escal;
      continue;
    }
    if (res <= target || reason != EXIT_CONV || restarts >= A.max_restarts || k >= A.maxit) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.ctl->res = res;
        A.ctl->converged = res <= target;
        A.ctl->breakdown = reason == EXIT_BREAK;
      }
      break;
    }
    ++restarts;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.ctl->passes = Cn.passes;
    A.ctl->rows = Cn.rows;
    A.ctl->cols = Cn.cols;
    A.ctl->barriers = (long long)G.epoch;
    A.ctl->iters = k;
    A.ctl->iters32 = k32;
    A.ctl->restarts = restarts;
    A.ctl->escalations = escal;
  }
}

struct Workspace {
  double *g, *t, *qt, *pt, *by, *q, *p0, *p1, *bw, *dwtmp;
  void *u, *z;
};

lpk_status get_ws(lpk_ctx *ctx, DevProblem &P, Workspace &W) {
  const size_t m = P.m > 0 ? P.m : 1, n = P.n > 0 ? P.n : 1;
  const size_t need = sizeof(double) * (6 * m + 6 * n) + 4096;
  if (P.ws_bytes < need) {
    if (P.ws) cudaFree(P.ws);
    P.ws = nullptr;
    P.ws_bytes = 0;
    LPK_CUDA_TRY(ctx, cudaMalloc(&P.ws, need));
    P.ws_bytes = need;
  }
  double *b = (double *)P.ws;
  W.g = b; b += m;
  W.t = b; b += m;
  W.qt = b; b += m;
  W.pt = b; b += m;
  W.by = b; b += m;
  W.z = b; b += m;
  W.q = b; b += n;
  W.p0 = b; b += n;
  W.p1 = b; b += n;
  W.bw = b; b += n;
  W.u = b; b += n;
  W.dwtmp = b; b += n;
  return LPK_OK;
}

lpk_status ensure_kctl(lpk_ctx *ctx) {
  if (ctx->kctl) return LPK_OK;
  LPK_CUDA_TRY(ctx, cudaMalloc(&ctx->kctl, sizeof(KrylovCtl)));
  LPK_CUDA_TRY(ctx, cudaMallocHost(&ctx->h_kctl, sizeof(KrylovCtl)));
  LPK_CUDA_TRY(ctx, cudaMalloc(&ctx->kpart, sizeof(double) * 8 * 4096));
  return LPK_OK;
}

void *kernel_for(int method, int f32) {
  if (method == M_MRNE) return f32 ? (void *)k_krylov<M_MRNE, float> : (void *)k_krylov<M_MRNE, double>;
  if (method == M_CGNE) return f32 ? (void *)k_krylov<M_CGNE, float> : (void *)k_krylov<M_CGNE, double>;
  return f32 ? (void *)k_krylov<M_SWEEP, float> : (void *)k_krylov<M_SWEEP, double>;
}

lpk_status launch(lpk_ctx *ctx, KArgs &A, int slot) {
  void *fn = kernel_for(A.method, A.f32);
  if (ctx->kgrid_cache[slot] == 0) {
    int per_sm = 0;
    LPK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, KTPB, 0));
    if (per_sm < 1) {
      ctx->err = "persistent Krylov kernel does not fit on an SM";
      return LPK_CUDA_ERROR;
    }
    ctx->kgrid_cache[slot] = ctx->num_sms;  // one CTA per SM keeps the barrier cheap
  }
  dim3 grid(ctx->kgrid_cache[slot]), block(KTPB);
  void *args[] = {&A};
  if (!ctx->ev0) {
    LPK_CUDA_TRY(ctx, cudaEventCreate(&ctx->ev0));
    LPK_CUDA_TRY(ctx, cudaEventCreate(&ctx->ev1));
  }
  LPK_CUDA_TRY(ctx, cudaMemsetAsync(ctx->kctl, 0, sizeof(KrylovCtl), ctx->stream));
  LPK_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  LPK_COUNT(ctx);
  LPK_CUDA_TRY(ctx, cudaLaunchCooperativeKernel(fn, grid, block, args, 0, ctx->stream));
  LPK_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  LPK_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_kctl, ctx->kctl, sizeof(KrylovCtl), cudaMemcpyDeviceToHost, ctx->stream));
  LPK_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const KrylovCtl *h = (const KrylovCtl *)ctx->h_kctl;
  float ms = 0.f;
  LPK_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  ctx->stats.krylov_launches++;
  ctx->stats.krylov_ms += ms;
  ctx->stats.krylov_iters += h->iters;
  ctx->stats.sweep_passes += h->passes;
  ctx->stats.row_passes += h->rows;
  ctx->stats.csc_passes += h->cols;
  ctx->stats.barriers += h->barriers;
  if (h->status == LPK_TIMEOUT) {
    ctx->err = "a grid barrier wait of the persistent Krylov kernel timed out";
    return LPK_TIMEOUT;
  }
  return LPK_OK;
}

KArgs base_args(lpk_ctx *ctx, DevProblem &P, Workspace &W, int ell, double omega) {
  KArgs A{};
  A.m = P.m;
  A.n = P.n;
  A.nc = P.n_colors;
  A.rp = P.rp;
  A.ci = P.ci;
  A.cptr = P.color_ptr;
  A.a64 = P.ah64;
  A.a32 = P.ah32;
  A.cp = P.cp;
  A.ri = P.ri;
  A.aht = P.aht;
  A.uw = W.dwtmp;
  A.ell = ell;
  A.omega = omega;
  A.g = W.g; A.t = W.t; A.qt = W.qt; A.pt = W.pt; A.by = W.by;
  A.q = W.q; A.p0 = W.p0; A.p1 = W.p1; A.bw = W.bw;
  A.u = W.u; A.z = W.z;
  A.part = ctx->kpart;
  A.ctl = (KrylovCtl *)ctx->kctl;
  return A;
}

}  // namespace

lpk_status krylov_solve(lpk_ctx *ctx, DevProblem &P, int method, int precision, int ell, double omega,
                        const double *f_hat, double tol, int maxit, double *dw, double *dy_hat,
                        KrylovResult *out, double *hist) {
  if (method != LPK_MRNE && method != LPK_CGNE) {
    ctx->err = "solver not available in the persistent kernel";
    return LPK_INVALID_ARG;
  }
  lpk_status st;
  if ((st = ensure_kctl(ctx)) != LPK_OK) return st;
  Workspace W;
  if ((st = get_ws(ctx, P, W)) != LPK_OK) return st;
  KArgs A = base_args(ctx, P, W, ell, omega);
  A.f = f_hat;
  A.tol = tol;
  A.maxit = maxit;
  A.method = method == LPK_MRNE ? M_MRNE : M_CGNE;
  // FP64: one cycle (plus up to 3 restarts when the explicit residual does not
  // confirm the recurrence); mixed: cycles of 1e-4 reduction each
  // FP64: the paper's recurrences; up to 3 restarts when the explicit residual
  // does not confirm the recurrence.  Mixed: sweeps over the FP32 copy of the
  // scaled matrix with FP64 accumulation, w-space images by FP64 CSC products.
  A.cycle_tol = 0.0;
  A.wy = precision == LPK_MIXED ? 1 : 0;
  A.f32 = precision == LPK_MIXED ? 1 : 0;
  A.stall = 1 << 30;  // no escalation: the FP32-valued preconditioner is a fixed SPD operator
  A.max_restarts = 3;
  A.dw = dw;
  A.dy = dy_hat;
  A.hist = hist;
  st = launch(ctx, A, 0);
  if (st != LPK_OK) return st;
  const KrylovCtl *h = (const KrylovCtl *)ctx->h_kctl;
  out->iters = h->iters;
  out->converged = h->converged;
  out->restarts = h->restarts;
  out->breakdown = h->breakdown;
  out->res0 = h->res0;
  out->res = h->res;
  out->iters32 = h->iters32;
  out->escalations = h->escalations;
  return LPK_OK;
}

lpk_status sweep_only(lpk_ctx *ctx, DevProblem &P, int kind, int precision, int ell, double omega,
                      const double *g_hat, double *z, double *u) {
  lpk_status st;
  if ((st = ensure_kctl(ctx)) != LPK_OK) return st;
  Workspace W;
  if ((st = get_ws(ctx, P, W)) != LPK_OK) return st;
  KArgs A = base_args(ctx, P, W, ell, omega);
  A.f = g_hat;
  A.method = kind == LPK_NE_SOR ? M_SWEEP_SOR : M_SWEEP_SSOR;
  // NE-SOR keeps the w-space iterate in u (n) and the row corrections in z (m)
  A.out_z = z;
  A.out_u = u;
  A.f32 = precision == LPK_MIXED ? 1 : 0;
  return launch(ctx, A, 0);
}
