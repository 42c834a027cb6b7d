"""Benchmark of the search-direction hot path through the C ABI, on seeded
synthetic workloads.

Default (--workload large): the large power-law LP (m = 150,000, n = 434,580,
mean column degree 6, maximum 400, 406 colors).  A step is one lpk_sweep call
(D-scaling and row scaling of Sec. 3.5, then one NE-SOR pass of Algorithm 6
over the FP32 copy of the scaled matrix, mixed precision) followed by one
FP64 product y = A x (lpk_spmv); the value is the NE-sweep bandwidth: the
algorithmic bytes of one NE-SOR pass (the FP32 sweep formula of the scope
table, half of an NE-SSOR sweep) divided by the sweep kernel's CUDA-event
duration, measured live on the launching stream.  The L2 is flushed (256 MB
written) between timed steps.  The same line carries, as secondary keys, the
LP throughput of the degenerate assignment LP (lp_solve: a batch of LPs
solved side by side in mixed precision to gap <= 1e-8, against plain FP64 one
LP at a time) and the first interior-point iterations of the large LP itself
(large_solve), which the paper's method does not bring to gap <= 1e-8 within
its Krylov cap on this family.

Other workloads: --workload assignment|tiny|medium|medium_0.1 time complete
LP solves (a step = a batch of LPs, LPs/s); --workload serving replays the
Poisson stream through the continuous-batching server; --workload large_x8
measures the sparse products on the large matrix replicated 8x (larger than
L2).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload W]
                  [--batch B] [--precision mixed|fp64] [--solver mrne|cgne|abgmres]
                  [--impl lpk|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# one hardware work queue per stream: with the default of 8, the streams of
# more than 8 lanes share queues and a persistent kernel of one lane would
# hold back the launches of another (read when the CUDA context is created)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "LPs solved/s & p99 latency at gap≤1e-8 (mixed vs FP64); NE-sweep HBM GB/s"
UNIT = "LPs/s"
METRIC_SWEEP = METRIC   # the large LP's line reports the NE-sweep part (unit GB/s)
SOLVERS = {"mrne": 0, "cgne": 1, "abgmres": 2}

# workload -> generator options and LPs per step.  max_krylov 40000 is the
# relaxed Krylov cap the paper uses for difficult problems (Sec. 4.2).
WORKLOADS = {
    "large": dict(desc="large sparse LP m=150000 n=434580, power-law column degrees (mean 6, max 400), N(0,1), "
                       "x0/y0/s0 construction; NE-SOR sweep + FP64 SpMV, mixed precision",
                  opts=dict(solver=2, inner_sweeps=1, omega=1.0, max_krylov=40000), batch=1),
    "medium": dict(desc="rank-deficient sparse LP m=20000 n=60000, 8 nnz/col N(0,1), 1% dependent rows",
                   opts=dict(solver=0, inner_sweeps=5, omega=1.0, max_krylov=40000), batch=1),
    "assignment": dict(desc="degenerate assignment LP k=14 (n=38416, m=588), costs U{0..100}",
                       opts=dict(solver=2, inner_sweeps=3, omega=1.0), batch=16),
    "tiny": dict(desc="tiny sparse LP m=50 n=120 ~5% N(0,1)", opts=dict(solver=0, inner_sweeps=1), batch=16),
    "medium_0.1": dict(desc="medium family at scale 0.1 (m=2000 n=6000)",
                       opts=dict(solver=2, inner_sweeps=5, omega=1.0, max_krylov=6000), batch=8),
    "serving": dict(desc="Poisson stream (rate 50/s) of LPs, m log-uniform in [100, 20000], n=3m, 6 nnz/col",
                    opts=dict(solver=2, inner_sweeps=3, omega=1.0), batch=1),
    "large_x8": dict(desc="large LP matrix (m=150000, n=434580, power-law column degrees) replicated 8x "
                          "block-diagonally: SpMV bandwidth, not L2-resident",
                     opts=dict(solver=0, inner_sweeps=1), batch=1),
}


def make_lp(workload, seed_offset=0):
    from paper_1604_07491_gb300 import gen
    if workload == "large":
        return gen.large_lp(1.0)
    if workload == "medium":
        return gen.medium_lp(1.0, seed=gen.SEED_BASE + 2 + 1000 * seed_offset)
    if workload == "medium_0.1":
        return gen.medium_lp(0.1, seed=gen.SEED_BASE + 2 + 1000 * seed_offset)
    if workload == "assignment":
        return gen.assignment_lp(seed=gen.SEED_BASE + 3 + 1000 * seed_offset)
    if workload == "tiny":
        return gen.tiny_lp(seed=gen.SEED_BASE + 1 + 1000 * seed_offset)
    if workload == "serving":
        return gen.serving_lp(seed_offset)
    raise KeyError(workload)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def algorithmic_bytes(stats, m, n, nnz, precision):
    """Bytes the persistent Krylov kernel must move, from its work counters.
    Inner sweep pass: per nonzero the value (8 B FP64 or 4 B FP32 copy), the
    column index (4 B) and one gather plus one scatter of u (8 + 8 B); per row
    the row pointer (4 B), g (8 B) and z read+write (16 B).
    FP64 row pass over A_hat (t = A_hat p, residuals): value + index + gathered
    vector entry (8 + 4 + 8 B) per nonzero, row pointer + result (4 + 8 B) per row.
    CSC pass (w-space image): same per nonzero, 12 B per column.
    Vector work per Krylov iteration: about 12 n-vectors and 12 m-vectors of
    8 B streamed (updates, fused norms and the p/q recurrences).
    AB-GMRES basis: 8 B per row for every m-row pass over a basis vector
    (counted by the kernel: four per vector per iteration, one in V p)."""
    vb = 4 if precision == "mixed" else 8
    per_pass = nnz * (vb + 4 + 16) + m * 28
    per_row = nnz * 20 + m * 12
    per_col = nnz * 20 + n * 12
    per_iter = 8 * (12 * n + 12 * m)
    return (stats["sweep_passes"] * per_pass + stats["row_passes"] * per_row
            + stats["csc_passes"] * per_col + stats["krylov_iters"] * per_iter
            + stats.get("basis_passes", 0) * 8 * m)


def sweep_pass_bytes(nnz, m):
    """Algorithmic bytes of one NE-SOR pass over the FP32 copy of the scaled
    matrix, by the FP32 sweep formula of the scope table (half of its NE-SSOR
    sweep): per nonzero the value and column index (4 + 4 B) and one read and
    one write of the gathered/scattered u entry (4 + 4 B); per row the row
    pointer (8 B), g (4 B) and the z read-modify-write (8 B)."""
    return nnz * 16 + m * 20


def sweep_pass_bytes_moved(nnz, m):
    """The same pass with u kept in FP64, as this implementation does (its
    u gather and scatter move 8 + 8 B per nonzero)."""
    return nnz * 24 + m * 20


def spmv_bytes(nnz, m, n):
    """FP64 y = A x by the scope table's formula: value and column index
    (8 + 4 B) per nonzero, row pointer and result (8 + 8 B) per row, x read
    once (8 B per column)."""
    return nnz * 12 + m * 16 + n * 8


def source_digest(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(kernel_key):
    """DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
    a kernel from the committed ncu record (profiles/ncu_traffic.json), or
    None when the record is missing or the kernel's sources changed since the
    capture (the record stores the SHA-256 of the sources it was taken on)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None, "no ncu record"
    rec = json.load(open(path)).get(kernel_key)
    if not rec:
        return None, "no ncu record for this kernel"
    if rec.get("sources_sha256") != source_digest(rec["sources"]):
        return None, "kernel sources changed since the ncu capture"
    return float(rec["dram_bytes_per_launch"]), rec.get("command", "")


def replica_offsets(rank, batch):
    """Seed offsets of the LPs rank `rank` solves: replicas are independent
    units (weak scaling), every rank gets its own LPs of the family."""
    return [rank * batch + i for i in range(batch)]


def max_over_ranks(value, dist, device=None):
    """The largest value over all ranks (the job's time); the value itself
    without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_throughput(world, batch, steps, total_ms):
    """Whole-job LPs/s: every rank solved batch x steps LPs in at most total_ms."""
    return world * batch * steps / (total_ms / 1e3)


def percentile(vals, q):
    v = sorted(vals)
    return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_kw(opts):
    return dict(method=opts.get("solver", 0), inner_sweeps=opts.get("inner_sweeps", 1),
                omega=opts.get("omega", 1.0), max_krylov=opts.get("max_krylov", 0))


def _oracle_worker(job):
    """One LP of the workload solved by the oracle in a spawned process:
    returns (seconds, ipm_iters, krylov_iters, status)."""
    workload, seed_offset, opts, max_ipm = job
    sys.path.insert(0, ROOT)
    import oracle
    lp = make_lp(workload, seed_offset)
    kw = _oracle_kw(opts)
    if max_ipm:
        kw["max_ipm"] = max_ipm
    t0 = time.perf_counter()
    x, y, s, info = oracle.lp_solve_lp(lp, **kw)
    return time.perf_counter() - t0, info["ipm_iters"], info["krylov_iters_total"], info["status_name"]


def oracle_throughput(workload, opts, count, seed_base=0, pool=None, max_ipm=0):
    """LPs/s of the oracle on min(count, host cores) processes, one LP per
    process at a time; returns (LPs/s, cores, per-LP seconds, sample text)."""
    import oracle
    oracle.build()
    cores = max(1, min(count, os.cpu_count() or 1))
    jobs = [(workload, seed_base + i, opts, max_ipm) for i in range(count)]
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores)
    try:
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        if own:
            pool.close()
            pool.join()
    per = [r[0] for r in res]
    sample = (f"{count} LPs of the workload (seeds {seed_base}..{seed_base + count - 1}) solved by the oracle "
              f"(single-threaded C, FP64), one LP per process on {cores} host cores in parallel: "
              f"{wall:.1f} s wall, {statistics.mean(per):.2f} s per LP, status "
              f"{sorted(set(r[3] for r in res))}")
    if max_ipm:
        sample += f", capped at {max_ipm} interior-point iterations per LP"
    return count / wall, cores, per, sample


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def oracle_sweep_rate(lp, passes, warmup=1):
    """The oracle's NE-SOR pass (plain C, FP64, one thread) on the large LP's
    scaled matrix: (GB/s by the same byte formula as the GPU arm, seconds per
    pass, sample text).  The matrix is scaled once, outside the timing."""
    import numpy as np
    import oracle
    oracle.build()
    d2, g, _ = large_inputs(lp)
    nc, col, perm, cptr = oracle.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 0x5EED)
    ahat, rho = oracle.scale_rows(lp.m, lp.row_ptr, lp.col_idx, lp.val, d2)
    for _ in range(warmup):   # g is in the scaled space, as lpk_sweep takes it
        oracle.nesor(lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, g, 1, 1.0)
    t0 = time.perf_counter()
    for _ in range(passes):
        oracle.nesor(lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, g, 1, 1.0)
    sec = (time.perf_counter() - t0) / passes
    gbs = sweep_pass_bytes(lp.nnz, lp.m) / sec / 1e9
    sample = (f"{passes} NE-SOR passes (Algorithm 6, ell = 1) of the oracle (single-threaded C, FP64) over the "
              f"large LP's scaled matrix (m={lp.m}, n={lp.n}, nnz={lp.nnz}, {nc} colors), {sec:.3f} s per pass, "
              f"after {warmup} untimed pass(es)")
    return gbs, sec, sample


def large_inputs(lp):
    """Seeded inputs of the large-LP sweep benchmark: d2 = x/s spread over
    e^[-4, 4], g ~ N(0, 1), x ~ N(0, 1) for the product."""
    import numpy as np
    rng = np.random.default_rng(20160407 + 4)
    return np.exp(rng.uniform(-4.0, 4.0, lp.n)), rng.standard_normal(lp.m), rng.standard_normal(lp.n)


def run_reference_large(args, wl):
    from paper_1604_07491_gb300 import gen
    lp = gen.large_lp(1.0)
    vals, samples = [], []
    for i in range(args.warmup + args.steps):
        gbs, sec, sample = oracle_sweep_rate(lp, passes=1, warmup=0)
        if i >= args.warmup:
            vals.append(gbs)
            samples.append(sample)
    val = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC_SWEEP, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sweep_pass_bytes(lp.nnz, lp.m) / (val * 1e9),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": large_config(lp, None, "mixed"),
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": samples[-1]},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def large_config(lp, n_colors, precision):
    return {"workload": f"large: {WORKLOADS['large']['desc']}", "m": lp.m, "n": lp.n, "nnz": lp.nnz,
            "n_colors": n_colors, "precision": precision, "sweep": "NE-SOR (Algorithm 6), ell = 1, omega = 1",
            "inputs": "d2 = exp(U(-4, 4)), g ~ N(0,1), x ~ N(0,1) (seeded), resident in HBM",
            "l2": "256 MB buffer written between timed steps", "parallelism": "replicas"}


def run_reference(args, wl, opts):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "large":
        return run_reference_large(args, wl)
    B = args.batch if args.batch > 0 else wl["batch"]
    # serving and medium LPs take the oracle minutes each: one interior-point
    # iteration per LP bounds a step there (said in the sample text)
    max_ipm = 1 if args.workload in ("serving", "medium") else 0
    vals, samples = [], []
    cores = 1
    pool = mp.get_context("spawn").Pool(max(1, min(B, os.cpu_count() or 1)))
    try:
        for i in range(args.warmup + args.steps):
            v, cores, per, sample = oracle_throughput(args.workload, opts, B, seed_base=0, pool=pool,
                                                      max_ipm=max_ipm)
            if i >= args.warmup:
                vals.append(v)
                samples.append(sample)
    finally:
        pool.close()
        pool.join()
    val = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * B / val,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": reference_config(args, wl, opts, B),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": samples[-1]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reference_config(args, wl, opts, B):
    """The GPU arm's config keys for the same workload (the oracle runs FP64
    whatever the GPU arm's precision; the precision key names the GPU arm's)."""
    lp0 = make_lp(args.workload, 0)
    return {"workload": f"{args.workload}: {wl['desc']}", "m": lp0.m, "n": lp0.n, "nnz": lp0.nnz,
            "batch": B, "global_batch": B * args.gpus, "precision": args.precision,
            "solver": ["MRNE", "CGNE", "AB-GMRES"][opts["solver"]], "inner_sweeps": opts["inner_sweeps"],
            "omega": opts.get("omega", 1.0), "max_krylov": opts.get("max_krylov", 0)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def sum_stats(ctxs):
    tot = {}
    for c in ctxs:
        for k, v in c.stats().items():
            if k in ("last_cluster_size", "last_resident"):
                tot.setdefault(k, []).append(v)
            elif isinstance(v, list):
                tot[k] = [a + b for a, b in zip(tot.get(k, [0.0] * len(v)), v)]
            else:
                tot[k] = tot.get(k, 0) + v
    return tot


def roofline(stats, lp, precision, makespan_ms, traffic=None):
    hbm, src = peaks()
    launches = max(1, stats["krylov_launches"])
    bytes_total = algorithmic_bytes(stats, lp.m, lp.n, lp.nnz, precision)
    achieved = bytes_total / (stats["krylov_ms"] / 1e3) / 1e9 if stats["krylov_ms"] > 0 else 0.0
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "kernel": "k_krylov (persistent search-direction solve)",
            "peak_source": f"{src} hbm_gbs", "avg_launch_ms": stats["krylov_ms"] / launches,
            "launches": stats["krylov_launches"], "bytes_per_launch": bytes_total / launches,
            "barriers_per_launch": stats["barriers"] / launches,
            "us_per_barrier_phase": 1e3 * stats["krylov_ms"] / max(1, stats["barriers"]),
            "aggregate_gbs": bytes_total / (makespan_ms / 1e3) / 1e9 if makespan_ms > 0 else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lpk", choices=["lpk", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0, help="LPs per step solved side by side (0: workload's)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cluster", type=int, default=0, choices=[0, 4, 8, 16],
                    help="batch path: CTAs per LP's cluster (0: chosen from the problem)")
    ap.add_argument("--solver", default="", choices=[""] + sorted(SOLVERS),
                    help="Krylov solver (default: the workload's)")
    ap.add_argument("--compare-fp64", type=int, default=3,
                    help="FP64 LPs timed one at a time on the single-LP path (0: skip)")
    ap.add_argument("--e2e", type=int, default=1)
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--serving-count", type=int, default=48, help="serving: LPs of the stream replayed")
    ap.add_argument("--lanes", type=int, default=16, help="serving: server lanes")
    ap.add_argument("--serving-max-m", type=int, default=0,
                    help="serving: replay only the stream's LPs with m <= this (0: all)")
    ap.add_argument("--lp-steps", type=int, default=2,
                    help="large: timed steps of the assignment-LP solve throughput (0: skip)")
    ap.add_argument("--x8", type=int, default=1,
                    help="large: also time the sparse products on the matrix replicated 8x (0: skip)")
    ap.add_argument("--large-ipm", type=int, default=6,
                    help="large: interior-point iterations of the large LP run once (0: skip)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    opts = dict(wl["opts"])
    if args.solver:
        opts["solver"] = SOLVERS[args.solver]
    if args.impl == "reference":
        return run_reference(args, wl, opts)

    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = f"cuda:{local}"
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1604_07491_gb300 import lpk

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    if args.workload == "large":
        line = run_large(args, wl, opts, lpk, torch, dev, local, rank, world, barrier, dist)
    elif args.workload == "serving":
        line = run_serving(args, wl, opts, lpk, local, rank, world, barrier)
    elif args.workload == "large_x8":
        line = run_bandwidth(args, wl, lpk, torch, dev, local, rank, world, barrier)
    else:
        line = run_batch(args, wl, opts, lpk, torch, dev, local, rank, world, barrier, dist)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_large(args, wl, opts, lpk, torch, dev, local, rank, world, barrier, dist):
    """The default line: NE-sweep and SpMV bandwidth on the large LP, plus the
    assignment LP's solve throughput and the large LP's first interior-point
    iterations as secondary keys."""
    import numpy as np
    from paper_1604_07491_gb300 import gen
    lp = gen.large_lp(1.0)
    stream = torch.cuda.current_stream(dev)
    ctx = lpk.Context(local, stream.cuda_stream)
    P = lpk.Problem.from_lp(ctx, lp, device=dev)
    d2_h, g_h, x_h = large_inputs(lp)
    d2, g, x = (torch.from_numpy(v).to(dev) for v in (d2_h, g_h, x_h))
    prec = lpk.MIXED if args.precision == "mixed" else lpk.FP64
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    bsw, bsp = sweep_pass_bytes(lp.nnz, lp.m), spmv_bytes(lp.nnz, lp.m, lp.n)

    def step(d2v, gv, xv):
        P.sweep(d2v, gv, kind=lpk.NE_SOR, inner_sweeps=1, omega=1.0, precision=prec)
        return P.spmv(xv)

    for _ in range(args.warmup):
        step(d2, g, x)
    torch.cuda.synchronize(dev)
    ctx.reset_stats()
    step_ms, spmv_ms = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            P.sweep(d2, g, kind=lpk.NE_SOR, inner_sweeps=1, omega=1.0, precision=prec)
            e1.record(stream)
            P.spmv(x)
            e2.record(stream)
            barrier()
            step_ms.append(e0.elapsed_time(e2))
            spmv_ms.append(e1.elapsed_time(e2))
    st = ctx.stats()
    sweep_ms = st["krylov_ms"] / max(1, st["krylov_launches"])     # the sweep kernel alone (library events)
    sweep_ms = max_over_ranks(sweep_ms, dist, dev)
    spmv_kernel_ms = max_over_ranks(st["spmv_ms"] / max(1, st["spmv_launches"]), dist, dev)
    spmv_call_ms = max_over_ranks(statistics.median(spmv_ms), dist, dev)
    gbs = world * bsw / (sweep_ms / 1e3) / 1e9
    gbs_spmv = world * bsp / (spmv_kernel_ms / 1e3) / 1e9
    hbm, src = peaks()
    traffic, traffic_src = measured_traffic("sweep_large_mixed")
    launches = st["launches"]

    # end to end through the C ABI with host buffers (copies inside the timing)
    out_z, out_u, out_y = np.empty(lp.m), np.empty(lp.n), np.empty(lp.m)
    e2e_s = []
    for i in range(3):
        barrier()
        t0 = time.perf_counter()
        P.sweep(d2_h, g_h, kind=lpk.NE_SOR, inner_sweeps=1, omega=1.0, precision=prec)
        P.spmv(x_h)
        t1 = time.perf_counter()
        if i:
            e2e_s.append(t1 - t0)
    e2e = {"value": world * bsw / statistics.median(e2e_s) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": int(d2_h.nbytes + g_h.nbytes + x_h.nbytes),
           "d2h_bytes_per_step": int(out_z.nbytes + out_u.nbytes + out_y.nbytes),
           "what": "lpk_sweep + lpk_spmv on host arrays: host-to-device copies of d2, g, x and device-to-host "
                   "copies of z, u, y inside the timing; value = the sweep's algorithmic bytes / wall time"}

    # sparse products on the large matrix replicated 8x on the block diagonal
    # (170 MB of FP64 values and indices: larger than L2)
    spmv_x8 = None
    if args.x8:
        m8, n8, rp8, ci8, val8 = replicated_csr(lp, 8)
        P8 = lpk.Problem(ctx, m8, n8, torch.from_numpy(rp8).to(dev), torch.from_numpy(ci8).to(dev),
                         torch.from_numpy(val8).to(dev))
        gx = np.random.default_rng(7)
        x8 = torch.from_numpy(gx.standard_normal(n8)).to(dev)
        y8 = torch.from_numpy(gx.standard_normal(m8)).to(dev)
        res = {}
        for name, vec, tr in (("csr", x8, False), ("csc", y8, True)):
            for _ in range(2):
                P8.spmv(vec, transpose=tr)
            ctx.reset_stats()
            for _ in range(args.steps):
                flush.zero_()
                barrier()
                P8.spmv(vec, transpose=tr)
            st8 = ctx.stats()
            ms8 = max_over_ranks(st8["spmv_ms"] / st8["spmv_launches"], dist, dev)
            b8 = spmv_bytes(int(rp8[-1]), m8, n8) if not tr else spmv_bytes(int(rp8[-1]), n8, m8)
            res[name] = {"ms": ms8, "bytes": b8, "gbs": world * b8 / (ms8 / 1e3) / 1e9,
                         "frac": b8 / (ms8 / 1e3) / 1e9 / hbm}
        res.update({"m": m8, "n": n8, "nnz": int(rp8[-1]),
                    "what": "FP64 products A x (CSR) and A^T y (CSC) on the large matrix replicated 8x, kernel "
                            "time by CUDA events, L2 flushed before each"})
        spmv_x8 = res
        P8.free()

    # the large LP's first interior-point iterations (the method stalls later on this family)
    large_solve = None
    if args.large_ipm > 0:
        b, c = torch.from_numpy(lp.b).to(dev), torch.from_numpy(lp.c).to(dev)
        ctx.reset_stats()
        t0 = time.perf_counter()
        xs, ys, ss, info = P.lp_solve(b, c, precision=prec, max_ipm=args.large_ipm, **opts)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        st2 = ctx.stats()
        large_solve = {"max_ipm": args.large_ipm, "seconds": wall, "status": info["status_name"],
                       "ipm_iters": info["ipm_iters"], "krylov_iters": info["krylov_iters_total"],
                       "gamma": info["gamma"], "rel_gap": info["rel_gap"], "pinf": info["pinf"],
                       "dinf": info["dinf"], "ms_per_krylov_iter": st2["krylov_ms"] / max(1, st2["krylov_iters"]),
                       "solver": ["MRNE", "CGNE", "AB-GMRES"][opts["solver"]], "inner_sweeps": opts["inner_sweeps"]}
    P.free()
    ctx.close()

    # the assignment LP's solve throughput: batched mixed vs FP64 one LP at a time
    lp_solve = None
    if args.lp_steps > 0:
        sub = argparse.Namespace(**vars(args))
        sub.workload, sub.steps, sub.batch = "assignment", args.lp_steps, 0
        sub.cpu_baseline = args.cpu_baseline
        aw = WORKLOADS["assignment"]
        r = run_batch(sub, aw, dict(aw["opts"]), lpk, torch, dev, local, rank, world, barrier, dist)
        if r is not None:
            lp_solve = {k: r[k] for k in ("value", "unit", "ms_per_step", "p50_ms", "p99_ms", "solve", "fp64",
                                          "e2e", "cpu_baseline", "roofline", "config", "clocks", "gpu_launches")}
            lp_solve["steps"], lp_solve["warmup"] = sub.steps, sub.warmup

    if rank != 0:
        return None
    cpu = None
    if args.cpu_baseline and world == 1:
        v, sec, sample = oracle_sweep_rate(lp, passes=3)
        cpu = {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample, "seconds_per_pass": sec}
    return {
        "metric": METRIC_SWEEP, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 values / f64 accumulation" if prec == lpk.MIXED else "f64", "data": "synthetic",
        "config": large_config(lp, P.n_colors, args.precision),
        "value_is": "NE-sweep bandwidth: algorithmic bytes of one NE-SOR pass / sweep-kernel time (LPs/s of the "
                    "metric's first part: lp_solve)",
        "sweep": {"ms": sweep_ms, "bytes": bsw, "bytes_moved_fp64_u": sweep_pass_bytes_moved(lp.nnz, lp.m),
                  "gbs": gbs, "frac": gbs / hbm / world, "colors": P.n_colors,
                  "us_per_color_phase": 1e3 * sweep_ms / max(1, P.n_colors)},
        "spmv": {"ms": spmv_kernel_ms, "bytes": bsp, "gbs": gbs_spmv, "frac": gbs_spmv / hbm / world,
                 "call_ms": spmv_call_ms,
                 "what": "y = A x in FP64: the product kernel's CUDA-event time inside lpk_spmv (call_ms: the whole "
                         "call on the stream, with the gather/scatter between numberings and launch gaps)"},
        "spmv_x8": spmv_x8,
        "roofline": {"bound": "hbm", "achieved": gbs / world, "peak": hbm, "unit": "GB/s", "frac": gbs / world / hbm,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "kernel": "k_krylov<M_SWEEP, float, GridGrp> (one NE-SOR pass, grid path, rows cached in "
                               "shared memory)",
                     "peak_source": f"{src} hbm_gbs", "avg_launch_ms": sweep_ms, "bytes_per_launch": bsw,
                     "launches": st["krylov_launches"]},
        "lp_solve": lp_solve, "large_solve": large_solve,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
    }


def run_batch(args, wl, opts, lpk, torch, dev, local, rank, world, barrier, dist):
    import numpy as np
    B = args.batch if args.batch > 0 else wl["batch"]
    prec = lpk.MIXED if args.precision == "mixed" else lpk.FP64
    # replicas: rank r solves its own LPs of the same family (weak scaling)
    lps = [make_lp(args.workload, seed_offset=o) for o in replica_offsets(rank, B)]
    main_stream = torch.cuda.current_stream(dev)
    streams = [main_stream] if B == 1 else [torch.cuda.Stream(dev) for _ in range(B)]
    ctxs = [lpk.Context(local, st.cuda_stream) for st in streams]
    if B > 1 and args.cluster:
        for c in ctxs:
            c.set_exec(lpk.EXEC_BATCH, args.cluster)
    probs = [lpk.Problem.from_lp(ctxs[i], lps[i], device=dev) for i in range(B)]
    bs = [torch.from_numpy(lp.b).to(dev) for lp in lps]
    cs = [torch.from_numpy(lp.c).to(dev) for lp in lps]
    outs = [(torch.empty(lp.n, dtype=torch.float64, device=dev), torch.empty(lp.m, dtype=torch.float64, device=dev),
             torch.empty(lp.n, dtype=torch.float64, device=dev)) for lp in lps]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    torch.cuda.synchronize(dev)

    def step(p):
        if B == 1:
            return [probs[0].lp_solve(bs[0], cs[0], out=outs[0], precision=p, **opts)]
        return lpk.solve_batch(probs, bs, cs, outs=outs, precision=p, **opts)

    for _ in range(args.warmup):
        step(prec)
    for c in ctxs:
        c.reset_stats()
    step_ms, lat_ms, infos = [], [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main_stream)
            res = step(prec)
            e1.record(main_stream)
            barrier()
            step_ms.append(e0.elapsed_time(e1))
            for r in res:
                lat_ms.append(r[3]["solve_ms"])
                infos.append(r[3])
    stats = sum_stats(ctxs)
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    lps_per_s = weak_throughput(world, B, args.steps, total_ms)
    worst = max(infos, key=lambda d: (d["status"] != 0, d["rel_gap"]))

    # plain FP64, one LP at a time, on the autotuned single-LP path
    fp64 = None
    if args.compare_fp64 > 0:
        ctx1 = lpk.Context(local, main_stream.cuda_stream)
        k = min(args.compare_fp64, B)
        p1 = [lpk.Problem.from_lp(ctx1, lps[i], device=dev) for i in range(k)]
        p1[0].lp_solve(bs[0], cs[0], out=outs[0], precision=lpk.FP64, **opts)  # warm-up (and autotune)
        ms64, inf64 = [], []
        for i in range(k):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main_stream)
            r = p1[i].lp_solve(bs[i], cs[i], out=outs[i], precision=lpk.FP64, **opts)[3]
            e1.record(main_stream)
            barrier()
            ms64.append(e0.elapsed_time(e1))
            inf64.append(r)
        fp64 = {"value": world * k / (sum(ms64) / 1e3), "unit": UNIT, "mode": "FP64, one LP at a time",
                "ms_per_lp": statistics.mean(ms64), "lps": k,
                "status": sorted({d["status_name"] for d in inf64}),
                "max_rel_gap": max(d["rel_gap"] for d in inf64), "max_pinf": max(d["pinf"] for d in inf64),
                "max_dinf": max(d["dinf"] for d in inf64),
                "obj_rel_diff_vs_batch": max(abs(inf64[i]["obj_primal"] - infos[i]["obj_primal"])
                                             / max(1.0, abs(inf64[i]["obj_primal"])) for i in range(k))}
        for p in p1:
            p.free()
        ctx1.close()

    # end to end through the C ABI with host buffers: prepare from host CSR
    # (H2D of A inside), b, c from host, x, y, s back to host, all timed
    e2e = None
    if args.e2e:
        h_out = [(np.empty(lp.n), np.empty(lp.m), np.empty(lp.n)) for lp in lps]
        barrier()
        t0 = time.perf_counter()
        ph = [lpk.Problem.from_lp(ctxs[i], lps[i]) for i in range(B)]
        if B == 1:
            r = [ph[0].lp_solve(lps[0].b, lps[0].c, out=h_out[0], precision=prec, **opts)]
        else:
            r = lpk.solve_batch(ph, [lp.b for lp in lps], [lp.c for lp in lps], outs=h_out, precision=prec,
                                **opts)
        for p in ph:
            p.free()
        t1 = time.perf_counter()
        h2d = sum(lp.row_ptr.nbytes + lp.col_idx.nbytes + lp.val.nbytes + lp.b.nbytes + lp.c.nbytes for lp in lps)
        d2h = sum(a.nbytes for t in h_out for a in t)
        e2e = {"value": world * B / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "status": sorted({x[3]["status_name"] for x in r})}

    if rank != 0:
        return None
    cpu = None
    if args.cpu_baseline and world == 1:
        v, cores, per, sample = oracle_throughput(args.workload, opts, min(B, os.cpu_count() or 1))
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "seconds_per_lp": statistics.mean(per)}
    lp0 = lps[0]
    return {
        "metric": METRIC, "value": lps_per_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 values / f64 accumulation" if prec == lpk.MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "m": lp0.m, "n": lp0.n, "nnz": lp0.nnz,
                   "n_colors": probs[0].n_colors, "batch": B, "global_batch": B * world,
                   "precision": args.precision, "solver": ["MRNE", "CGNE", "AB-GMRES"][opts["solver"]],
                   "inner_sweeps": opts["inner_sweeps"], "omega": opts.get("omega", 1.0),
                   "max_krylov": opts.get("max_krylov", 0),
                   "exec": "batch path: one context, stream and thread-block cluster per LP" if B > 1
                   else "single-LP path (autotuned)",
                   "cluster_sizes": sorted(set(stats.get("last_cluster_size", []))),
                   "parallelism": f"replicas x{world}", "l2": "256 MB buffer written between timed steps",
                   "inputs": "resident in HBM (prepare outside the timed region)"},
        "p50_ms": percentile(lat_ms, 0.50), "p99_ms": percentile(lat_ms, 0.99),
        "latency": "per-LP solve time (CUDA events on the LP's stream) within its batch",
        "solve": {"status": sorted({d["status_name"] for d in infos}), "ipm_iters": worst["ipm_iters"],
                  "krylov_iters_mean": statistics.mean(d["krylov_iters_total"] for d in infos),
                  "max_rel_gap": max(d["rel_gap"] for d in infos), "max_pinf": max(d["pinf"] for d in infos),
                  "max_dinf": max(d["dinf"] for d in infos)},
        "fp64": fp64,
        "roofline": roofline(stats, lp0, args.precision, total_ms,
                             measured_traffic(f"krylov_{args.workload}_{args.precision}")[0]),
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": stats["launches"], "clocks": clk.summary(),
    }


def replicated_csr(lp, copies):
    """lp's matrix repeated `copies` times on the block diagonal (CSR)."""
    import numpy as np
    nnz = int(lp.row_ptr[-1])
    rp = np.concatenate([lp.row_ptr[:-1] + k * nnz for k in range(copies)] + [[copies * nnz]]).astype(np.int64)
    ci = np.concatenate([lp.col_idx + k * lp.n for k in range(copies)]).astype(np.int32)
    val = np.tile(lp.val, copies)
    return copies * lp.m, copies * lp.n, rp, ci, val


def run_bandwidth(args, wl, lpk, torch, dev, local, rank, world, barrier):
    """Bandwidth of the sparse products on a matrix larger than L2: y = A x
    and w = A^T y in FP64 through lpk_spmv (gather to the internal numbering,
    CSR or CSC product, scatter back).  The sweep is not measured here: on the
    grid path each warp keeps a slot per row it sweeps in shared memory, which
    caps a sweep at about 1,400 slots per warp (rows / 1,216 warps + colors),
    below this matrix's 1.2 M rows with 400+ colors."""
    from paper_1604_07491_gb300 import gen
    base = gen.large_lp(1.0)
    m, n, rp, ci, val = replicated_csr(base, 8)
    nnz = int(rp[-1])
    ctx = lpk.Context(local, torch.cuda.current_stream(dev).cuda_stream)
    P = lpk.Problem(ctx, m, n, torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                    torch.from_numpy(val).to(dev))
    gx = torch.Generator(device="cpu").manual_seed(7)
    x = torch.rand(n, generator=gx, dtype=torch.float64).to(dev)
    yv = torch.rand(m, generator=gx, dtype=torch.float64).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            fn()
        ms = []
        for _ in range(reps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            barrier()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    with ClockSampler(local) as clk:
        ms_a = timed(lambda: P.spmv(x), args.steps)
        ms_t = timed(lambda: P.spmv(yv, transpose=True), args.steps)
    hbm, src = peaks()
    # algorithmic bytes: value + index + gathered vector entry per nonzero
    # (8 + 4 + 8), pointer + result per row/column (4 + 8), and the gather and
    # scatter between input and internal numbering (16 B per entry of x and y)
    b_a = nnz * 20 + m * 12 + 16 * (n + m)
    b_t = nnz * 20 + n * 12 + 16 * (n + m)
    if rank != 0:
        return None
    ga, gt = b_a / (ms_a / 1e3) / 1e9, b_t / (ms_t / 1e3) / 1e9
    return {
        "metric": "SpMV HBM GB/s (A x and A^T y, FP64)", "value": ga, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_a, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"large_x8: {wl['desc']}", "m": m, "n": n, "nnz": nnz,
                   "n_colors": P.n_colors, "l2": "256 MB buffer written between timed calls",
                   "inputs": "resident in HBM"},
        "spmv_csr": {"ms": ms_a, "bytes": b_a, "gbs": ga, "frac": ga / hbm},
        "spmv_csc": {"ms": ms_t, "bytes": b_t, "gbs": gt, "frac": gt / hbm},
        "roofline": {"bound": "hbm", "achieved": ga, "peak": hbm, "unit": "GB/s", "frac": ga / hbm,
                     "traffic": None, "kernel": "lpk_spmv (k_gather, k_seg_spmv + k_seg_fix, k_scatter)",
                     "peak_source": f"{src} hbm_gbs"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk.summary(),
    }


def run_serving(args, wl, opts, lpk, local, rank, world, barrier):
    """Replay the first N LPs of the Poisson stream through the server: each is
    submitted at its arrival time; latency = result ready - arrival."""
    from paper_1604_07491_gb300 import gen
    N = args.serving_count
    # the stream's LPs in arrival order, optionally only those with m <= max_m
    # (each keeps its own arrival time; the stream is thinned, not re-timed)
    arrivals_all = gen.serving_arrivals(200000)
    lps, arrivals = [], []
    i = rank * 100000
    while len(lps) < N:
        lp = make_lp("serving", seed_offset=i)
        if args.serving_max_m <= 0 or lp.m <= args.serving_max_m:
            lps.append(lp)
            arrivals.append(arrivals_all[i - rank * 100000])
        i += 1
    prec = lpk.MIXED if args.precision == "mixed" else lpk.FP64
    srv = lpk.Server(local, lanes=args.lanes)
    # warm-up: a few small LPs (kernel loading, pool growth)
    for t in [srv.submit_lp(make_lp("tiny", i), precision=prec, **WORKLOADS["tiny"]["opts"]) for i in range(3)]:
        srv.wait(t)
    barrier()
    tickets = []
    with ClockSampler(local) as clk:
        t0 = srv.now()
        for i, lp in enumerate(lps):
            delay = t0 + arrivals[i] - srv.now()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit_lp(lp, precision=prec, **opts))
        res = [srv.wait(t) for t in tickets]
        barrier()
    st = srv.stats()
    srv.close()
    lat = [1e3 * (r[3]["t_end"] - r[3]["t_submit"]) for r in res]
    span = max(r[3]["t_end"] for r in res) - min(r[3]["t_submit"] for r in res)
    infos = [r[3]["info"] for r in res]
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": world * N / span, "unit": UNIT, "n_gpus": world, "steps": 1,
        "warmup": 3, "ms_per_step": 1e3 * span, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 values / f64 accumulation" if prec == lpk.MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": f"serving: {wl['desc']}", "lps": N, "lanes": args.lanes,
                   "stream": ("the first LPs of the stream" if args.serving_max_m <= 0 else
                              f"the first LPs of the stream with m <= {args.serving_max_m} (thinned stream)"),
                   "m_range": [min(lp.m for lp in lps), max(lp.m for lp in lps)], "precision": args.precision,
                   "solver": ["MRNE", "CGNE", "AB-GMRES"][opts["solver"]], "inner_sweeps": opts["inner_sweeps"],
                   "l2": "inputs of every LP differ (no reuse)", "inputs": "host CSR submitted at arrival"},
        "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99),
        "latency": "arrival to result (queueing + prepare + solve + copy-out)",
        "solve": {"status": sorted({d["status_name"] for d in infos}),
                  "max_rel_gap": max(d["rel_gap"] for d in infos)},
        "server": st, "roofline": None, "cpu_baseline": None,
        "e2e": {"value": world * N / span, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(lp.row_ptr.nbytes + lp.col_idx.nbytes + lp.val.nbytes
                                              + lp.b.nbytes + lp.c.nbytes for lp in lps)),
                "d2h_bytes_per_step": int(sum(8 * (2 * lp.n + lp.m) for lp in lps))},
        "gpu_launches": None, "clocks": clk.summary(),
    }


if __name__ == "__main__":
    main()
