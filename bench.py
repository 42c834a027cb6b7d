"""Benchmark: LP solves per second on a seeded synthetic workload.

A step is one complete interior-point solve (Algorithm 1 with the Krylov
search-direction solves) of one LP whose data is already resident in HBM.
Prints one JSON line (rank 0).  See the design doc for the workload recipes, the
algorithmic byte counts behind the roofline figure and the timing rules.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload medium]
                  [--precision mixed|fp64] [--impl lpk|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LPs solved/s & p99 latency at gap≤1e-8 (mixed vs FP64); NE-sweep HBM GB/s"
UNIT = "LPs/s"

# workload -> (generator, options).  max_krylov 40000 is the relaxed Krylov cap
# the paper uses for difficult problems (Sec. 4.2).
WORKLOADS = {
    "medium": dict(desc="rank-deficient sparse LP m=20000 n=60000, 8 nnz/col N(0,1), 1% dependent rows",
                   opts=dict(solver=0, inner_sweeps=5, omega=1.0, max_krylov=40000)),
    "assignment": dict(desc="degenerate assignment LP k=14 (n=38416, m=588), costs U{0..100}",
                       opts=dict(solver=0, inner_sweeps=3, omega=1.0)),
    "tiny": dict(desc="tiny sparse LP m=50 n=120 ~5% N(0,1)", opts=dict(solver=0, inner_sweeps=1)),
    "medium_0.1": dict(desc="medium family at scale 0.1 (m=2000 n=6000)",
                       opts=dict(solver=0, inner_sweeps=5, omega=1.0, max_krylov=6000)),
}


SOLVERS = {"mrne": 0, "cgne": 1, "abgmres": 2}


def make_lp(workload, seed_offset=0):
    from paper_1604_07491_gb300 import gen
    if workload == "medium":
        return gen.medium_lp(1.0, seed=gen.SEED_BASE + 2 + 1000 * seed_offset)
    if workload == "medium_0.1":
        return gen.medium_lp(0.1, seed=gen.SEED_BASE + 2 + 1000 * seed_offset)
    if workload == "assignment":
        return gen.assignment_lp(seed=gen.SEED_BASE + 3 + 1000 * seed_offset)
    if workload == "tiny":
        return gen.tiny_lp(seed=gen.SEED_BASE + 1 + 1000 * seed_offset)
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


def _oracle_kw(opts):
    return dict(method=opts.get("solver", 0), inner_sweeps=opts.get("inner_sweeps", 1),
                omega=opts.get("omega", 1.0), max_krylov=opts.get("max_krylov", 0))


def oracle_lp_seconds(lp, opts, krylov_iters_full, max_seconds=30.0):
    """Seconds the oracle (single-threaded C) needs for one LP of the workload.
    A first sample (starting point + first interior-point iteration, max_ipm=1)
    gives its time per Krylov iteration; if the whole solve is estimated to
    fit in max_seconds it is run and timed in full, else the estimate (time per
    Krylov iteration x the Krylov iterations of the full solve) is returned."""
    import oracle
    oracle.build()
    kw = _oracle_kw(opts)
    t0 = time.perf_counter()
    x, y, s, info = oracle.lp_solve_lp(lp, max_ipm=1, **kw)
    dt = time.perf_counter() - t0
    its = max(1, int(info["krylov_iters_total"]))
    est = dt / its * max(krylov_iters_full, its)
    if est <= max_seconds:
        t0 = time.perf_counter()
        x, y, s, info = oracle.lp_solve_lp(lp, **kw)
        full = time.perf_counter() - t0
        return full, (f"one full oracle lp_solve of the same LP on 1 host thread: {full:.2f} s, "
                      f"{info['ipm_iters']} IPM / {info['krylov_iters_total']} Krylov iterations, "
                      f"status {info['status_name']}")
    return est, (f"oracle lp_solve with max_ipm=1 (starting point + 1 IPM iteration, {its} Krylov "
                 f"iterations in {dt:.2f} s on 1 host thread), scaled by the {krylov_iters_full} "
                 f"Krylov iterations of the full solve: {est:.1f} s per LP")


def cpu_baseline(lp, opts, krylov_iters_full):
    sec, sample = oracle_lp_seconds(lp, opts, krylov_iters_full)
    return {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "seconds_per_lp": sec}


def run_reference(args):
    """--impl reference: the oracle on the host cores; each step is one LP of
    the workload (a full oracle solve when it takes under 30 s, else the
    bounded sample of oracle_lp_seconds)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    lp = make_lp(args.workload)
    opts = dict(wl["opts"])
    if args.solver:
        opts["solver"] = SOLVERS[args.solver]
    secs, samples = [], []
    for i in range(args.warmup + args.steps):
        sec, sample = oracle_lp_seconds(lp, opts, args.ref_full_krylov)
        if i >= args.warmup:
            secs.append(sec)
            samples.append(sample)
    sec = statistics.mean(secs)
    val = 1.0 / sec
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}", **{k: v for k, v in opts.items()}},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": samples[-1]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lpk", choices=["lpk", "reference"])
    # default: the assignment LP; a medium LP solve takes minutes with the
    # current kernels (several hundred thousand Krylov iterations), too long
    # for a default run with three warm-up solves
    ap.add_argument("--workload", default="assignment", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--solver", default="", choices=["", "mrne", "cgne", "abgmres"],
                    help="Krylov solver (default: the workload's)")
    ap.add_argument("--compare-fp64", type=int, default=1, help="also time K FP64 solves")
    ap.add_argument("--e2e", type=int, default=1)
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--ref-full-krylov", type=int, default=0,
                    help="reference arm: Krylov iterations of a full solve (0: measured by one GPU solve)")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.ref_full_krylov <= 0:
            args.ref_full_krylov = {"medium": 700000, "medium_0.1": 69305, "assignment": 9333,
                                    "tiny": 515}[args.workload]
        return run_reference(args)

    import numpy as np
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

    wl = WORKLOADS[args.workload]
    opts = dict(wl["opts"])
    if args.solver:
        opts["solver"] = SOLVERS[args.solver]
    prec = lpk.MIXED if args.precision == "mixed" else lpk.FP64
    # replicas: each rank solves its own LP of the same family (weak scaling)
    lp = make_lp(args.workload, seed_offset=rank)
    stream = torch.cuda.current_stream(dev)
    ctx = lpk.Context(local, stream.cuda_stream)
    P = lpk.Problem.from_lp(ctx, lp, device=dev)
    b = torch.from_numpy(lp.b).to(dev)
    c = torch.from_numpy(lp.c).to(dev)
    out = (torch.empty(lp.n, dtype=torch.float64, device=dev), torch.empty(lp.m, dtype=torch.float64, device=dev),
           torch.empty(lp.n, dtype=torch.float64, device=dev))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def solve(p):
        return P.lp_solve(b, c, out=out, precision=p, **opts)

    infos = []
    for _ in range(args.warmup):
        infos.append(solve(prec)[3])
    ctx.reset_stats()
    step_ms = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, y, s, info = solve(prec)
            e1.record(stream)
            barrier()
            step_ms.append(e0.elapsed_time(e1))
            infos.append(info)
    stats = ctx.stats()
    total_ms = sum(step_ms)
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    total_ms = float(tmax.item())
    lps = world * args.steps / (total_ms / 1e3)
    last = infos[-1]

    # FP64 comparison on the same LP (same steps)
    fp64 = None
    if args.compare_fp64 and prec == lpk.MIXED:
        solve(lpk.FP64)  # warm the FP64 kernels
        ms64 = []
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r64 = solve(lpk.FP64)[3]
            e1.record(stream)
            barrier()
            ms64.append(e0.elapsed_time(e1))
        fp64 = {"value": world * args.steps / (sum(ms64) / 1e3), "unit": UNIT,
                "ms_per_step": statistics.mean(ms64), "status": r64["status_name"],
                "ipm_iters": r64["ipm_iters"], "krylov_iters": r64["krylov_iters_total"],
                "obj": r64["obj_primal"]}

    # end to end through the C ABI with host buffers: prepare from host CSR,
    # H2D of A, b, c and D2H of x, y, s inside the timed region
    e2e = None
    if args.e2e:
        h_out = (np.empty(lp.n), np.empty(lp.m), np.empty(lp.n))
        barrier()
        t0 = time.perf_counter()
        Ph = lpk.Problem.from_lp(ctx, lp)
        r = Ph.lp_solve(lp.b, lp.c, out=h_out, precision=prec, **opts)
        Ph.free()
        t1 = time.perf_counter()
        h2d = lp.row_ptr.nbytes + lp.col_idx.nbytes + lp.val.nbytes + lp.b.nbytes + lp.c.nbytes
        d2h = sum(a.nbytes for a in h_out)
        e2e = {"value": world / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "status": r[3]["status_name"]}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    hbm, src = peaks()
    kernel_ms = stats["krylov_ms"] / max(1, stats["krylov_launches"])
    bytes_total = algorithmic_bytes(stats, lp.m, lp.n, lp.nnz, args.precision)
    achieved = bytes_total / (stats["krylov_ms"] / 1e3) / 1e9 if stats["krylov_ms"] > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": "k_krylov (persistent search-direction solve)",
                "peak_source": f"{src} hbm_gbs", "avg_launch_ms": kernel_ms,
                "launches": stats["krylov_launches"], "bytes_per_launch": bytes_total / max(1, stats["krylov_launches"]),
                "barriers_per_launch": stats["barriers"] / max(1, stats["krylov_launches"]),
                "us_per_barrier_phase": 1e3 * stats["krylov_ms"] / max(1, stats["barriers"])}
    cpu = None
    if args.cpu_baseline and world == 1:
        cpu = cpu_baseline(lp, opts, int(last["krylov_iters_total"]))
    lat = sorted(step_ms)
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    line = {
        "metric": METRIC, "value": lps, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 values / f64 accumulation" if prec == lpk.MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "m": lp.m, "n": lp.n, "nnz": lp.nnz,
                   "n_colors": P.n_colors, "precision": args.precision,
                   "solver": ["MRNE", "CGNE", "AB-GMRES"][opts["solver"]], "inner_sweeps": opts["inner_sweeps"],
                   "omega": opts.get("omega", 1.0), "max_krylov": opts.get("max_krylov", 0),
                   "parallelism": f"replicas x{world}", "l2": "256 MB buffer written between timed steps",
                   "inputs": "resident in HBM (prepare outside the timed region)"},
        "p50_ms": statistics.median(step_ms), "p99_ms": p99,
        "solve": {"status": last["status_name"], "ipm_iters": last["ipm_iters"],
                  "krylov_iters": last["krylov_iters_total"], "obj": last["obj_primal"],
                  "gamma": last["gamma"], "rel_gap": last["rel_gap"], "pinf": last["pinf"], "dinf": last["dinf"]},
        "fp64": fp64, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": stats["launches"], "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
