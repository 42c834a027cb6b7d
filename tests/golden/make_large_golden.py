"""Writes the large power-law LP's oracle fixtures (gen.large_lp: mean column
degree 6, maximum 400), AB-GMRES (Algorithm 4) with one NE-SOR sweep
(Algorithm 6) per inner application, FP64:

  large_ipm2.json   full size (m = 150,000, n = 434,580), Krylov cap 40,000
                    (the paper's relaxed cap, Sec. 4.2): the iterates after
                    one and after two interior-point iterations of Algorithm 1
                    (the full vectors are too large for a text fixture, so a
                    fixed, seeded sample of entries of x, y and s is stored,
                    with the norms of the full vectors, the objective values
                    and the oracle's per-iteration trace);
  large_s003_solve.json  the same family at scale 0.03 (m = 4,500,
                    n = 13,037), Krylov cap m, solved to gap <= 1e-8:
                    objective, certificates, trace and a sample of x, y, s.

Only the oracle is called.  Run from the repository root:
    python tests/golden/make_large_golden.py [ipm2|solve003|all]
(ipm2: about two minutes on one core; solve003: about 25 minutes)."""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1604_07491_gb300 import gen  # noqa: E402

OPTS = dict(method=oracle.ABGMRES, inner_sweeps=1, omega=1.0, max_krylov=40000)
SAMPLES = dict(x=1500, s=1500, y=1000)


def sample_indices(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def sample(vec, idx):
    return {kk: [float(repr(float(vec[kk][i]))) for i in idx[kk]] for kk in vec}


def info_json(info):
    return {kk: (vv if not isinstance(vv, float) else float(repr(vv))) for kk, vv in info.items()}


def write_ipm2():
    lp = gen.large_lp(1.0)
    idx = {"x": sample_indices(lp.n, SAMPLES["x"], 1), "s": sample_indices(lp.n, SAMPLES["s"], 2),
           "y": sample_indices(lp.m, SAMPLES["y"], 3)}
    out = {"lp": lp.name, "m": lp.m, "n": lp.n, "nnz": lp.nnz, "options": OPTS,
           "indices": {k: v.tolist() for k, v in idx.items()}, "iterates": {}}
    for k in (1, 2):
        t0 = time.time()
        x, y, s, info, tr = oracle.lp_solve_lp(lp, trace=True, max_ipm=k, **OPTS)
        vec = {"x": x, "y": y, "s": s}
        out["iterates"][str(k)] = {
            "seconds": time.time() - t0, "info": info_json(info),
            "trace": [dict(zip(oracle.TRACE_FIELDS, map(float, row))) for row in tr],
            "norms": {kk: float(np.linalg.norm(v)) for kk, v in vec.items()}, "samples": sample(vec, idx)}
        print(f"max_ipm={k}: {time.time() - t0:.1f} s, {info['krylov_iters_total']} Krylov iterations, "
              f"Gamma {info['gamma']:.3e}", flush=True)
    with open(os.path.join(HERE, "large_ipm2.json"), "w") as f:
        json.dump(out, f, indent=0)


SOLVE_OPTS = dict(method=oracle.ABGMRES, inner_sweeps=1, omega=1.0, max_krylov=0)


def write_solve003():
    lp = gen.large_lp(0.03)
    idx = {"x": sample_indices(lp.n, 1000, 4), "s": sample_indices(lp.n, 1000, 5),
           "y": sample_indices(lp.m, 1000, 6)}
    t0 = time.time()
    x, y, s, info, tr = oracle.lp_solve_lp(lp, trace=True, **SOLVE_OPTS)
    vec = {"x": x, "y": y, "s": s}
    out = {"lp": lp.name, "scale": 0.03, "m": lp.m, "n": lp.n, "nnz": lp.nnz, "options": SOLVE_OPTS,
           "seconds": time.time() - t0, "info": info_json(info),
           "trace": [dict(zip(oracle.TRACE_FIELDS, map(float, row))) for row in tr],
           "norms": {kk: float(np.linalg.norm(v)) for kk, v in vec.items()},
           "indices": {k: v.tolist() for k, v in idx.items()}, "samples": sample(vec, idx)}
    print(f"scale 0.03: {time.time() - t0:.1f} s, {info['status_name']}, {info['ipm_iters']} interior-point and "
          f"{info['krylov_iters_total']} Krylov iterations, objective {info['obj_primal']!r}", flush=True)
    with open(os.path.join(HERE, "large_s003_solve.json"), "w") as f:
        json.dump(out, f, indent=0)


def main():
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("ipm2", "all"):
        write_ipm2()
    if what in ("solve003", "all"):
        write_solve003()


if __name__ == "__main__":
    main()
