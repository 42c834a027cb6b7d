"""Writes large_ipm2.json: the oracle's interior-point iterates on the large
power-law LP (m = 150,000, n = 434,580, mean column degree 6, maximum 400;
gen.large_lp) after one and after two iterations of Algorithm 1, with
AB-GMRES (Algorithm 4) and one NE-SOR sweep (Algorithm 6) per inner
application, FP64.  The full vectors are too large for a text fixture, so a
fixed, seeded sample of entries of x, y and s is stored, with the norms of the
full vectors, the objective values and the oracle's per-iteration trace.

Only the oracle is called.  Run from the repository root:
    python tests/golden/make_large_golden.py
(about two minutes on one core)."""
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


def main():
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
            "seconds": time.time() - t0,
            "info": {kk: (vv if not isinstance(vv, float) else float(repr(vv))) for kk, vv in info.items()},
            "trace": [dict(zip(oracle.TRACE_FIELDS, map(float, row))) for row in tr],
            "norms": {kk: float(np.linalg.norm(v)) for kk, v in vec.items()},
            "samples": {kk: [float(repr(float(vec[kk][i]))) for i in idx[kk]] for kk in vec},
        }
        print(f"max_ipm={k}: {time.time() - t0:.1f} s, {info['krylov_iters_total']} Krylov iterations, "
              f"Gamma {info['gamma']:.3e}", flush=True)
    with open(os.path.join(HERE, "large_ipm2.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
