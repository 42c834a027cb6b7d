"""The autotuner and its cache.  On the first Krylov solve of a problem in
LPK_EXEC_AUTO the library times a few iterations of every execution path
(the grid; clusters of 16, 8, 4 CTAs with u in shared or global memory) and
keeps the fastest; the choice is cached by problem shape, for the process and
in the file LPK_TUNE_CACHE names.  Checked: a second problem of the same shape
takes the cached path without probes and solves to the bitwise-same result; a
new process reads the choice back from the file; and the tuned path is not
slower than the batch lanes' fixed choice on the assignment LP."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1604_07491_gb300 import gen  # noqa: E402


@pytest.fixture(scope="module")
def lpk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07491_gb300 import build, lpk as L
    build.build()
    return L


def _solve(lpk, ctx, lp, **kw):
    P = lpk.Problem.from_lp(ctx, lp, device="cuda")
    b, c = torch.from_numpy(lp.b).cuda(), torch.from_numpy(lp.c).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, y, s, info = P.lp_solve(b, c, **kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    P.free()
    return x, info, dt


def test_tuning_cache_and_tuned_path(lpk, tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("LPK_TUNE_CACHE", str(path))
    # a shape no other test uses: the medium family at an odd scale
    lp = gen.medium_lp(0.0173)
    kw = dict(solver=lpk.ABGMRES, inner_sweeps=2, precision=lpk.MIXED, max_krylov=10 * lp.m)
    c1 = lpk.Context(0)
    x1, info1, _ = _solve(lpk, c1, lp, **kw)
    s1 = c1.stats()
    assert info1["status_name"] == "OK"
    assert s1["tune_probes"] >= 2 and s1["tune_cache_hits"] == 0
    lines = [l for l in path.read_text().splitlines() if l.startswith("lpk-tune")]
    assert len(lines) == 1 and lines[0].split()[1:4] == [str(lp.m), str(lp.n), str(lp.nnz)]
    c2 = lpk.Context(0)
    x2, info2, _ = _solve(lpk, c2, lp, **kw)
    s2 = c2.stats()
    assert s2["tune_probes"] == 0 and s2["tune_cache_hits"] == 1
    assert (s2["last_cluster_size"], s2["last_u_global"]) == (s1["last_cluster_size"], s1["last_u_global"])
    assert torch.equal(x1, x2) and info1["krylov_iters_total"] == info2["krylov_iters_total"]
    c1.close()
    c2.close()
    # a new process reads the choice back from the file
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys, torch; sys.path.insert(0, %r); from paper_1604_07491_gb300 import gen, lpk; "
            "lp = gen.medium_lp(0.0173); c = lpk.Context(0); P = lpk.Problem.from_lp(c, lp, device='cuda'); "
            "P.lp_solve(torch.from_numpy(lp.b).cuda(), torch.from_numpy(lp.c).cuda(), solver=2, inner_sweeps=2, "
            "precision=1, max_krylov=10 * lp.m); st = c.stats(); "
            "print(st['tune_probes'], st['tune_cache_hits'], st['last_cluster_size'], st['last_u_global'])" % root)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, LPK_TUNE_CACHE=str(path)))
    assert out.returncode == 0, out.stderr
    probes, hits, cs, ug = map(int, out.stdout.split()[-4:])
    assert probes == 0 and hits == 1 and (cs, ug) == (s1["last_cluster_size"], s1["last_u_global"])


def test_tuned_path_not_slower_than_batch_lanes(lpk):
    """The assignment LP alone: the autotuned path against the cluster size
    the batch lanes fix from the problem alone (best of two solves each)."""
    lp = gen.assignment_lp()
    kw = dict(solver=lpk.ABGMRES, inner_sweeps=3, precision=lpk.MIXED)
    ct = lpk.Context(0)
    cb = lpk.Context(0)
    cb.set_exec(lpk.EXEC_BATCH)
    _solve(lpk, ct, lp, **kw)          # tunes
    t_tuned = min(_solve(lpk, ct, lp, **kw)[2] for _ in range(2))
    t_batch = min(_solve(lpk, cb, lp, **kw)[2] for _ in range(2))
    assert t_tuned <= 1.1 * t_batch, (t_tuned, t_batch)
    ct.close()
    cb.close()
