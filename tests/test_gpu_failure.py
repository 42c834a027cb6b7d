"""Failure detection on the GPU without a fault: every wait of the grid
path's software barrier is bounded.  With a short bound and the test hook
that makes CTA 0 withhold its arrival at one barrier, every CTA's wait runs
out, the call returns LPK_TIMEOUT within the bound, and the same context then
solves the same problem to the bitwise-same result as before."""
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


@pytest.mark.parametrize("solver", [0, 2])
def test_grid_barrier_wait_times_out_and_context_recovers(lpk, solver):
    lp = gen.medium_lp(0.05)
    ctx = lpk.Context(0)
    ctx.set_exec(lpk.EXEC_GRID)
    P = lpk.Problem.from_lp(ctx, lp, device="cuda")
    rng = np.random.default_rng(9)
    d2 = torch.from_numpy(np.exp(rng.uniform(-3, 3, lp.n))).cuda()
    f = torch.from_numpy(lp.scipy() @ (d2.cpu().numpy() * rng.standard_normal(lp.n))).cuda()
    dy0, dw0, info0 = P.ne_solve(d2, f, solver=solver, tol=1e-9, max_iter=20 * lp.m)
    assert info0["converged"]
    ctx.set_wait_limit(0.02, test_stall_barrier=7)
    t0 = time.time()
    with pytest.raises(lpk.LpkError) as e:
        P.ne_solve(d2, f, solver=solver, tol=1e-9, max_iter=20 * lp.m)
    elapsed = time.time() - t0
    assert e.value.status == lpk.TIMEOUT and "timed out" in str(e.value)
    assert elapsed < 2.0, elapsed
    ctx.set_wait_limit(5.0, 0)
    dy1, dw1, info1 = P.ne_solve(d2, f, solver=solver, tol=1e-9, max_iter=20 * lp.m)
    assert info1["iters"] == info0["iters"]
    assert torch.equal(dy1, dy0) and torch.equal(dw1, dw0)
    with pytest.raises(lpk.LpkError) as e:
        ctx.set_wait_limit(0.0)
    assert e.value.status == lpk.INVALID_ARG
    P.free()
    ctx.close()
