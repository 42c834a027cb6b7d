"""lpk_ne_solve_noalloc: the search-direction solve for callers that cannot
call cudaMalloc while they solve (applications whose device memory belongs to
their own allocator, services that must not run out of memory mid-solve).  Its
temporaries live in a fixed device array reserved when the first context on a
device is created.  The test calls it through the C ABI and checks it against
the allocating lpk_ne_solve on the same path, twice in a row (the shared array
keeps the previous call's contents), and checks that an oversized problem, host
memory and badly typed or short tensors are rejected with a clear error.
Collected last so that a stop at the first failure has run every other test."""
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


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("name,solver,precision", [("medium_0.05", 0, 0), ("assignment", 1, 1)])
def test_noalloc_matches_ne_solve_twice(lpk, name, solver, precision):
    lp = gen.medium_lp(0.05) if name == "medium_0.05" else gen.assignment_lp()
    ctx = lpk.Context(0)
    ctx.set_exec(lpk.EXEC_GRID)          # the no-allocation variant runs the grid path
    P = lpk.Problem.from_lp(ctx, lp, device="cuda")
    rng = np.random.default_rng(11)
    ell = 3 if name == "assignment" else 1
    for call in range(2):
        d2 = torch.from_numpy(np.exp(rng.uniform(-3, 3, lp.n))).cuda()
        f = torch.from_numpy(lp.scipy() @ (d2.cpu().numpy() * rng.standard_normal(lp.n))).cuda()
        dy_ref, dw_ref, info_ref = P.ne_solve(d2, f, inner_sweeps=ell, solver=solver,
                                              precision=precision, tol=1e-9, max_iter=20 * lp.m)
        dy = torch.full((lp.m,), float("nan"), dtype=torch.float64, device="cuda")
        dw = torch.full((lp.n,), float("nan"), dtype=torch.float64, device="cuda")
        info = P.ne_solve_noalloc(d2, f, dy, dw, inner_sweeps=ell, solver=solver, precision=precision,
                                  tol=1e-9, max_iter=20 * lp.m)
        torch.cuda.synchronize()
        assert info["converged"] and info_ref["converged"], (call, info, info_ref)
        assert info["iters"] == info_ref["iters"]
        assert rel(dy, dy_ref) < 1e-11 and rel(dw, dw_ref) < 1e-11, call
    P.free()
    ctx.close()


def test_noalloc_rejects_oversized_problem(lpk):
    m = n = 300_000                    # about 8 doubles per row and column: more than 32 MiB
    rp = np.arange(m + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    ctx = lpk.Context(0)
    P = lpk.Problem(ctx, m, n, rp, ci, np.ones(n))
    d2 = torch.ones(n, dtype=torch.float64, device="cuda")
    f = torch.ones(m, dtype=torch.float64, device="cuda")
    dy = torch.empty(m, dtype=torch.float64, device="cuda")
    with pytest.raises(lpk.LpkError) as e:
        P.ne_solve_noalloc(d2, f, dy)
    assert e.value.status == lpk.INVALID_ARG and "MiB" in str(e.value)
    P.free()
    ctx.close()


def test_noalloc_rejects_bad_buffers(lpk):
    """Host memory is refused by the C entry point; the binding refuses
    tensors of the wrong type or length before the call (the C call takes
    no lengths)."""
    import ctypes as C
    lp = gen.tiny_lp()
    ctx = lpk.Context(0)
    P = lpk.Problem.from_lp(ctx, lp, device="cuda")
    d2 = torch.ones(lp.n, dtype=torch.float64, device="cuda")
    f = torch.ones(lp.m, dtype=torch.float64, device="cuda")
    dy = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    host_d2 = np.ones(lp.n)
    ki = lpk.KrylovInfo()
    st = lpk.load().lpk_ne_solve_noalloc(ctx.handle, P._h, C.c_void_p(host_d2.ctypes.data),
                                         C.c_void_p(f.data_ptr()), 1, 1.0, lpk.MRNE, lpk.FP64, 1e-8, 0,
                                         C.c_void_p(dy.data_ptr()), None, C.byref(ki))
    assert st == lpk.INVALID_ARG and "device" in ctx.last_error()
    with pytest.raises(ValueError):
        P.ne_solve_noalloc(d2.float(), f, dy)
    with pytest.raises(ValueError):
        P.ne_solve_noalloc(d2, f, dy[: lp.m - 1])
    with pytest.raises(ValueError):
        P.ne_solve_noalloc(d2.cpu(), f, dy)
    info = P.ne_solve_noalloc(d2, f, dy, tol=1e-10)
    assert info["converged"]
    P.free()
    ctx.close()
