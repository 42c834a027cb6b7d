"""Dataflow sweeps (grid path, rows cached in shared memory; LPK_EXEC_DATAFLOW):
instead of a grid barrier after every color, each warp waits on the flags of
the rows before its rows that touch their columns (the previous row of each
column in the sweep order), and one barrier ends each pass.  Rows of one
color share no column, so every row reads exactly the u values it reads with
a barrier per color: the results must be bitwise those of the per-color
barrier order.  Checked for lone sweeps (NE-SOR and NE-SSOR, several inner
sweeps, omega != 1), Krylov solves and a complete LP solve, on short rows
(batched updates) and long rows, FP32 and FP64 values.  The flag waits are
bounded: with CTA 0's flags withheld the call returns LPK_TIMEOUT, and the
context then gives the bitwise-same result again."""
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


@pytest.fixture(scope="module")
def ctxs(lpk):
    flow = lpk.Context(0)
    flow.set_exec(lpk.EXEC_GRID | lpk.EXEC_DATAFLOW)
    bar = lpk.Context(0)
    bar.set_exec(lpk.EXEC_GRID | lpk.EXEC_COLOR_BARRIERS)
    yield flow, bar
    flow.close()
    bar.close()


_LPS = {}


def lp_named(name):
    if name not in _LPS:
        _LPS[name] = {"large": lambda: gen.large_lp(1.0), "medium": lambda: gen.medium_lp(1.0),
                      "medium_0.05": lambda: gen.medium_lp(0.05)}[name]()
    return _LPS[name]


def pair(lpk, ctxs, name):
    lp = lp_named(name)
    return lp, [lpk.Problem.from_lp(c, lp, device="cuda") for c in ctxs]


def inputs(lp, seed):
    rng = np.random.default_rng(seed)
    d2 = torch.from_numpy(np.exp(rng.uniform(-4, 4, lp.n))).cuda()
    g = torch.from_numpy(rng.standard_normal(lp.m)).cuda()
    return d2, g


CASES = [(1, 1, 1.0), (0, 2, 1.2), (1, 3, 0.8)]  # (kind NE_SOR=1 / NE_SSOR=0, inner sweeps, omega)


@pytest.mark.parametrize("name,precision", [("large", 1), ("medium", 1), ("medium", 0)])
def test_sweep_bitwise(lpk, ctxs, name, precision):
    """large: 406 colors, rows of at most 39 entries (batched short rows);
    medium: 50 colors, rows up to 68 entries (one row at a time)."""
    lp, (Pf, Pb) = pair(lpk, ctxs, name)
    assert Pf.n_colors >= 32
    for kind, ell, om in CASES:
        d2, g = inputs(lp, 100 + ell)
        zf, uf = Pf.sweep(d2, g, kind=kind, inner_sweeps=ell, omega=om, precision=precision)
        sf = ctxs[0].stats()
        zb, ub = Pb.sweep(d2, g, kind=kind, inner_sweeps=ell, omega=om, precision=precision)
        sb = ctxs[1].stats()
        assert sf["last_resident"] == 1 and sf["last_dataflow"] == 1, sf
        assert sb["last_resident"] == 1 and sb["last_dataflow"] == 0, sb
        assert torch.equal(zf, zb) and torch.equal(uf, ub), (kind, ell, om)
        assert torch.isfinite(zf).all()
    Pf.free()
    Pb.free()


@pytest.mark.parametrize("solver,precision", [(2, 1), (0, 1), (2, 0)])
def test_ne_solve_bitwise(lpk, ctxs, solver, precision):
    lp, (Pf, Pb) = pair(lpk, ctxs, "medium_0.05")
    rng = np.random.default_rng(5)
    d2 = torch.from_numpy(np.exp(rng.uniform(-3, 3, lp.n))).cuda()
    f = torch.from_numpy(lp.scipy() @ (d2.cpu().numpy() * rng.standard_normal(lp.n))).cuda()
    rf = Pf.ne_solve(d2, f, inner_sweeps=2, solver=solver, precision=precision, tol=1e-9, max_iter=10 * lp.m)
    rb = Pb.ne_solve(d2, f, inner_sweeps=2, solver=solver, precision=precision, tol=1e-9, max_iter=10 * lp.m)
    assert ctxs[0].stats()["last_dataflow"] == 1 and ctxs[1].stats()["last_dataflow"] == 0
    assert rf[2]["converged"] and rf[2]["iters"] == rb[2]["iters"]
    assert torch.equal(rf[0], rb[0]) and torch.equal(rf[1], rb[1])
    Pf.free()
    Pb.free()


def test_lp_solve_bitwise(lpk, ctxs):
    lp, (Pf, Pb) = pair(lpk, ctxs, "medium_0.05")
    b, c = torch.from_numpy(lp.b).cuda(), torch.from_numpy(lp.c).cuda()
    kw = dict(solver=2, inner_sweeps=2, precision=1)
    xf, yf, sf, inf_f = Pf.lp_solve(b, c, **kw)
    xb, yb, sb, inf_b = Pb.lp_solve(b, c, **kw)
    assert inf_f["status_name"] == "OK"
    assert inf_f["ipm_iters"] == inf_b["ipm_iters"]
    assert torch.equal(xf, xb) and torch.equal(yf, yb) and torch.equal(sf, sb)
    Pf.free()
    Pb.free()


def test_flag_wait_times_out_and_context_recovers(lpk):
    lp = lp_named("medium_0.05")
    ctx = lpk.Context(0)
    ctx.set_exec(lpk.EXEC_GRID | lpk.EXEC_DATAFLOW)
    P = lpk.Problem.from_lp(ctx, lp, device="cuda")
    d2, g = inputs(lp, 3)
    z0, u0 = P.sweep(d2, g, kind=1, inner_sweeps=3, precision=1)
    assert ctx.stats()["last_dataflow"] == 1
    ctx.set_wait_limit(0.02, test_stall_barrier=-2)  # CTA 0 publishes no flag from pass 2 on
    t0 = time.time()
    with pytest.raises(lpk.LpkError) as e:
        P.sweep(d2, g, kind=1, inner_sweeps=3, precision=1)
    assert e.value.status == lpk.TIMEOUT and "timed out" in str(e.value)
    assert time.time() - t0 < 2.0
    ctx.set_wait_limit(5.0, 0)
    z1, u1 = P.sweep(d2, g, kind=1, inner_sweeps=3, precision=1)
    assert torch.equal(z1, z0) and torch.equal(u1, u0)
    P.free()
    ctx.close()
