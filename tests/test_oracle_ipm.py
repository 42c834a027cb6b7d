"""Pins of the oracle's interior-point method (Algorithm 1): closed forms, brute
force vertex enumeration, and the HiGHS simplex/IPM in scipy.  CPU only."""
import itertools

import numpy as np
import pytest
from scipy.optimize import linprog

from paper_1604_07491_gb300 import gen


def highs(lp):
    r = linprog(lp.c, A_eq=lp.scipy(), b_eq=lp.b, bounds=(0, None), method="highs")
    assert r.status == 0
    return r.fun


def certificates_ok(lp, x, y, s, tol=1e-8):
    A = lp.scipy()
    pinf = np.linalg.norm(lp.b - A @ x) / max(np.linalg.norm(lp.b), 1)
    dinf = np.linalg.norm(lp.c - A.T @ y - s) / max(np.linalg.norm(lp.c), 1)
    pobj, dobj = lp.c @ x, lp.b @ y
    gap = abs(pobj - dobj) / (1 + abs(pobj))
    return pinf <= tol and dinf <= tol and gap <= tol and (x > 0).all() and (s > 0).all()


def vertex_optimum(A, b, c):
    """min c^T x over {Ax = b, x >= 0} by enumerating all bases (tiny, full row rank)."""
    m, n = A.shape
    best = np.inf
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-12:
            continue
        xB = np.linalg.solve(AB, b)
        if (xB >= -1e-12).all():
            best = min(best, c[list(B)] @ xB)
    return best


def test_closed_form_two_variables(orc):
    # min x1 s.t. x1 + x2 = 1, x >= 0  ->  x = (0, 1), y = 0, s = (1, 0), optimum 0
    rp = np.array([0, 2], np.int64)
    ci = np.array([0, 1], np.int32)
    v = np.array([1.0, 1.0])
    x, y, s, info = orc.lp_solve(1, 2, rp, ci, v, np.array([1.0]), np.array([1.0, 0.0]))
    assert info["status_name"] == "OK"
    assert np.allclose(x, [0, 1], atol=1e-7) and np.allclose(s, [1, 0], atol=1e-7)
    assert abs(y[0]) < 1e-7 and abs(info["obj_primal"]) < 1e-7


@pytest.mark.parametrize("seed", range(6))
def test_micro_lps_match_vertex_enumeration(orc, seed):
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(2, 5)), int(rng.integers(5, 10))
    lp = gen.random_density_lp(m, n, 0.7, seed=200 + seed)
    A = lp.scipy().toarray()
    if np.linalg.matrix_rank(A) < m:
        pytest.skip("rank-deficient draw")
    opt = vertex_optimum(A, lp.b, lp.c)
    x, y, s, info = orc.lp_solve_lp(lp)
    assert info["status_name"] == "OK"
    assert abs(info["obj_primal"] - opt) <= 1e-7 * (1 + abs(opt))
    assert certificates_ok(lp, x, y, s)


def test_micro_rank_deficient_lp(orc):
    # a duplicated row: A A^T is singular, the LP keeps its optimum
    lp = gen.random_density_lp(3, 8, 0.8, seed=77)
    A = lp.scipy().toarray()
    A2 = np.vstack([A, 2.0 * A[1]])
    b2 = np.concatenate([lp.b, [2.0 * lp.b[1]]])
    import scipy.sparse as sp
    S = sp.csr_matrix(A2)
    x, y, s, info = orc.lp_solve(4, 8, S.indptr.astype(np.int64), S.indices.astype(np.int32),
                                 S.data, b2, lp.c)
    assert info["status_name"] == "OK"
    opt = vertex_optimum(A, lp.b, lp.c)
    assert abs(info["obj_primal"] - opt) <= 1e-7 * (1 + abs(opt))


@pytest.mark.parametrize("method", [0, 1, 2])
def test_tiny_lp_matches_highs(orc, method):
    lp = gen.tiny_lp()
    x, y, s, info = orc.lp_solve_lp(lp, method=method, inner_sweeps=1 if method < 2 else 2)
    assert info["status_name"] == "OK"
    ref = highs(lp)
    assert abs(info["obj_primal"] - ref) <= 1e-7 * abs(ref)
    assert certificates_ok(lp, x, y, s)
    # the construction's feasible pair brackets the optimum (weak duality)
    assert lp.b @ lp.y0 - 1e-9 <= info["obj_primal"] <= lp.c @ lp.x0 + 1e-9


def test_assignment_lp_matches_highs(orc):
    lp = gen.assignment_lp()
    x, y, s, info = orc.lp_solve_lp(lp, inner_sweeps=3)
    assert info["status_name"] == "OK"
    ref = highs(lp)
    assert abs(info["obj_primal"] - ref) <= 1e-7 * abs(ref)
    assert certificates_ok(lp, x, y, s)


def test_medium_family_small_scale_matches_highs(orc):
    lp = gen.medium_lp(scale=0.03)   # m = 600, n = 1800, 6 dependent rows
    x, y, s, info = orc.lp_solve_lp(lp, inner_sweeps=3, max_krylov=3 * lp.m)
    assert info["status_name"] == "OK"
    ref = highs(lp)
    assert abs(info["obj_primal"] - ref) <= 1e-7 * abs(ref)
    assert certificates_ok(lp, x, y, s)


def test_empty_rows_and_columns_are_removed(orc):
    lp = gen.tiny_lp()
    A = lp.scipy().toarray()
    # insert an empty row (b = 0) and an empty column (c = 3)
    A2 = np.zeros((lp.m + 1, lp.n + 1))
    A2[:lp.m, :lp.n] = A
    b2 = np.concatenate([lp.b, [0.0]])
    c2 = np.concatenate([lp.c, [3.0]])
    import scipy.sparse as sp
    S = sp.csr_matrix(A2)
    x, y, s, info = orc.lp_solve(lp.m + 1, lp.n + 1, S.indptr.astype(np.int64),
                                 S.indices.astype(np.int32), S.data, b2, c2)
    assert info["status_name"] == "OK"
    assert x[-1] == 0.0 and s[-1] == 3.0 and y[-1] == 0.0
    assert abs(info["obj_primal"] - highs(lp)) <= 1e-7 * abs(highs(lp))
    # inconsistent empty row / unbounded empty column
    b3 = b2.copy()
    b3[-1] = 1.0
    *_, info = orc.lp_solve(lp.m + 1, lp.n + 1, S.indptr.astype(np.int64),
                            S.indices.astype(np.int32), S.data, b3, c2)
    assert info["status_name"] == "EMPTY_ROW_INCONSISTENT"
    c3 = c2.copy()
    c3[-1] = -1.0
    *_, info = orc.lp_solve(lp.m + 1, lp.n + 1, S.indptr.astype(np.int64),
                            S.indices.astype(np.int32), S.data, b2, c3)
    assert info["status_name"] == "EMPTY_COL_UNBOUNDED"


def test_oracle_is_deterministic(orc):
    lp = gen.tiny_lp()
    r1 = orc.lp_solve_lp(lp)
    r2 = orc.lp_solve_lp(lp)
    for a, b in zip(r1[:3], r2[:3]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("method", [0, 2])
def test_tiny_lp_with_bagmres_corrector_matches_highs(orc, method):
    # the corrector stage solved in least-squares form by BA-GMRES (Sec. 3.2)
    lp = gen.tiny_lp()
    x, y, s, info = orc.lp_solve_lp(lp, method=method, inner_sweeps=1 if method < 2 else 2,
                                    corrector_ba=1)
    assert info["status_name"] == "OK"
    ref = highs(lp)
    assert abs(info["obj_primal"] - ref) <= 1e-7 * abs(ref)
    assert certificates_ok(lp, x, y, s)


@pytest.mark.parametrize("name", ["tiny", "micro_rank_deficient", "assignment"])
def test_multiple_centrality_correctors_reach_the_optimum(orc, name):
    # the multi-corrector interior-point framework (Sec. 4.3 and 5): the same
    # optimum, at most as many interior-point iterations, correctors accepted
    if name == "tiny":
        lp, kw = gen.tiny_lp(), dict(inner_sweeps=1)
    elif name == "assignment":
        lp, kw = gen.assignment_lp(), dict(inner_sweeps=3, method=2)
    else:
        lp, kw = gen.medium_lp(scale=0.004, seed=21), dict(inner_sweeps=3)
    x0, y0, s0, i0 = orc.lp_solve_lp(lp, **kw)
    x, y, s, info = orc.lp_solve_lp(lp, max_correctors=2, **kw)
    assert info["status_name"] == "OK" and i0["status_name"] == "OK"
    ref = highs(lp)
    assert abs(info["obj_primal"] - ref) <= 1e-7 * max(1.0, abs(ref))
    assert certificates_ok(lp, x, y, s)
    assert info["correctors"] > 0
    assert info["ipm_iters"] <= i0["ipm_iters"]
