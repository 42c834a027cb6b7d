"""Seeded generators: determinism and the structure of each workload family."""
import numpy as np

from paper_1604_07491_gb300 import gen


def test_deterministic():
    a, b = gen.medium_lp(0.05), gen.medium_lp(0.05)
    for f in ("row_ptr", "col_idx", "val", "b", "c"):
        assert np.array_equal(getattr(a, f), getattr(b, f))


def test_tiny_structure():
    lp = gen.tiny_lp()
    assert (lp.m, lp.n) == (50, 120)
    A = lp.scipy().toarray()
    assert (A != 0).any(axis=0).all() and (A != 0).any(axis=1).all()
    assert 0.03 < (A != 0).mean() < 0.08
    assert np.allclose(A @ lp.x0, lp.b) and np.allclose(A.T @ lp.y0 + lp.s0, lp.c)


def test_medium_structure():
    lp = gen.medium_lp()
    assert (lp.m, lp.n) == (20000, 60000)
    A = lp.scipy()
    base = A[:19800]
    assert (np.diff(base.tocsc().indptr) == 8).all()        # 8 distinct rows per column
    assert 480_000 < lp.nnz < 500_000
    assert np.allclose(A @ lp.x0, lp.b)


def test_assignment_structure():
    lp = gen.assignment_lp()
    assert (lp.m, lp.n, lp.nnz) == (588, 38416, 115248)
    A = lp.scipy()
    assert (np.diff(A.tocsc().indptr) == 3).all()
    assert np.allclose(A @ np.full(lp.n, 1 / 196), 1.0)
    assert set(np.unique(lp.c)) <= set(range(101))


def test_large_degrees():
    lp = gen.large_lp(scale=0.1)
    deg = np.diff(lp.scipy().tocsc().indptr)
    assert deg.max() == 400 and abs(deg.mean() - 6.0) < 0.05


def test_serving_sizes():
    t = gen.serving_arrivals(2000)
    assert np.all(np.diff(t) > 0) and 30 < t[-1] < 50
    lp = gen.serving_lp(3)
    assert 100 <= lp.m <= 20000 and lp.n == 3 * lp.m
