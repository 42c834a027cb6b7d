"""Seeded synthetic LP generators.

This module only draws random numbers and assembles standard-form LP data
(min c^T x s.t. Ax = b, x >= 0).  It holds none of the interior-point or Krylov
arithmetic; both the CUDA path and the CPU oracle are fed from here.

Feasibility construction used by the random families: draw x0 ~ U(0.5, 2),
y0 ~ N(0, 1), s0 ~ U(0.5, 2) and set b = A x0, c = A^T y0 + s0, so (x0, y0, s0)
is a strictly interior primal-dual pair and an optimum exists (the paper assumes
one exists, Sec. 1 after the primal-dual pair).

Families (sizes are the workloads the benchmarks and tests use):
  tiny_lp        m=50,  n=120, ~5% density (entries N(0,1) at uniform positions)
  medium_lp      m=20,000, n=60,000, 8 nnz per column, plus 1% of rows that are
                 linear combinations of two other rows (rank-deficient)
  assignment_lp  k=14: K=k^2=196, n=K^2=38,416 0/1 columns, row-sum, column-sum
                 and k^2 block-coupling equalities (m=588), integer costs U{0..100}
  large_lp       m=150,000, n=434,580, power-law column degrees (mean 6, max 400)
  serving_stream arrival times and sizes of a Poisson stream of random LPs
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

SEED_BASE = 20160407


@dataclasses.dataclass
class LP:
    """Standard-form LP in CSR (row_ptr int64, col_idx int32, val float64)."""
    name: str
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    b: np.ndarray
    c: np.ndarray
    x0: np.ndarray | None = None   # known feasible primal point (construction)
    y0: np.ndarray | None = None   # known feasible dual point (construction)
    s0: np.ndarray | None = None

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.m, self.n))


def _csr_from_coo(m, n, rows, cols, vals) -> sp.csr_matrix:
    A = sp.coo_matrix((vals, (rows, cols)), shape=(m, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def _distinct_rows_per_column(rng, m, degrees):
    """For column j draw degrees[j] distinct row indices uniformly from [0, m)."""
    n = len(degrees)
    cols = np.repeat(np.arange(n, dtype=np.int64), degrees)
    rows = rng.integers(0, m, size=cols.size, dtype=np.int64)
    while True:
        order = np.lexsort((rows, cols))
        rs, cs = rows[order], cols[order]
        dup = np.zeros(rs.size, dtype=bool)
        dup[1:] = (rs[1:] == rs[:-1]) & (cs[1:] == cs[:-1])
        if not dup.any():
            return rs, cs
        idx = order[dup]
        rows[np.sort(idx)] = rng.integers(0, m, size=idx.size, dtype=np.int64)


def _fill_empty_rows(rng, m, n, rows, cols):
    """Give every empty row one entry at a uniform column (empty rows are removed
    by the method's preprocessing, so the generators never emit them)."""
    counts = np.bincount(rows, minlength=m)
    empty = np.flatnonzero(counts == 0)
    if empty.size == 0:
        return rows, cols, 0
    extra_cols = rng.integers(0, n, size=empty.size, dtype=np.int64)
    return (np.concatenate([rows, empty]), np.concatenate([cols, extra_cols]), empty.size)


def _feasible_pair(rng, A: sp.csr_matrix):
    m, n = A.shape
    x0 = rng.uniform(0.5, 2.0, size=n)
    y0 = rng.standard_normal(m)
    s0 = rng.uniform(0.5, 2.0, size=n)
    b = A @ x0
    c = A.T @ y0 + s0
    return x0, y0, s0, np.asarray(b, dtype=np.float64), np.asarray(c, dtype=np.float64)


def _pack(name, A: sp.csr_matrix, b, c, x0=None, y0=None, s0=None) -> LP:
    m, n = A.shape
    return LP(name=name, m=m, n=n,
              row_ptr=A.indptr.astype(np.int64), col_idx=A.indices.astype(np.int32),
              val=A.data.astype(np.float64), b=np.ascontiguousarray(b, dtype=np.float64),
              c=np.ascontiguousarray(c, dtype=np.float64), x0=x0, y0=y0, s0=s0)


def random_density_lp(m=50, n=120, density=0.05, seed=SEED_BASE + 1, name=None) -> LP:
    """Entries nonzero with probability `density`, N(0,1); every column and row
    gets at least one nonzero; x0/y0/s0 feasibility construction."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    for j in np.flatnonzero(~mask.any(axis=0)):
        mask[rng.integers(0, m), j] = True
    for i in np.flatnonzero(~mask.any(axis=1)):
        mask[i, rng.integers(0, n)] = True
    rows, cols = np.nonzero(mask)
    vals = rng.standard_normal(rows.size)
    A = _csr_from_coo(m, n, rows, cols, vals)
    x0, y0, s0, b, c = _feasible_pair(rng, A)
    return _pack(name or f"tiny_m{m}_n{n}", A, b, c, x0, y0, s0)


def tiny_lp(seed=SEED_BASE + 1) -> LP:
    """m=50, n=120, ~5% nonzeros N(0,1) at uniform positions."""
    return random_density_lp(50, 120, 0.05, seed, name="tiny_m50_n120")


def column_degree_lp(m_base, n, degrees, n_dup_rows=0, seed=SEED_BASE, name="lp") -> LP:
    """Column j gets degrees[j] distinct uniform rows among the m_base base rows
    with N(0,1) values; then n_dup_rows rows a*row_i + b*row_j (i != j uniform,
    a, b ~ N(0,1)) are appended; then the x0/y0/s0 construction."""
    rng = np.random.default_rng(seed)
    degrees = np.asarray(degrees, dtype=np.int64)
    rows, cols = _distinct_rows_per_column(rng, m_base, degrees)
    rows, cols, _ = _fill_empty_rows(rng, m_base, n, rows, cols)
    vals = rng.standard_normal(rows.size)
    A = _csr_from_coo(m_base, n, rows, cols, vals)
    if n_dup_rows:
        i = rng.integers(0, m_base, size=n_dup_rows)
        j = rng.integers(0, m_base - 1, size=n_dup_rows)
        j = j + (j >= i)                              # j != i, uniform
        a = rng.standard_normal(n_dup_rows)
        bb = rng.standard_normal(n_dup_rows)
        extra = sp.diags(a) @ A[i] + sp.diags(bb) @ A[j]
        extra = sp.csr_matrix(extra)
        extra.eliminate_zeros()
        A = sp.vstack([A, extra], format="csr")
        A.sort_indices()
    x0, y0, s0, b, c = _feasible_pair(rng, A)
    return _pack(name, A, b, c, x0, y0, s0)


def medium_lp(scale=1.0, seed=SEED_BASE + 2) -> LP:
    """Rank-deficient sparse LP: m = 20,000 * scale rows (99% base rows with
    8 nonzeros per column, 1% duplicated as combinations of two base rows),
    n = 60,000 * scale."""
    m = int(round(20000 * scale))
    n = int(round(60000 * scale))
    n_dup = max(1, int(round(0.01 * m)))
    return column_degree_lp(m - n_dup, n, np.full(n, 8), n_dup, seed,
                            name=f"medium_m{m}_n{n}")


def assignment_lp(k=14, seed=SEED_BASE + 3) -> LP:
    """Degenerate assignment-structured LP with K = k^2 and n = K^2 variables
    X[p,q] (index p*K + q): K row sums = 1, K column sums = 1, and k^2 block
    rows (one per block (I, J) of the k x k block partition of p and q) = 1.
    All coefficients 1, costs integers U{0..100}; X = 1/K is strictly
    feasible. Rank-deficient (block rows sum to row sums)."""
    rng = np.random.default_rng(seed)
    K = k * k
    n = K * K
    p = np.repeat(np.arange(K), K)
    q = np.tile(np.arange(K), K)
    j = np.arange(n)
    rows = np.concatenate([p, K + q, 2 * K + (p // k) * k + (q // k)])
    cols = np.concatenate([j, j, j])
    A = _csr_from_coo(2 * K + k * k, n, rows, cols, np.ones(rows.size))
    b = np.ones(A.shape[0])
    c = rng.integers(0, 101, size=n).astype(np.float64)
    return _pack(f"assign_k{k}", A, b, c, x0=np.full(n, 1.0 / K))


def power_law_degrees(rng, n, mean=6.0, d_min=2, d_max=400):
    """d_j = min(d_max, max(1, floor(d_min * U^(-1/(a-1))))) with the exponent a
    bisected so the sample mean is mean +- 0.02; column 0 has degree d_max."""
    U = rng.random(n)
    U[U == 0.0] = 0.5

    def degs(a):
        d = np.floor(d_min * U ** (-1.0 / (a - 1.0)))
        d = np.minimum(d_max, np.maximum(1, d)).astype(np.int64)
        d[0] = d_max
        return d

    lo, hi = 1.05, 50.0                    # mean decreases as a grows
    for _ in range(200):
        a = 0.5 * (lo + hi)
        mu = degs(a).mean()
        if abs(mu - mean) <= 0.02:
            break
        if mu > mean:
            lo = a
        else:
            hi = a
    return degs(a)


def large_lp(scale=1.0, seed=SEED_BASE + 4) -> LP:
    """m = 150,000 * scale, n = 434,580 * scale, power-law column degrees with
    mean 6 and maximum 400, N(0,1) values, x0/y0/s0 construction."""
    m = int(round(150000 * scale))
    n = int(round(434580 * scale))
    rng = np.random.default_rng(seed)
    d = power_law_degrees(rng, n, d_max=min(400, m))
    sub = int(rng.integers(0, 2**62))
    return column_degree_lp(m, n, d, 0, sub, name=f"large_m{m}_n{n}")


def serving_lp(index, seed_base=SEED_BASE + 5) -> LP:
    """LP number `index` of the serving stream: m = floor(exp(U(ln 100, ln 20000))),
    n = 3m, 6 distinct uniform rows per column with N(0,1) values."""
    rng = np.random.default_rng(seed_base + index)
    m = int(math.floor(math.exp(rng.uniform(math.log(100), math.log(20000)))))
    n = 3 * m
    sub = int(rng.integers(0, 2**62))
    return column_degree_lp(m, n, np.full(n, 6), 0, sub, name=f"serve{index}_m{m}")


def serving_arrivals(count=2000, rate=50.0, seed=SEED_BASE + 5):
    """Arrival times (seconds) of a Poisson stream: gaps ~ Exp(1/rate)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


CONFIGS = {
    "tiny": tiny_lp,
    "medium": medium_lp,
    "assignment": assignment_lp,
    "large": large_lp,
}
