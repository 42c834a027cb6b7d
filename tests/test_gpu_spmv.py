"""GPU parity of the sparse products y = A x and y = A^T x (lpk_spmv) on
matrices built to hit every case of the entry-balanced kernel: a warp takes
256 consecutive entries, a lane 8, so rows of 1, 7, 8, 9, 255, 256 and 257
entries, rows that span many warps (up to 20,000 entries), rows starting
exactly at a warp or lane boundary, empty rows and columns (removed by
lpk_prepare, written as zero), a single entry, and entry counts that end
mid-lane, mid-warp and exactly on a warp boundary.

Reference: the definition y_i = sum_j a_ij x_j with the products summed
exactly (math.fsum).  The kernel runs a multiply-add chain per lane and
combines lanes and warps in a fixed tree, so each entry may differ from the
exactly summed value by the summation error of any order:
|y_i - ref_i| <= (2 len_i + 4) u (|A| |x|)_i, u = 2^-53."""
import math
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def lpk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07491_gb300 import build, lpk as L
    build.build()
    return L


@pytest.fixture(scope="module")
def ctx(lpk):
    c = lpk.Context(0)
    yield c
    c.close()


def csr_from_lengths(lengths, n, seed):
    rng = np.random.default_rng(seed)
    rp = np.zeros(len(lengths) + 1, np.int64)
    rp[1:] = np.cumsum(lengths)
    ci = np.empty(rp[-1], np.int32)
    for i, L in enumerate(lengths):
        ci[rp[i]:rp[i + 1]] = np.sort(rng.choice(n, size=L, replace=False))
    val = rng.standard_normal(rp[-1]) * np.exp(rng.uniform(-3, 3, rp[-1]))
    return rp, ci, val


def exact_products(m, n, rp, ci, val, x, transpose):
    out, bound = [], []
    if not transpose:
        for i in range(m):
            pr = val[rp[i]:rp[i + 1]] * x[ci[rp[i]:rp[i + 1]]]
            out.append(math.fsum(pr))
            bound.append((2 * len(pr) + 4) * U * float(np.abs(pr).sum()))
        return np.array(out), np.array(bound)
    rows = np.repeat(np.arange(m), np.diff(rp))
    order = np.argsort(ci, kind="stable")
    cp = np.zeros(n + 1, np.int64)
    np.add.at(cp, ci + 1, 1)
    cp = np.cumsum(cp)
    for j in range(n):
        q = order[cp[j]:cp[j + 1]]
        pr = val[q] * x[rows[q]]
        out.append(math.fsum(pr))
        bound.append((2 * len(pr) + 4) * U * float(np.abs(pr).sum()))
    return np.array(out), np.array(bound)


def pattern(name):
    rng = np.random.default_rng(7)
    if name == "lane_edges":      # lengths around a lane (8) and a warp (256)
        return [1, 7, 8, 9, 255, 256, 257, 8, 8, 8, 1, 1, 1, 1, 1, 1, 1, 1] * 9, 600
    if name == "long_rows":       # rows spanning many warps, between short ones
        return [3, 20000, 1, 5, 700, 256, 256, 2, 4096, 9], 21000
    if name == "empty_rows":      # empty rows (removed by lpk_prepare) between rows
        return [0, 0, 3, 0, 5, 0, 0, 256, 0, 1, 0, 0, 40, 0], 300
    if name == "power_law":       # ragged power-law rows
        return list(np.minimum(rng.zipf(1.7, size=3000), 5000)), 6000
    if name == "single":
        return [1], 4
    if name == "warp_multiple":   # nnz exactly 4 warps
        return [16] * 64, 64
    if name == "ragged_tail":     # nnz = 4 warps + 3 entries
        return [16] * 64 + [3], 64
    raise KeyError(name)


@pytest.mark.parametrize("name", ["lane_edges", "long_rows", "empty_rows", "power_law", "single",
                                  "warp_multiple", "ragged_tail"])
@pytest.mark.parametrize("transpose", [False, True])
def test_spmv_structures(lpk, ctx, name, transpose):
    lengths, n = pattern(name)
    m = len(lengths)
    rp, ci, val = csr_from_lengths(lengths, n, seed=zlib.crc32(name.encode()))
    P = lpk.Problem(ctx, m, n, rp, ci, val)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(m if transpose else n)
    y = P.spmv(x, transpose=transpose)
    ref, bound = exact_products(m, n, rp, ci, val, x, transpose)
    err = np.abs(y - ref)
    assert np.all(err <= bound), (int(np.argmax(err - bound)), float(np.max(err - bound)))
    # empty rows / columns are written as exact zeros
    empty = (np.diff(rp) == 0) if not transpose else (np.bincount(ci, minlength=n) == 0)
    assert np.all(y[empty] == 0.0)
    # the same call twice gives the same bits (fixed combination order)
    assert np.array_equal(P.spmv(x, transpose=transpose), y)
    P.free()


def test_spmv_large_rows_sampled(lpk, ctx):
    """The large power-law LP at full size (150,000 x 434,580, 2.6 M entries):
    500 sampled rows and columns against the exact sums."""
    from paper_1604_07491_gb300 import gen
    lp = gen.large_lp(1.0)
    P = lpk.Problem.from_lp(ctx, lp)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(lp.n)
    yv = rng.standard_normal(lp.m)
    y = P.spmv(x)
    yt = P.spmv(yv, transpose=True)
    A = lp.scipy()
    At = A.T.tocsr()
    for M, vec, out, rows in ((A, x, y, rng.choice(lp.m, 500, replace=False)),
                              (At, yv, yt, rng.choice(lp.n, 500, replace=False))):
        for i in rows:
            lo, hi = M.indptr[i], M.indptr[i + 1]
            pr = M.data[lo:hi] * vec[M.indices[lo:hi]]
            assert abs(out[i] - math.fsum(pr)) <= (2 * len(pr) + 4) * U * np.abs(pr).sum()
    P.free()
