"""Pins of the CPU oracle against values and properties fixed by the paper and by
mathematics (not by the oracle itself).  CPU only."""
import os

import numpy as np
import pytest

from paper_1604_07491_gb300 import gen

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = 0x9E3779B97F4A7C15


def small_lp(m=12, n=30, density=0.3, seed=7):
    return gen.random_density_lp(m, n, density, seed)


def dense(lp):
    return lp.scipy().toarray()


# ---------------------------------------------------------------- splitmix64
def test_splitmix64_published_sequence(orc):
    want = [int(l, 16) for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    got = [orc.splitmix64((k * GOLDEN) % 2**64) for k in range(3)]
    assert got == want


# ---------------------------------------------------------------- coloring
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_coloring_is_valid_greedy_first_fit(orc, seed):
    lp = gen.random_density_lp(60, 90, 0.06, seed)
    A = dense(lp) != 0
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 0x5EED)
    conflict = (A.astype(int) @ A.T.astype(int)) > 0
    np.fill_diagonal(conflict, False)
    # (1) rows of one color share no column
    for c in range(nc):
        rows = np.flatnonzero(color == c)
        assert not conflict[np.ix_(rows, rows)].any()
    # (2) first fit in decreasing priority: a row's color is the smallest one
    #     not taken by a higher-priority neighbour
    prio = np.array([orc.splitmix64(0x5EED ^ i) for i in range(lp.m)], dtype=object)

    def before(k, i):
        return prio[k] > prio[i] or (prio[k] == prio[i] and k < i)

    for i in range(lp.m):
        higher = [k for k in np.flatnonzero(conflict[i]) if before(k, i)]
        used = {int(color[k]) for k in higher}
        want = 0
        while want in used:
            want += 1
        assert color[i] == want
    # (3) perm lists rows by color, then by row index; color_ptr delimits colors
    assert sorted(perm.tolist()) == list(range(lp.m))
    keys = [(color[r], r) for r in perm]
    assert keys == sorted(keys)
    assert cptr[0] == 0 and cptr[-1] == lp.m
    for c in range(nc):
        assert (color[perm[cptr[c]:cptr[c + 1]]] == c).all()


# ---------------------------------------------------------------- scaling
def test_row_scaling_unit_norms_and_normal_diagonal(orc):
    lp = small_lp()
    rng = np.random.default_rng(0)
    d2 = np.exp(rng.uniform(-8, 8, lp.n))
    ahat, rho = orc.scale_rows(lp.m, lp.row_ptr, lp.col_idx, lp.val, d2)
    A = dense(lp)
    # rho_i^2 is the diagonal of the normal matrix A D^2 A^T (Sec. 3.5)
    assert np.allclose(rho**2, np.diag(A @ np.diag(d2) @ A.T), rtol=1e-13)
    Ah = np.zeros_like(A)
    for i in range(lp.m):
        Ah[i, lp.col_idx[lp.row_ptr[i]:lp.row_ptr[i + 1]]] = ahat[lp.row_ptr[i]:lp.row_ptr[i + 1]]
    assert np.allclose(np.linalg.norm(Ah, axis=1), 1.0, rtol=1e-14)
    # same normal equations up to the row scaling: Ah Ah^T = R^-1 A D^2 A^T R^-1
    R = np.diag(1 / rho)
    assert np.allclose(Ah @ Ah.T, R @ A @ np.diag(d2) @ A.T @ R, atol=1e-13)


# ---------------------------------------------------------------- sweeps
def splitting_ssor(Ad, perm, g, ell, omega):
    """Stationary SSOR iteration on B z = g, B = A A^T, in the permuted order,
    written in splitting-matrix form (Sec. 3.3: A A^T = M - N, H = M^-1 N):
    forward half step with M_F = D/omega + L, backward with M_B = D/omega + L^T."""
    P = np.eye(len(perm))[perm]
    B = P @ Ad @ Ad.T @ P.T
    D = np.diag(np.diag(B))
    L = np.tril(B, -1)
    MF = D / omega + L
    MB = D / omega + L.T
    gp = P @ g
    x = np.zeros_like(gp)
    for _ in range(ell):
        x = x + np.linalg.solve(MF, gp - B @ x)
        x = x + np.linalg.solve(MB, gp - B @ x)
    z = P.T @ x
    return z, Ad.T @ z


def splitting_sor(Ad, perm, g, ell, omega):
    P = np.eye(len(perm))[perm]
    B = P @ Ad @ Ad.T @ P.T
    MF = np.diag(np.diag(B)) / omega + np.tril(B, -1)
    gp = P @ g
    x = np.zeros_like(gp)
    for _ in range(ell):
        x = x + np.linalg.solve(MF, gp - B @ x)
    y = P.T @ x
    return Ad.T @ y, y


@pytest.mark.parametrize("ell,omega", [(1, 1.0), (3, 1.3), (2, 0.7)])
def test_nessor_equals_splitting_form(orc, ell, omega):
    lp = small_lp(m=15, n=40, density=0.25, seed=3)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 11)
    g = np.random.default_rng(1).standard_normal(lp.m)
    z, u = orc.nessor(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, g, ell, omega)
    z2, u2 = splitting_ssor(dense(lp), perm, g, ell, omega)
    assert np.allclose(z, z2, rtol=1e-10, atol=1e-12)
    assert np.allclose(u, u2, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("ell,omega", [(1, 1.0), (4, 1.2)])
def test_nesor_equals_splitting_form(orc, ell, omega):
    lp = small_lp(m=15, n=40, density=0.25, seed=4)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 12)
    g = np.random.default_rng(2).standard_normal(lp.m)
    z, y = orc.nesor(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, g, ell, omega)
    z2, y2 = splitting_sor(dense(lp), perm, g, ell, omega)
    assert np.allclose(z, z2, rtol=1e-10, atol=1e-12)
    assert np.allclose(y, y2, rtol=1e-10, atol=1e-12)
    assert np.allclose(z, dense(lp).T @ y, atol=1e-12)


def test_nessor_symmetric_positive_definite_for_odd_ell(orc):
    # Sec. 3.3: C^<ell> is SPD for ell odd and omega in (0, 2)
    lp = small_lp(m=10, n=30, density=0.3, seed=5)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 3)
    for ell, om in [(1, 1.0), (3, 1.5), (5, 0.6)]:
        C = np.column_stack([orc.nessor(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, e, ell,
                                        om)[0] for e in np.eye(lp.m)])
        assert np.allclose(C, C.T, atol=1e-12 * np.abs(C).max())
        assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0


def test_sweep_rows_of_a_color_commute(orc):
    # rows of one color touch disjoint entries of u: any order inside a color
    # gives bitwise the same sweep
    lp = gen.random_density_lp(80, 200, 0.03, 9)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 5)
    g = np.random.default_rng(3).standard_normal(lp.m)
    z, u = orc.nessor(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, g, 2, 1.1)
    rng = np.random.default_rng(4)
    p2 = perm.copy()
    for c in range(nc):
        seg = p2[cptr[c]:cptr[c + 1]]
        rng.shuffle(seg)
    z2, u2 = orc.nessor(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, p2, g, 2, 1.1)
    assert np.array_equal(z, z2) and np.array_equal(u, u2)


def test_orthogonal_rows_solved_by_one_sor_sweep(orc):
    # rows with disjoint supports are orthogonal: one NE-SOR sweep with omega = 1
    # solves A w = g exactly with the minimum-norm w
    m, n = 6, 18
    rp = np.arange(0, 3 * m + 1, 3, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    val = np.random.default_rng(5).standard_normal(n)
    perm = np.arange(m, dtype=np.int32)
    g = np.random.default_rng(6).standard_normal(m)
    z, y = orc.nesor(m, n, rp, ci, val, perm, g, 1, 1.0)
    A = np.zeros((m, n))
    for i in range(m):
        A[i, ci[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    assert np.allclose(A @ z, g, atol=1e-13)
    assert np.allclose(z, np.linalg.pinv(A) @ g, atol=1e-13)


def test_kaczmarz_limit_is_min_norm_solution(orc):
    # many NE-SOR sweeps with omega = 1 (Kaczmarz) from 0 converge to the
    # minimum-norm solution of a consistent system (Sec. 3.4, semiconvergence)
    lp = small_lp(m=8, n=20, density=0.4, seed=8)
    A = dense(lp)
    g = A @ np.random.default_rng(7).standard_normal(lp.n)
    perm = np.arange(lp.m, dtype=np.int32)
    z, y = orc.nesor(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, g, 3000, 1.0)
    assert np.allclose(z, np.linalg.pinv(A) @ g, atol=1e-9)


# ---------------------------------------------------------------- Krylov
def scaled_system(orc, lp, seed=0, spread=4.0):
    rng = np.random.default_rng(seed)
    d2 = np.exp(rng.uniform(-spread, spread, lp.n))
    ahat, rho = orc.scale_rows(lp.m, lp.row_ptr, lp.col_idx, lp.val, d2)
    Ah = np.zeros((lp.m, lp.n))
    for i in range(lp.m):
        Ah[i, lp.col_idx[lp.row_ptr[i]:lp.row_ptr[i + 1]]] = ahat[lp.row_ptr[i]:lp.row_ptr[i + 1]]
    return ahat, Ah


@pytest.mark.parametrize("method", [0, 1, 2])
def test_krylov_min_norm_solution(orc, method):
    lp = small_lp(m=20, n=50, density=0.2, seed=10)
    ahat, Ah = scaled_system(orc, lp)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 1)
    f = Ah @ np.random.default_rng(11).standard_normal(lp.n)
    ell = 2 if method == 2 else 1
    dw, dy, info = orc.krylov(method, lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, f, ell, 1.0,
                              1e-12, 500)
    assert info["converged"]
    assert np.allclose(dw, np.linalg.pinv(Ah) @ f, atol=1e-9 * np.linalg.norm(dw))
    # dw = A_hat^T dy: the row-space shadow recovers dy without a product
    assert np.allclose(dw, Ah.T @ dy, atol=1e-10 * np.linalg.norm(dw))


@pytest.mark.parametrize("method", [0, 1, 2])
def test_krylov_rank_deficient_no_breakdown(orc, method):
    # duplicate rows make A A^T singular; f in R(A) is still solved (Sec. 3)
    lp = gen.medium_lp(scale=0.004, seed=21)   # m = 80 with 1 dependent row
    ahat, Ah = scaled_system(orc, lp, seed=3)
    assert np.linalg.matrix_rank(Ah) < lp.m
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 2)
    f = Ah @ np.random.default_rng(12).standard_normal(lp.n)
    dw, dy, info = orc.krylov(method, lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, f,
                              3 if method < 2 else 2, 1.0, 1e-10, 2000)
    assert info["converged"] and not info["breakdown"]
    assert np.allclose(dw, np.linalg.pinv(Ah) @ f, atol=1e-7 * np.linalg.norm(dw))


def test_abgmres_residual_is_monotone(orc):
    # AB-GMRES minimises ||f - A B z|| in the 2-norm over growing Krylov
    # spaces (Sec. 3.2, right preconditioning)
    lp = small_lp(m=25, n=60, density=0.15, seed=13)
    ahat, Ah = scaled_system(orc, lp, spread=6)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 3)
    f = Ah @ np.random.default_rng(14).standard_normal(lp.n)
    dw, dy, info, hist = orc.krylov(2, lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, f, 1,
                                    1.0, 1e-12, 200, history=True)
    h = hist[np.isfinite(hist)]
    assert (np.diff(h) <= 1e-12 * h[0]).all()


def test_mrne_residual_is_monotone_in_the_preconditioner_norm(orc):
    # preconditioned MRNE is MINRES (conjugate residual) on A A^T with the SPD
    # preconditioner C^<ell>: it minimises (g, C g) over the Krylov space, so
    # the C-norm of the explicit residual never grows with the iteration count
    lp = small_lp(m=25, n=60, density=0.15, seed=13)
    ahat, Ah = scaled_system(orc, lp, spread=6)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 3)
    f = Ah @ np.random.default_rng(14).standard_normal(lp.n)
    C = np.column_stack([orc.nessor(lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, e, 1, 1.0)[0]
                         for e in np.eye(lp.m)])
    cn = []
    for k in range(1, 26):
        dw, dy, info = orc.krylov(0, lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, f, 1, 1.0,
                                  1e-300, k)
        g = f - Ah @ dw
        cn.append(g @ C @ g)
    cn = np.array(cn)
    assert (np.diff(cn) <= 1e-10 * cn[0]).all()
    assert cn[-1] < 1e-12 * cn[0]


# ---------------------------------------------------------------- Newton step
def test_w_recurrence_solves_the_newton_system(orc):
    """Eqs. (aff2)-(aff3), (cc2)-(cc3) recover the three block rows of Eq. (SE1)
    from dw without the product A^T dy (Sec. 2.2)."""
    lp = gen.tiny_lp()
    A = dense(lp)
    rng = np.random.default_rng(15)
    x = rng.uniform(0.1, 2, lp.n)
    s = rng.uniform(0.1, 2, lp.n)
    y = rng.standard_normal(lp.m)
    rp = lp.b - A @ x
    rd = lp.c - A.T @ y - s
    d2 = x / s
    d = np.sqrt(d2)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 1)
    f = lp.b + A @ (d2 * rd)
    dy, dw, info = orc.ne_solve(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, d2, f, 1, 1.0, 0,
                                1e-13, 500)
    assert info["converged"]
    assert np.allclose(dw, d * (A.T @ dy), atol=1e-10)
    ds = rd - dw / d
    dx = -d2 * ds - x
    assert np.allclose(A @ dx, rp, atol=1e-9)                    # second block row
    assert np.allclose(A.T @ dy + ds, rd, atol=1e-10)            # first block row
    assert np.allclose(s * dx + x * ds, -x * s, atol=1e-12)      # third row, r_c = -XSe
    # corrector: right-hand side -dX ds + sigma mu e, zero residual rows
    smu = 0.1
    h = (dx * ds - smu) / s
    f2 = A @ h
    dy2, dw2, info2 = orc.ne_solve(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, d2, f2, 1, 1.0,
                                   0, 1e-13, 500)
    ds2 = -dw2 / d
    dx2 = -d2 * ds2 - h
    assert np.allclose(A @ dx2, 0, atol=1e-9)
    assert np.allclose(A.T @ dy2 + ds2, 0, atol=1e-10)
    assert np.allclose(s * dx2 + x * ds2, -dx * ds + smu, atol=1e-10)


# ---------------------------------------------------------------- BA-GMRES (corrector, Sec. 3.2)
@pytest.mark.parametrize("ell,omega", [(1, 1.0), (3, 1.2)])
def test_nrsor_equals_sor_on_first_kind_normal_equations(orc, ell, omega):
    # NR-SOR for min ||A^T y - c|| is SOR on A A^T y = A c (written densely in
    # splitting form) from y = 0
    lp = small_lp(m=15, n=40, density=0.25, seed=5)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 13)
    c = np.random.default_rng(4).standard_normal(lp.n)
    y = orc.nrsor(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, c, ell, omega)
    _, y2 = splitting_sor(dense(lp), perm, dense(lp) @ c, ell, omega)
    assert np.allclose(y, y2, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("rank_deficient", [False, True])
def test_bagmres_least_squares_solution(orc, rank_deficient):
    # min ||A^T dy - r||: dw = A^T dy is the projection of r onto R(A^T), unique
    # also when A A^T is singular
    lp = gen.medium_lp(scale=0.004, seed=21) if rank_deficient else small_lp(m=20, n=50, density=0.2, seed=9)
    ahat, Ah = scaled_system(orc, lp, seed=5)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 3)
    r = np.random.default_rng(6).standard_normal(lp.n)
    dw, dy, info = orc.ls_krylov(lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, r, 2, 1.0, 1e-12, 2000)
    assert info["converged"] and not info["breakdown"]
    ref = Ah.T @ np.linalg.lstsq(Ah.T, r, rcond=None)[0]
    assert np.allclose(dw, ref, atol=1e-8 * np.linalg.norm(ref))
    assert np.allclose(dw, Ah.T @ dy, atol=1e-12 * np.linalg.norm(dw))
    # the normal equations of the first kind hold for dy
    assert np.linalg.norm(Ah @ (Ah.T @ dy) - Ah @ r) <= 1e-11 * np.linalg.norm(Ah @ r)


def test_ls_solve_gives_the_min_norm_direction_of_ne_solve(orc):
    # the corrector in least-squares form (BA-GMRES) and in w-form (MRNE) give
    # the same minimum-norm dw for f = A D r
    lp = small_lp(m=20, n=50, density=0.2, seed=12)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 4)
    rng = np.random.default_rng(7)
    d2 = np.exp(rng.uniform(-3, 3, lp.n))
    r = rng.standard_normal(lp.n)
    dy, dw, info = orc.ls_solve(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, d2, r, 2, 1.0, 1e-12, 500)
    f = dense(lp) @ (np.sqrt(d2) * r)
    dy2, dw2, info2 = orc.ne_solve(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, perm, d2, f, 1, 1.0, 0,
                                   1e-12, 500)
    assert info["converged"] and info2["converged"]
    assert np.allclose(dw, dw2, atol=1e-8 * np.linalg.norm(dw))
    assert np.allclose(dw, np.sqrt(d2) * (dense(lp).T @ dy), atol=1e-10 * np.linalg.norm(dw))


@pytest.mark.parametrize("method,ell,omega", [(0, 1, 1.4), (1, 3, 0.8), (2, 2, 1.5), (2, 1, 0.6)])
def test_krylov_solution_does_not_depend_on_the_inner_parameters(orc, method, ell, omega):
    # ell and omega only change the preconditioner; the minimum-norm solution
    # of A_hat dw = f is the same (Sec. 3: B = A^T C with C SPD / nonsingular)
    lp = small_lp(m=18, n=45, density=0.2, seed=14)
    ahat, Ah = scaled_system(orc, lp, seed=8)
    nc, color, perm, cptr = orc.color_rows(lp.m, lp.n, lp.row_ptr, lp.col_idx, 5)
    f = Ah @ np.random.default_rng(13).standard_normal(lp.n)
    dw, dy, info = orc.krylov(method, lp.m, lp.n, lp.row_ptr, lp.col_idx, ahat, perm, f, ell, omega,
                              1e-12, 2000)
    assert info["converged"]
    assert np.allclose(dw, np.linalg.pinv(Ah) @ f, atol=1e-8 * np.linalg.norm(dw))
