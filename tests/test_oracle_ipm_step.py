"""Pins of the oracle's interior-point step logic against an independent dense
computation.  CPU only.

On micro LPs the oracle is stopped after k and after k + 1 iterations
(max_ipm), so its iterate k and iterate k + 1 are both visible.  From iterate k
the test recomputes one step of Algorithm 1 in numpy with DENSE DIRECT solves
of the normal equations (no Krylov method, no inner iterations, no row
scaling), written from the paper:

  * residuals r_p = b - Ax, r_d = c - A^T y - s, mu = x^T s / n and
    Gamma = max(mu, ||r_p||/max(||b||,1), ||r_d||/max(||c||,1)) (Eq.
    errorMeasureDef, with the relative residuals of the stopping test);
  * the predictor (affine) direction of Eq. SE1 through A D^2 A^T dy = b +
    A D^2 r_d, ds = r_d - A^T dy, dx = -x - D^2 ds (Sec. 2.1-2.2);
  * step lengths of Eq. steplength with eta;
  * sigma (Sec. 2.1; the reading of the late phase: Gamma < 1e-3 gives
    min(sigma_max, 10 Gamma), otherwise min(sigma_max, (mu_af / mu)^2)), or the
    affine direction alone when both affine steps reach 1;
  * the corrector A D^2 A^T dy = A S^-1 (dX_af ds_af - sigma mu e) and the
    combined direction;
  * the centrality backtracking of Sec. 2.1: the largest tau in
    {1, beta, beta^2, ...} with min_j x_j s_j >= phi x^T s / n at the trial
    point;
  * the update x + tau alpha_p dx, y + tau alpha_d dy, s + tau alpha_d ds.

The oracle runs its Krylov solves to a tolerance of 1e-13 here, so its
directions agree with the dense ones to about 1e-10: a wrong term or factor in
any of the steps above (sigma from mu_af instead of mu, a missing square, the
corrector's centring term, the backtracking condition, the dual step length
on y) moves iterate k + 1 by orders of magnitude more.

The Krylov tolerance schedule of Sec. 4.2 is pinned on the trace of a run
with a small Krylov cap (so that some solves fail): eps_in is multiplied by
1.5 after a failed step, then by the factor of the Gamma band (1 while
log10 Gamma > 1, 0.75 while > -3, 0.375 below), then clamped to
[1e-14, 1e-4]."""
import numpy as np
import pytest

from paper_1604_07491_gb300 import gen

ETA, PHI, SIGMA_MAX, BETA = 0.9995, 1e-5, 0.208, 0.95


def micro_lp(seed, m, n):
    lp = gen.random_density_lp(m, n, 0.6, seed=seed)
    A = lp.scipy().toarray()
    if np.linalg.matrix_rank(A) < m:
        return None
    return lp


def step_len(v, dv, eta=ETA):
    neg = dv < 0
    if not neg.any():
        return 1.0
    return min(1.0, eta * float(np.min(-v[neg] / dv[neg])))


def dense_step(lp, x, y, s, phi=PHI):
    """One iteration of Algorithm 1 from (x, y, s) with dense direct solves.
    Returns (x+, y+, s+, sigma, Gamma, tau, alpha_p_af, alpha_d_af)."""
    A = lp.scipy().toarray()
    b, c = lp.b, lp.c
    n = lp.n
    rp = b - A @ x
    rd = c - A.T @ y - s
    mu = x @ s / n
    gam = max(mu, np.linalg.norm(rp) / max(np.linalg.norm(b), 1.0), np.linalg.norm(rd) / max(np.linalg.norm(c), 1.0))
    d2 = x / s
    M = (A * d2) @ A.T
    dya = np.linalg.solve(M, b + A @ (d2 * rd))
    dsa = rd - A.T @ dya
    dxa = -x - d2 * dsa
    apa, ada = step_len(x, dxa), step_len(s, dsa)
    if min(apa, ada) >= 1.0:
        sigma, dx, dy, ds = 0.0, dxa, dya, dsa
    else:
        muaf = (x + apa * dxa) @ (s + ada * dsa) / n
        sigma = min(SIGMA_MAX, 10.0 * gam) if gam < 1e-3 else min(SIGMA_MAX, (muaf / mu) ** 2)
        h = (dxa * dsa - sigma * mu) / s
        dyc = np.linalg.solve(M, A @ h)
        dsc = -A.T @ dyc
        dxc = -d2 * dsc - h
        dx, dy, ds = dxa + dxc, dya + dyc, dsa + dsc
    ap, ad = step_len(x, dx), step_len(s, ds)
    tau = 1.0
    for _ in range(60):
        pr = (x + tau * ap * dx) * (s + tau * ad * ds)
        if pr.min() >= phi * pr.sum() / n:
            break
        tau *= BETA
    return x + tau * ap * dx, y + tau * ad * dy, s + tau * ad * ds, sigma, gam, tau, apa, ada


def ew(a, b):
    """Largest element-wise error, each entry relative to max(|b_i|, rms(b))."""
    scale = np.maximum(np.abs(b), max(np.sqrt(np.mean(b * b)), 1e-300))
    return float(np.max(np.abs(a - b) / scale))


TIGHT = dict(eps_in0=1e-13, start_tol=1e-13, max_krylov=400)


@pytest.mark.parametrize("seed", [11, 12, 13, 14])
@pytest.mark.parametrize("method", [0, 2])
def test_ipm_step_matches_dense_step(orc, seed, method):
    lp = micro_lp(seed, 6, 14)
    if lp is None:
        pytest.skip("rank-deficient draw")
    kw = dict(TIGHT, method=method, inner_sweeps=3)
    checked = set()
    for k in range(0, 8):
        x, y, s, info = orc.lp_solve_lp(lp, max_ipm=k, **kw)
        if info["status_name"] == "OK":
            break
        x1, y1, s1, info1, tr = orc.lp_solve_lp(lp, max_ipm=k + 1, trace=True, **kw)
        row = dict(zip(orc.TRACE_FIELDS, tr[k]))
        xd, yd, sd, sigma, gam, tau, apa, ada = dense_step(lp, x, y, s)
        assert row["gamma"] == pytest.approx(gam, rel=1e-10)
        assert row["alpha_p_af"] == pytest.approx(apa, rel=1e-7)
        assert row["alpha_d_af"] == pytest.approx(ada, rel=1e-7)
        assert row["sigma"] == pytest.approx(sigma, rel=1e-7, abs=1e-12)
        assert row["tau"] == tau
        assert ew(x1, xd) < 1e-7 and ew(s1, sd) < 1e-7 and ew(y1, yd) < 1e-7, k
        checked.add("late" if gam < 1e-3 else "early")
        checked.add("affine" if sigma == 0.0 else "corrected")
    # the step logic was exercised in both sigma phases and with a corrector
    assert "corrected" in checked and "early" in checked


def test_backtracking_engages_and_keeps_centrality(orc):
    """With a demanding centrality bound (phi = 0.3 instead of the paper's
    1e-5, which micro LPs never hit) the backtracking shrinks some steps: the
    oracle's factor tau equals the dense step's (the first power of beta that
    meets the bound), and every accepted iterate satisfies
    min x_j s_j >= phi x^T s / n."""
    phi = 0.3
    kw = dict(TIGHT, phi=phi)
    hits = 0
    for seed in range(30, 40):
        lp = micro_lp(seed, 5, 12)
        if lp is None:
            continue
        x, y, s, info, tr = orc.lp_solve_lp(lp, trace=True, max_ipm=12, **kw)
        for k in range(info["ipm_iters"]):
            row = dict(zip(orc.TRACE_FIELDS, tr[k]))
            xk, yk, sk, _ = orc.lp_solve_lp(lp, max_ipm=k, **kw)
            xd, yd, sd, sigma, gam, tau, apa, ada = dense_step(lp, xk, yk, sk, phi=phi)
            assert row["tau"] == tau
            hits += tau < 1.0
            xk1, _, sk1, _ = orc.lp_solve_lp(lp, max_ipm=k + 1, **kw)
            pr = xk1 * sk1
            assert pr.min() >= phi * pr.sum() / lp.n * (1 - 1e-9)
    assert hits > 0, "no draw needed backtracking"


def test_eps_in_schedule_from_trace(orc):
    """Sec. 4.2: the Krylov tolerance of step k follows from the tolerance of
    step k - 1, the failure of step k - 1 and the Gamma band of iterate k.
    Three runs together take every branch: failed solves (a Krylov cap of
    m / 2 on a medium LP), all three Gamma bands, and the lower clamp (an
    initial tolerance of 1e-13)."""
    lp_med = gen.medium_lp(0.01)
    runs = [(lp_med, dict(method=0, inner_sweeps=1, max_krylov=lp_med.m // 2, max_ipm=40)),
            (gen.tiny_lp(), dict()),
            (gen.tiny_lp(), dict(eps_in0=1e-13, start_tol=1e-13))]
    seen = set()
    for lp, kw in runs:
        x, y, s, info, tr = orc.lp_solve_lp(lp, trace=True, **kw)
        rows = [dict(zip(orc.TRACE_FIELDS, r)) for r in tr]
        assert rows[0]["eps_in"] == kw.get("eps_in0", 1e-6)
        for k in range(1, len(rows)):
            e = rows[k - 1]["eps_in"]
            if rows[k - 1]["failed"]:
                e *= 1.5
                seen.add("failed")
            lg = np.log10(rows[k]["gamma"])
            if lg <= -3.0:
                e *= 0.375
                seen.add("band<=-3")
            elif lg <= 1.0:
                e *= 0.75
                seen.add("band<=1")
            else:
                seen.add("band>1")
            if e < 1e-14 or e > 1e-4:
                seen.add("clamp")
            e = min(max(e, 1e-14), 1e-4)
            assert rows[k]["eps_in"] == pytest.approx(e, rel=1e-15), (lp.name, k)
    assert seen >= {"failed", "band<=-3", "band<=1", "clamp"}, seen
