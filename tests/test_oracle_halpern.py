"""Pins of the oracle's restarted (reflected) Halpern PDHG, the variant the
Conclusion names as future work (Lu and Yang, 2024).

Each pin rests on mathematics, not on the oracle's own formulas:
- the PDHG step is firmly nonexpansive in the metric P that the oracle's
  ``pnorm2`` implements (a wrong sign of its cross term breaks that);
- on an LP whose PDHG map is affine (equality rows, free variables) the
  Halpern iterates with weights (k + 1) / (k + 2) are exactly the running means
  of the plain iterates of the reflected map (1 + rho) T - rho I;
- Halpern's O(1/k) bound on the fixed-point residual against a planted saddle
  point, which holds with projections too;
- the restarted solver reaches the planted optimum and the vertex optimum.
"""
import math

import numpy as np
import pytest

from paper_2508_16806_gb300 import synth


def _steps(lp, omega=1.0, frac=0.9):
    eta = frac / np.linalg.norm(lp.dense(), 2)
    return eta / omega, eta * omega


def _lps():
    return [synth.small_dense_lp(), synth.shuffle_sense(synth.small_dense_lp(), 3),
            synth.power_law_lp(300, 500, 2, 40, seed=4)]


@pytest.mark.parametrize("idx", range(3))
@pytest.mark.parametrize("omega", [0.3, 1.0, 3.0])
def test_step_is_firmly_nonexpansive_in_p(oracle_mod, idx, omega):
    """For tau sigma ||K||^2 < 1: ||Tz1 - Tz2||_P^2 <= <Tz1 - Tz2, z1 - z2>_P
    (inner product by polarisation of pnorm2)."""
    lp = _lps()[idx]
    tau, sigma = _steps(lp, omega)
    rng = np.random.default_rng(idx * 10 + int(omega * 10))
    for _ in range(12):
        x1, x2 = rng.normal(size=(2, lp.n)) * 3
        y1, y2 = rng.normal(size=(2, lp.m)) * 3
        t1 = oracle_mod.pdhg_step(lp, x1, y1, tau, sigma)
        t2 = oracle_mod.pdhg_step(lp, x2, y2, tau, sigma)
        a = (t1[0] - t2[0], t1[1] - t2[1])
        b = (x1 - x2, y1 - y2)

        na = oracle_mod.pnorm2(lp, a[0], a[1], tau, sigma)
        assert na > 0
        assert na <= _ip(oracle_mod, lp, a, b, tau, sigma) * (1 + 1e-12) + 1e-12


def _ip(oracle_mod, lp, a, b, tau, sigma):
    """<a, b>_P by polarisation of pnorm2."""
    p = oracle_mod.pnorm2(lp, a[0] + b[0], a[1] + b[1], tau, sigma)
    mnus = oracle_mod.pnorm2(lp, a[0] - b[0], a[1] - b[1], tau, sigma)
    return (p - mnus) / 4


@pytest.mark.parametrize("omega", [0.5, 2.0])
def test_p_is_the_metric_of_the_step(oracle_mod, omega):
    """Where no projection acts (equality rows, free variables) the step solves
    P (z - Tz) = F(Tz) with F(z) = (c - K^T y, K x - q), the monotone operator of
    the saddle problem min_x max_y c^T x - y^T (K x - q).  So for every direction
    d: <d, z - Tz>_P = <d, F(Tz)>; a wrong sign or weight in P breaks this."""
    lp = _affine_lp(11)
    Kd = lp.dense()
    tau, sigma = _steps(lp, omega)
    rng = np.random.default_rng(2)
    for _ in range(10):
        x, y = rng.normal(size=lp.n), rng.normal(size=lp.m)
        xh, yh = oracle_mod.pdhg_step(lp, x, y, tau, sigma)
        F = (lp.c - Kd.T @ yh, Kd @ xh - lp.q)
        d = (rng.normal(size=lp.n), rng.normal(size=lp.m))
        lhs = _ip(oracle_mod, lp, d, (x - xh, y - yh), tau, sigma)
        rhs = float(d[0] @ F[0] + d[1] @ F[1])
        assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-9)


def test_pnorm_is_positive_definite(oracle_mod):
    """P is positive definite exactly when tau sigma ||K||^2 < 1: random
    directions are positive at 0.99 / ||K||, and the top singular pair of K
    (x = v, y = -u, scaled) gives a negative value at 1.2 / ||K||."""
    lp = synth.small_dense_lp()
    Kd = lp.dense()
    U, S, Vt = np.linalg.svd(Kd)
    tau, sigma = _steps(lp, 1.0, 0.99)
    rng = np.random.default_rng(1)
    for _ in range(20):
        assert oracle_mod.pnorm2(lp, rng.normal(size=lp.n), rng.normal(size=lp.m), tau, sigma) > 0
    tau, sigma = _steps(lp, 1.0, 1.2)
    # K v = s u with s = ||K||: the value is 2 - 2 s sqrt(tau sigma) = 2 - 2.4
    val = oracle_mod.pnorm2(lp, math.sqrt(tau) * Vt[0], -math.sqrt(sigma) * U[:, 0], tau, sigma)
    assert val == pytest.approx(2 - 2 * 1.2, rel=1e-9)


def _affine_lp(seed):
    """Equality rows and free variables: T is affine (no projection acts)."""
    rng = np.random.default_rng(seed)
    m, n = 12, 20
    K = rng.normal(size=(m, n)) * (rng.random((m, n)) < 0.5)
    return synth.from_dense(K, np.zeros(m, int), rng.normal(size=n), rng.normal(size=m),
                            np.full(n, -np.inf), np.full(n, np.inf), name="affine")


@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
def test_affine_halpern_is_running_mean_of_reflected_iterates(oracle_mod, rho):
    """For affine S = (1 + rho) T - rho I, Halpern with weights (k+1)/(k+2)
    and anchor z0 gives z_k = (1 / (k + 1)) sum_{j <= k} S^j z0 (induction on k)."""
    lp = _affine_lp(3)
    tau, sigma = _steps(lp, 1.7)
    rng = np.random.default_rng(5)
    x0, y0 = rng.normal(size=lp.n), rng.normal(size=lp.m)
    x, y = x0.copy(), y0.copy()
    px, py = x0.copy(), y0.copy()          # Picard iterates S^j z0
    sx, sy = x0.copy(), y0.copy()          # their sums
    for k in range(60):
        _, (x, y), _ = oracle_mod.halpern_step(lp, x, y, x0, y0, tau, sigma, k, rho)
        tx, ty = oracle_mod.pdhg_step(lp, px, py, tau, sigma)
        px, py = (1 + rho) * tx - rho * px, (1 + rho) * ty - rho * py
        sx += px
        sy += py
        scale = 1 + np.max(np.abs(sx / (k + 2)))
        np.testing.assert_allclose(x, sx / (k + 2), rtol=0, atol=1e-11 * scale)
        np.testing.assert_allclose(y, sy / (k + 2), rtol=0, atol=1e-11 * scale)


@pytest.mark.parametrize("rho", [0.0, 1.0])
@pytest.mark.parametrize("idx", range(3))
def test_halpern_residual_bound(oracle_mod, idx, rho):
    """Halpern on the nonexpansive S = (1 + rho) T - rho I: for every k,
    ||z_k - T z_k||_P = ||z_k - S z_k||_P / (1 + rho) <= 2 ||z0 - z*||_P / ((1 + rho)(k + 1)),
    z* the planted saddle point (a fixed point of T)."""
    lp = _lps()[idx]
    tau, sigma = _steps(lp, 1.0)
    x0, y0 = np.clip(np.zeros(lp.n), lp.l, lp.u), np.zeros(lp.m)
    d0 = math.sqrt(oracle_mod.pnorm2(lp, x0 - lp.x_star, y0 - lp.y_star, tau, sigma))
    x, y = x0, y0
    worst = 0.0
    for k in range(400):
        _, (xn, yn), r = oracle_mod.halpern_step(lp, x, y, x0, y0, tau, sigma, k, rho)
        bound = 2 * d0 / ((1 + rho) * (k + 1))
        assert r <= bound * (1 + 1e-9) + 1e-12, (k, r, bound)
        worst = max(worst, r / bound)
        x, y = xn, yn
    assert worst > 1e-3      # the bound is not vacuous on these problems


def test_residual_is_zero_at_saddle_point(oracle_mod):
    lp = synth.small_dense_lp()
    tau, sigma = _steps(lp, 1.0)
    (xh, yh), (xn, yn), r = oracle_mod.halpern_step(lp, lp.x_star, lp.y_star, lp.x_star,
                                                    lp.y_star, tau, sigma, 5, 1.0)
    assert r < 1e-10
    np.testing.assert_allclose(xn, lp.x_star, atol=1e-12)
    np.testing.assert_allclose(yn, lp.y_star, atol=1e-12)


@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_restarted_halpern_reaches_planted_optimum(oracle_mod, rho):
    for lp in (synth.small_dense_lp(), synth.shuffle_sense(synth.small_dense_lp(), 3)):
        x, y, info, trace = oracle_mod.solve(lp, tol=1e-8, max_iters=300000, halpern=1,
                                             reflect=rho)
        assert info["status"] == 1
        assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-6)
        k = oracle_mod.kkt(lp, x, y)
        assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-8
        assert info["restarts"] == sum(int(t["restart"]) for t in trace)
        assert all(t["cand_is_avg"] == 1.0 and t["kkt_cand"] == t["kkt_avg"] for t in trace)
        assert info["attempts"] == info["iters"]


@pytest.mark.parametrize("seed", range(4))
def test_restarted_halpern_matches_vertex_optimum(oracle_mod, seed):
    """LPs with costs that are not planted, solved exactly by enumerating
    vertices (n = 6; the brute force of the restarted PDHG pin)."""
    from tests.test_oracle_pins import _vertex_enumeration
    rng = np.random.default_rng(200 + seed)
    m, n = 4, 6
    K = rng.normal(size=(m, n))
    sense = np.array([1, 1, 1, 0]) if seed % 2 else np.array([1, 0, 1, 1])
    l = rng.uniform(-1, 0, n)
    u = rng.uniform(0.5, 2, n)
    q = K @ rng.uniform(l, u) - np.where(sense == 1, rng.uniform(0, 1, m), 0.0)
    lp = synth.from_dense(K, sense, rng.normal(size=n), q, l, u)
    f_exact = _vertex_enumeration(lp)
    x, y, info, _ = oracle_mod.solve(lp, tol=1e-9, max_iters=500000, halpern=1)
    assert info["status"] == 1
    assert float(lp.c @ x) == pytest.approx(f_exact, rel=1e-6, abs=1e-7)


@pytest.mark.parametrize("check_every", [1, 64])
def test_halpern_restart_records_follow_the_criteria(oracle_mod, check_every):
    """Replay of the restart decisions from the logged residuals: each check's
    restart flag equals the three criteria (beta 0.2 / 0.8 / 0.36) on the
    residual r of the iteration just taken, r0 of the epoch's first iteration and
    r at the epoch's previous check; with a check after every iteration, r0 of
    the first record of an epoch is that record's own r."""
    lp = synth.small_dense_lp()
    tol = 1e-8
    _, _, info, trace = oracle_mod.solve(lp, tol=tol, max_iters=300000, halpern=1,
                                         check_every=check_every)
    assert info["status"] == 1
    prev = math.inf
    epoch_start = 0
    for j, t in enumerate(trace[1:], start=1):
        converged = max(t["rel_gap"], t["rel_pres"], t["rel_dres"]) <= tol
        r, r0 = t["fpr"], t["fpr0"]
        if check_every == 1 and t["k"] == epoch_start + 1:
            assert r0 == r
        expect = (not converged) and (r <= 0.2 * r0 or (r <= 0.8 * r0 and r > prev)
                                      or (t["k"] - epoch_start) > 0.36 * t["k"])
        assert bool(t["restart"]) == expect, (j, t)
        if t["restart"]:
            prev, epoch_start = math.inf, t["k"]
        else:
            prev = r
    assert info["restarts"] == sum(int(t["restart"]) for t in trace) > 0
