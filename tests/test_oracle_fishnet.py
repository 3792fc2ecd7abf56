"""Pins of the oracle's Algorithm 7 (fishnet casting, Section 2.5).

Checked against facts outside the oracle: the spectral norm from LAPACK's SVD
(the casting radius), Y^0 = K X^0 and the linearity of convex combinations
(with no PDHG steps the survivor's dual is K times its primal), the convex hull
of the casting points, the duality gap recomputed in numpy from its definition
(the better of two columns survives), and the column schedule of the loop.
"""
import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

RAW = dict(ruiz_iters=0, power_iters=2000)


def _lp():
    return synth.random_planted(30, 50, density=0.2, seed=4)


def _gap(lp, x, y):
    """|c^T x - (q^T y + l^T lambda^+ + u^T lambda^-)|, lambda = proj_Lambda(c - K^T y)."""
    K = lp.dense()
    v = lp.c - K.T @ y
    lf, uf = np.isfinite(lp.l), np.isfinite(lp.u)
    lam = np.where(~lf & ~uf, 0.0, v)
    lam = np.where(~lf & uf, np.minimum(v, 0.0), lam)
    lam = np.where(lf & ~uf, np.maximum(v, 0.0), lam)
    lt = np.where(lam > 0, lp.l * np.where(lam > 0, lam, 0.0), 0.0) + \
        np.where(lam < 0, lp.u * np.where(lam < 0, lam, 0.0), 0.0)
    return abs(float(lp.c @ x) - float(lp.q @ y + lt.sum()))


def test_one_point_is_the_casting_point(oracle_mod):
    """P = 1: no round runs; x0 = (||K||_2 / sqrt(n)) g, y0 = K x0."""
    lp = _lp()
    g = np.random.default_rng(1).standard_normal((lp.n, 1))
    x, y, gaps, rounds = oracle_mod.fishnet(lp, 1, 5, g, [], **RAW)
    assert rounds == 0 and gaps.shape[0] == 0
    r = np.linalg.norm(lp.dense(), 2)
    np.testing.assert_allclose(x, r / np.sqrt(lp.n) * g[:, 0], rtol=1e-9)
    np.testing.assert_allclose(y, lp.dense() @ x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_two_points_keep_the_smaller_gap(oracle_mod, seed):
    """P = 2: one round of k fixed steps, then the column with the smaller
    duality gap (recomputed here from its definition) is returned."""
    lp = _lp()
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((lp.n, 2))
    k, eta, omega = 7, 0.05, 1.3
    x, y, gaps, rounds = oracle_mod.fishnet(lp, 2, k, g, [], eta0=eta, omega0=omega, **RAW)
    assert rounds == 1
    r = np.linalg.norm(lp.dense(), 2)
    ends = []
    for p in range(2):
        xp = r / np.sqrt(lp.n) * g[:, p]
        yp = lp.dense() @ xp
        for _ in range(k):
            xp, yp = oracle_mod.pdhg_step(lp, xp, yp, eta / omega, eta * omega)
        ends.append((xp, yp, _gap(lp, xp, yp)))
    np.testing.assert_allclose(gaps[0], [ends[0][2], ends[1][2]], rtol=1e-6)
    best = 0 if ends[0][2] <= ends[1][2] else 1
    np.testing.assert_allclose(x, ends[best][0], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(y, ends[best][1], rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("P", [4, 8, 32])
def test_no_steps_stays_in_the_hull_and_dual_linear(oracle_mod, P):
    """k = 0: culls and convex repopulations only, so the survivor lies in the
    convex hull of the casting points and, as both sides use the same weights,
    its dual is K times its primal (Y^0 = K X^0)."""
    lp = _lp()
    rng = np.random.default_rng(P)
    g = rng.standard_normal((lp.n, P))
    z = rng.standard_normal(oracle_mod.fishnet_draws(P))
    x, y, _, _ = oracle_mod.fishnet(lp, P, 0, g, z, **RAW)
    pts = np.linalg.norm(lp.dense(), 2) / np.sqrt(lp.n) * g
    assert np.all(x >= pts.min(axis=1) - 1e-9) and np.all(x <= pts.max(axis=1) + 1e-9)
    np.testing.assert_allclose(y, lp.dense() @ x, rtol=1e-9, atol=1e-9)


def test_column_schedule_of_32_points(oracle_mod):
    """32 columns: culls to 16, repopulation back to 16 at odd rounds while more
    than two columns enter the round -> 32, 16, 16, 8, 8, 4, 4, 2 columns over
    8 rounds, 8^2 + 4^2 + 2^2 = 84 repopulation draws."""
    lp = _lp()
    rng = np.random.default_rng(5)
    g = rng.standard_normal((lp.n, 32))
    assert oracle_mod.fishnet_draws(32) == 84
    z = rng.standard_normal(84)
    _, _, gaps, rounds = oracle_mod.fishnet(lp, 32, 3, g, z, **RAW)
    assert rounds == 8
    assert [int(np.isfinite(r).sum()) for r in gaps] == [32, 16, 16, 8, 8, 4, 4, 2]
    with pytest.raises(ValueError):
        oracle_mod.fishnet(lp, 32, 3, g, z[:83], **RAW)
    with pytest.raises(ValueError):
        oracle_mod.fishnet(lp, 6, 3, g[:, :6], z, **RAW)


def test_warm_start_reaches_tolerance(oracle_mod):
    """The fishnet point is a valid warm start: the restarted solver from it
    reaches the tolerance (the paper reports mixed iteration effects)."""
    lp = synth.small_dense_lp()
    rng = np.random.default_rng(9)
    g = rng.standard_normal((lp.n, 32))
    z = rng.standard_normal(84)
    x0, y0, _, _ = oracle_mod.fishnet(lp, 32, 20, g, z)
    x, y, info, _ = oracle_mod.solve(lp, tol=1e-6, x0=x0, y0=y0)
    assert info["status"] == 1
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-6 * (1 + 1e-9)
