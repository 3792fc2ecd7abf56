"""Pins of the oracle's Algorithm 6 (infeasibility detection, Section 2.4.5).

Each pin rests on something other than the oracle itself: Farkas certificates
worked out by hand for two-variable problems (closed-form normalised terms),
scale invariance of a direction, and the infeasible / unbounded status that
scipy's HiGHS gives the same LP.
"""
import math

import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

INF = np.inf

# x in [0, 1]^2, x1 + x2 >= 3, x1 - x2 >= 0: no point satisfies x1 + x2 >= 3.
P_HAND = synth.from_dense([[1, 1], [1, -1]], [1, 1], [0, 0], [3, 0], [0, 0], [1, 1], name="P2")
# min -x1  s.t.  x1 - x2 = 0, x1 + x2 >= 1, x >= 0: x = (t, t) is feasible for
# every t >= 1/2 and the objective -t is unbounded below.
D_HAND = synth.from_dense([[1, -1], [1, 1]], [0, 1], [-1, 0], [0, 1], [0, 0], [INF, INF],
                          name="D2")


def test_primal_certificate_by_hand(oracle_mod):
    """Farkas: w = (1, 0) on the rows, lambda = c - K^T w = (-1, -1) as the
    dual direction; K^T w + lambda = 0, w >= 0 and
    q^T w + l^T lambda^+ + u^T lambda^- = 3 - 1 - 1 = 1 > 0.  Normalised by
    ||(w, lambda)|| = sqrt(3): psi = 1 / sqrt(3)."""
    st, t = oracle_mod.infeasibility(P_HAND, np.zeros(2), [1.0, 0.0], [-1.0, -1.0], 1e-6)
    assert st == 2
    assert t["psi"] == pytest.approx(1.0 / math.sqrt(3.0), rel=1e-14)
    assert t["ktdy_res"] == 0.0 and t["dy_ineq_min"] == 0.0


def test_dual_certificate_by_hand(oracle_mod):
    """v = (1, 1): A v = 0, G v = 2 >= 0, c^T v = -1 < 0, v in R+^2.
    Normalised: c^T v / ||v|| = -1 / sqrt(2), G v / ||v|| = sqrt(2)."""
    st, t = oracle_mod.infeasibility(D_HAND, [1.0, 1.0], np.zeros(2), np.zeros(2), 1e-6)
    assert st == 3
    assert t["cdx"] == pytest.approx(-1.0 / math.sqrt(2.0), rel=1e-14)
    assert t["gdx_min"] == pytest.approx(math.sqrt(2.0), rel=1e-14)
    assert t["adx"] == 0.0 and t["v_dist"] == 0.0


def test_non_certificates_rejected(oracle_mod):
    """Directions that fail one condition each."""
    # w = (0, 1): lambda = (-1, 1); psi = 0 + l2 * 1 + u1 * (-1) = -1 < 0
    st, t = oracle_mod.infeasibility(P_HAND, np.zeros(2), [0.0, 1.0], [-1.0, 1.0], 1e-6)
    assert st == 0 and t["psi"] == pytest.approx(-1.0 / math.sqrt(3.0), rel=1e-14)
    # w = (-1, 0) violates w_ineq >= 0
    st, _ = oracle_mod.infeasibility(P_HAND, np.zeros(2), [-1.0, 0.0], [1.0, 1.0], 1e-6)
    assert st == 0
    # residual K^T w + lambda != 0
    st, t = oracle_mod.infeasibility(P_HAND, np.zeros(2), [1.0, 0.0], [-1.0, 0.0], 1e-6)
    assert st == 0 and t["ktdy_res"] == pytest.approx(1.0 / math.sqrt(2.0), rel=1e-14)
    # v = (1, 0): A v = 1 != 0
    st, _ = oracle_mod.infeasibility(D_HAND, [1.0, 0.0], np.zeros(2), np.zeros(2), 1e-6)
    assert st == 0
    # v = (-1, -1): c^T v = +1 and v leaves R+^2
    st, t = oracle_mod.infeasibility(D_HAND, [-1.0, -1.0], np.zeros(2), np.zeros(2), 1e-6)
    assert st == 0 and t["v_dist"] == pytest.approx(1.0 / math.sqrt(2.0), rel=1e-14)
    # zero differences are no certificate
    st, _ = oracle_mod.infeasibility(D_HAND, np.zeros(2), np.zeros(2), np.zeros(2), 1e-6)
    assert st == 0


@pytest.mark.parametrize("scale", [1e-9, 1e-3, 1e3, 1e9])
def test_certificates_scale_invariant(oracle_mod, scale):
    """A certificate is a direction: its length does not change the verdict."""
    st, _ = oracle_mod.infeasibility(P_HAND, np.zeros(2), [scale, 0.0], [-scale, -scale], 1e-6)
    assert st == 2
    st, _ = oracle_mod.infeasibility(D_HAND, [scale, scale], np.zeros(2), np.zeros(2), 1e-6)
    assert st == 3


def _highs_status(lp):
    """scipy linprog (HiGHS) status: 0 optimal, 2 infeasible, 3 unbounded."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    K = lp.dense()
    ge = lp.sense.astype(bool)
    eq = ~ge
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
              for a, b in zip(lp.l, lp.u)]
    r = scipy_opt.linprog(lp.c, A_ub=-K[ge] if ge.any() else None,
                          b_ub=-lp.q[ge] if ge.any() else None,
                          A_eq=K[eq] if eq.any() else None, b_eq=lp.q[eq] if eq.any() else None,
                          bounds=bounds, method="highs")
    return r.status


def _cases():
    base = synth.small_dense_lp()
    return [
        ("P2", P_HAND, 2),
        ("D2", D_HAND, 3),
        ("contradiction", synth.contradictory_rows_lp(base), 2),
        ("contradiction_gap0.1", synth.contradictory_rows_lp(base, seed=5, gap=0.1), 2),
        ("unbounded_col", synth.unbounded_column_lp(base), 3),
        ("unbounded_col9", synth.unbounded_column_lp(base, seed=9), 3),
        ("feasible", base, 1),
    ]


@pytest.mark.parametrize("adaptive", [1, 0])
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_solver_status_matches_highs(oracle_mod, case, adaptive):
    """The restarted solver with Algorithm 6 at every check reports what HiGHS
    finds: primal infeasible (2), dual infeasible = unbounded (3), or a
    feasible problem solved to tolerance without a false detection (1)."""
    name, lp, want = case
    highs = _highs_status(lp)
    assert highs == {1: 0, 2: 2, 3: 3}[want]
    _, _, info, _ = oracle_mod.solve(lp, tol=1e-8, max_iters=60000, infeas_detect=1,
                                     infeas_tol=1e-6, adaptive_step=adaptive)
    assert info["status"] == want, (name, info)


def test_detection_off_runs_to_limit(oracle_mod):
    """With Algorithm 6 off an infeasible problem ends at the iteration limit."""
    lp = synth.contradictory_rows_lp(synth.small_dense_lp())
    _, _, info, _ = oracle_mod.solve(lp, tol=1e-8, max_iters=3000, infeas_detect=0)
    assert info["status"] == 4 and info["iters"] == 3000
