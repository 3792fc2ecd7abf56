"""Pins of the oracle's Algorithm 4 (primal weight update) and Algorithm 5
(adaptive step size), and planted-mistake tests that show the pins bite.

Algorithm 4 and Algorithm 5 are decision rules: nothing outside the paper fixes
what they compute, so they are pinned by hand-worked values
(tests/golden/step_rules_hand.json, each with its arithmetic) at two levels:
the rules as functions of their scalar inputs, and their call sites inside the
solver (which distances, which k, which eta reach the rule), on a one-row LP
whose first steps can be worked by hand.  The invariant the paper states for
Algorithm 5 (an attempt is accepted exactly when eta <= eta_bar, and eta' is
the next attempt's step) is checked on every attempt of full solves.

The planted-mistake tests compile copies of the oracle with one plausible
misreading each (distances swapped, no smoothing, exponents exchanged, 0-based
k, ...) and check that at least one pin fails for every copy.
"""
import json
import math
import os
import subprocess

import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "step_rules_hand.json")
ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "pdhg_oracle.c")


def _gold():
    with open(GOLD) as f:
        return json.load(f)


def _num(v):
    return math.inf if v == "inf" else float(v)


def _lp(d, q=None):
    s = d["solve_lp"]
    return synth.from_dense(s["K"], s["sense"], s["c"], q if q is not None else s["q"], s["l"],
                            s["u"])


# ----------------------------------------------------------------- the pins
# Plain functions (raise AssertionError) so that the planted-mistake test can
# run them against broken copies of the oracle.

def pin_step_rule_values(orc):
    for case in _gold()["step_rule"]:
        acc, eb, en = orc.step_rule(case["eta"], case["omega"], case["dx2"], case["dy2"],
                                    case["inter"], case["accepted"])
        assert acc == case["accept"], case["_work"]
        want_eb = _num(case["eta_bar"])
        if math.isinf(want_eb):
            assert math.isinf(eb), case["_work"]
        else:
            assert eb == pytest.approx(want_eb, rel=1e-14), case["_work"]
        assert en == pytest.approx(case["eta_next"], rel=1e-13), case["_work"]


def pin_primal_weight_values(orc):
    for case in _gold()["primal_weight"]:
        got = orc.primal_weight(case["omega"], case["dx"], case["dy"], 1e-6)
        assert got == pytest.approx(case["out"], rel=1e-14), case["_work"]


def pin_adaptive_retry_then_accept(orc):
    d = _gold()
    f = d["adaptive_retry_then_accept"]
    x, y, info, _, att = orc.solve_logged(_lp(d), **f["opts"])
    assert len(att) == len(f["attempts"]) == info["attempts"], (att, info)
    for got, want in zip(att, f["attempts"]):
        assert got["k"] == 0.0
        assert got["accept"] == want["accept"], f["_work"]
        for key in ("eta", "eta_bar", "eta_next"):
            assert got[key] == pytest.approx(want[key], rel=1e-12), (key, f["_work"])
    assert info["iters"] == 1
    assert info["eta"] == pytest.approx(f["eta_after"], rel=1e-12)
    np.testing.assert_allclose(x, f["x"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(y, f["y"], rtol=1e-12, atol=1e-15)


def pin_restart_primal_weight(orc):
    d = _gold()
    for case in d["restart_weight"]:
        _, _, info, tr = orc.solve(_lp(d, case["q"]), **case["opts"])
        assert len(tr) == 2 and tr[1]["restart"] == 1.0, (tr, case["_work"])
        assert tr[1]["omega"] == pytest.approx(case["omega_after"], rel=1e-13), case["_work"]
        assert info["omega"] == pytest.approx(case["omega_after"], rel=1e-13)


def pin_eta_invariant(orc, lp, max_iters=600, **kw):
    """Every attempt: accepted exactly when eta <= eta_bar; eta' of an attempt
    is the step of the next attempt; k counts accepted attempts."""
    _, _, info, _, att = orc.solve_logged(lp, tol=1e-9, max_iters=max_iters, **kw)
    assert len(att) == info["attempts"] > 0
    accepted = 0
    for i, a in enumerate(att):
        assert a["k"] == accepted
        assert (a["eta"] <= a["eta_bar"]) == bool(a["accept"]), (i, a)
        assert a["eta_next"] > 0.0
        if i + 1 < len(att):
            assert att[i + 1]["eta"] == a["eta_next"], (i, a, att[i + 1])
        accepted += int(a["accept"])
    assert accepted == info["iters"]
    return att


def pin_first_attempt_terms(orc):
    """The first attempt's three terms and eta_bar against a numpy evaluation of
    one step from the start point (no scaling, so the scaled problem is the LP)."""
    lp = synth.small_dense_lp()
    _, _, info, _, att = orc.solve_logged(lp, ruiz_iters=0, max_iters=1, tol=0.0,
                                          infeas_detect=0)
    a = att[0]
    K = np.zeros((lp.m, lp.n))
    for i in range(lp.m):
        K[i, lp.col_idx[lp.row_ptr[i]:lp.row_ptr[i + 1]]] = lp.vals[lp.row_ptr[i]:lp.row_ptr[i + 1]]
    x0 = np.clip(np.zeros(lp.n), lp.l, lp.u)
    y0 = np.zeros(lp.m)
    tau, sigma = a["eta"] / a["omega"], a["eta"] * a["omega"]
    x1 = np.clip(x0 - tau * (lp.c - K.T @ y0), lp.l, lp.u)
    y1 = y0 + sigma * (lp.q - K @ (2 * x1 - x0))
    y1[lp.sense == 1] = np.maximum(y1[lp.sense == 1], 0.0)
    dx, dy = x1 - x0, y1 - y0
    inter = dy @ (K @ dx)
    assert a["dx2"] == pytest.approx(dx @ dx, rel=1e-12)
    assert a["dy2"] == pytest.approx(dy @ dy, rel=1e-12)
    assert a["inter"] == pytest.approx(inter, rel=1e-10)
    eb = (a["omega"] * (dx @ dx) + (dy @ dy) / a["omega"]) / (2 * abs(inter))
    assert a["eta_bar"] == pytest.approx(eb, rel=1e-10)


def run_all_pins(orc):
    """Runs every pin; returns the names of those that fail."""
    failed = []
    checks = [
        ("step_rule_values", lambda: pin_step_rule_values(orc)),
        ("primal_weight_values", lambda: pin_primal_weight_values(orc)),
        ("adaptive_retry_then_accept", lambda: pin_adaptive_retry_then_accept(orc)),
        ("restart_primal_weight", lambda: pin_restart_primal_weight(orc)),
        ("eta_invariant", lambda: pin_eta_invariant(orc, synth.small_dense_lp(), 300)),
        ("first_attempt_terms", lambda: pin_first_attempt_terms(orc)),
    ]
    for name, fn in checks:
        try:
            fn()
        except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError):
            failed.append(name)
    return failed


# ----------------------------------------------------------------- tests

def test_step_rule_hand_values(oracle_mod):
    """Algorithm 5 as a function: eta_bar, eta' and the outcome on hand-worked
    inputs (a rejection, an infinite eta_bar, acceptance at equality, two k)."""
    pin_step_rule_values(oracle_mod)


def test_primal_weight_hand_values(oracle_mod):
    """Algorithm 4 as a function, including the skips at eps_zero."""
    pin_primal_weight_values(oracle_mod)


def test_adaptive_retry_then_accept_in_solve(oracle_mod):
    """Algorithm 5 at its call site: a rejected attempt, the retry with eta',
    acceptance, and the eta carried to the next iteration."""
    pin_adaptive_retry_then_accept(oracle_mod)


def test_restart_primal_weight_in_solve(oracle_mod):
    """Algorithm 4 at its call site: the anchors' distances reach the rule in
    the right roles at the first restart (and the skips when one is zero)."""
    pin_restart_primal_weight(oracle_mod)


@pytest.mark.parametrize("name,eta_scale", [("small_dense", 0.9), ("small_dense", 10.0),
                                             ("ragged", 0.9), ("infeasible_rows", 0.9)])
def test_accepted_eta_never_exceeds_eta_bar(oracle_mod, name, eta_scale):
    """The invariant Algorithm 5 states: every accepted step has eta <= eta_bar,
    every rejected one eta > eta_bar, and each eta' is the next step tried, over
    whole solves with restarts (Ruiz scaling on).  A start at 10 / ||K~|| and the
    ragged LP make Algorithm 5 reject some attempts."""
    lp = {"small_dense": synth.small_dense_lp,
          "ragged": synth.ragged_lp,
          "infeasible_rows": lambda: synth.contradictory_rows_lp(synth.small_dense_lp())}[name]()
    att = pin_eta_invariant(oracle_mod, lp, 1500, eta_scale=eta_scale)
    if name == "ragged" or eta_scale > 1:
        assert any(not a["accept"] for a in att)


def test_first_attempt_terms_against_numpy(oracle_mod):
    pin_first_attempt_terms(oracle_mod)


# ----------------------------------------------------------------- planted mistakes

MUTANTS = {
    "alg4_distances_swapped": [("exp(0.5 * log(dy / dx) + 0.5 * log(omega))",
                                "exp(0.5 * log(dx / dy) + 0.5 * log(omega))")],
    "alg4_no_smoothing": [("exp(0.5 * log(dy / dx) + 0.5 * log(omega))", "dy / dx")],
    "alg4_call_site_swapped": [("omega = orc_primal_weight(omega, ddx, ddy, o->eps_zero);",
                                "omega = orc_primal_weight(omega, ddy, ddx, o->eps_zero);")],
    "alg5_exponents_exchanged": [("pow(kp1, -0.3)", "pow(kp1, -@6)"),
                                 ("pow(kp1, -0.6)", "pow(kp1, -0.3)"),
                                 ("pow(kp1, -@6)", "pow(kp1, -0.6)")],
    "alg5_zero_based_k": [("(double)accepted + 2.0", "(double)accepted + 1.0")],
    "alg5_weights_swapped": [("omega * dx2 + dy2 / omega", "dx2 / omega + omega * dy2")],
    "alg5_strict_acceptance": [("return eta <= eta_bar;", "return eta < eta_bar;")],
    "alg5_eta_kept_after_accept": [("eta = eta_next;            /* eta' is used",
                                    "if (!accept) eta = eta_next; /* eta' is used")],
    "alg5_k_counts_attempts": [("inter, k, &eta_bar, &eta_next)",
                                "inter, attempts, &eta_bar, &eta_next)")],
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(oracle_mod, tmp_path, mutant):
    """A copy of the oracle with one misreading of Algorithm 4 or 5 must fail at
    least one of the pins above (the unmodified oracle passes them all)."""
    src = open(ORACLE_SRC).read()
    for old, new in MUTANTS[mutant]:
        assert old in src, (mutant, old)
        src = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    c.write_text(src)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(c),
                           "-lm"])
    with oracle_mod.use_library(str(so)):
        with np.errstate(all="ignore"):
            failed = run_all_pins(oracle_mod)
    assert failed, f"{mutant}: every pin passed"


def test_unmodified_oracle_passes_all_pins(oracle_mod):
    assert run_all_pins(oracle_mod) == []


def test_replay_of_own_log_reproduces_the_run(oracle_mod):
    """The replay mode (used to extend GPU parity of the adaptive path): taking
    the step sizes and outcomes of a run's own attempt log reproduces that run
    bit for bit, and the replayed run's own eta_bar and eta' equal the logged ones."""
    lp = synth.ragged_lp()
    x, y, info, tr, att = oracle_mod.solve_logged(lp, tol=1e-9, max_iters=700)
    rows = np.array([[a[f] for f in oracle_mod.ATTEMPT_FIELDS] for a in att])
    x2, y2, i2, tr2, att2 = oracle_mod.solve_logged(lp, tol=1e-9, max_iters=700, replay=rows)
    np.testing.assert_array_equal(x, x2)
    np.testing.assert_array_equal(y, y2)
    assert att == att2 and tr == tr2 and i2["attempts"] == info["attempts"]


def test_replay_of_own_checks_reproduces_the_run(oracle_mod):
    """Replaying a run's own check decisions as well (restart, candidate) still
    reproduces it bit for bit; its own decisions are logged beside the replayed
    ones and agree with them, and the logged KKT values the restart criteria
    compared give the logged decision (Section 2.4.2: sufficient decay, necessary
    decay without progress, or the artificial restart, which the epoch length
    decides and which is therefore left out here)."""
    lp = synth.ragged_lp()
    x, y, info, tr, att = oracle_mod.solve_logged(lp, tol=1e-9, max_iters=700, check_every=32)
    rows = np.array([[a[f] for f in oracle_mod.ATTEMPT_FIELDS] for a in att])
    chk = np.array([[t["restart"], t["cand_is_avg"]] for t in tr])
    x2, y2, i2, tr2, att2 = oracle_mod.solve_logged(lp, tol=1e-9, max_iters=700, check_every=32,
                                                    replay=rows, replay_checks=chk)
    np.testing.assert_array_equal(x, x2)
    np.testing.assert_array_equal(y, y2)
    assert att == att2 and tr == tr2
    assert info["restarts"] > 0
    d = oracle_mod.DEFAULTS
    for t in tr[1:]:
        assert t["own_restart"] == t["restart"] and t["own_cand_is_avg"] == t["cand_is_avg"]
        c = t["kkt_cand"]
        crit1 = c <= d["beta_sufficient"] * t["kkt_anchor"]
        crit2 = c <= d["beta_necessary"] * t["kkt_anchor"] and c > t["kkt_prev"]
        if crit1 or crit2:
            assert t["restart"] == 1.0


def test_replayed_check_decision_is_followed(oracle_mod):
    """A replayed restart decision that differs from the run's own is taken (the
    trace shows the replayed one, the own one beside it) and changes the run."""
    lp = synth.ragged_lp()
    x, y, info, tr, _ = oracle_mod.solve_logged(lp, tol=1e-9, max_iters=400, check_every=32)
    chk = np.array([[t["restart"], t["cand_is_avg"]] for t in tr])
    c = next(i for i in range(1, len(tr)) if tr[i]["restart"] == 0.0)
    chk[c, 0] = 1.0
    x2, y2, i2, tr2, _ = oracle_mod.solve_logged(lp, tol=1e-9, max_iters=400, check_every=32,
                                                 replay_checks=chk)
    assert tr2[c]["restart"] == 1.0 and tr2[c]["own_restart"] == 0.0
    assert i2["restarts"] >= info["restarts"] + 1 or not np.array_equal(x, x2)
