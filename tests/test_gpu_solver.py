"""GPU parity of the CUDA solver against the FP64 CPU oracle, through the C ABI.

Tolerances: with the fixed step the FP64 path tracks the oracle's iterates to
<= 1e-10 relative (2-norm) over the first 1000 iterations, makes the same
restart decisions and reaches the same objective to <= 1e-6 relative; with the
adaptive step (Algorithm 5), whose map amplifies rounding differences
exponentially, tracking is checked over the first check period and the solve is
checked at the tolerance by the oracle's own KKT evaluation.
"""
import math

import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16806_gb300 import lp as L
    L.load()
    return L


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problems():
    return {
        "lp200x400": synth.small_dense_lp(),
        "ragged": synth.ragged_lp(),
        "shuffled": synth.shuffle_sense(synth.small_dense_lp(), 3),
        "powerlaw": synth.power_law_lp(4000, 8000, 4, 600, seed=11),
    }


PROBS = _problems()


# ---------------------------------------------------------------- one step

@pytest.mark.parametrize("name", ["lp200x400", "ragged", "powerlaw"])
def test_single_fixed_step_matches_oracle_step(L, oracle_mod, name):
    """One PDHG step (no scaling) from the start point equals the oracle's
    Algorithm 1 step: exercises both SpMVs (every row-length path) and the
    fused projections."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    eta, omega = 0.37, 1.3
    x, y, info, _ = prob.solve(tol=0.0, max_iters=1, check_every=1, ruiz_iters=0,
                               adaptive_step=0, restarts=0, primal_weight_update=0,
                               eta0=eta, omega0=omega)
    assert info["status"] == L.LP_ITERATION_LIMIT and info["iters"] == 1
    x0, y0 = oracle_mod.start_point(lp)
    xo, yo = oracle_mod.pdhg_step(lp, x0, y0, eta / omega, eta * omega)
    assert rel(x, xo) < 1e-13
    assert rel(y, yo) < 1e-13


# ---------------------------------------------------------------- iterate tracking

def _check_trace(tr, tro):
    """Every check record agrees.  The candidate choice is compared only when
    the two KKT values are not tied to rounding (a one-iterate average equals
    the iterate up to one rounding, so either choice is correct there)."""
    assert len(tr) == len(tro)
    for a, b in zip(tr, tro):
        assert a["k"] == b["k"] and a["attempts"] == b["attempts"]
        assert a["restart"] == b["restart"]
        tie = math.isfinite(b["kkt_avg"]) and abs(b["kkt_cur"] - b["kkt_avg"]) <= 1e-9 * b["kkt_cur"]
        if not tie:
            assert a["cand_is_avg"] == b["cand_is_avg"]
        for f in ("omega", "eta"):
            assert a[f] == pytest.approx(b[f], rel=1e-10), (f, a[f], b[f])
        # KKT terms near convergence are differences of O(|objective|) numbers
        # (gap) and of O(|q|) numbers (residuals): summation order changes them by
        # ~1e-16 of those scales, so the absolute floor is 1e-10
        for f in ("kkt_cur", "kkt_cand", "rel_gap", "rel_pres", "rel_dres"):
            assert a[f] == pytest.approx(b[f], rel=1e-8, abs=1e-10), (f, a[f], b[f])


FIXED = dict(adaptive_step=0)


@pytest.mark.parametrize("name", ["lp200x400", "ragged", "shuffled", "powerlaw"])
@pytest.mark.parametrize("iters", [1, 10, 100, 1000])
def test_fp64_iterates_track_oracle(L, oracle_mod, name, iters):
    """Restarted FP64 PDHG with Ruiz scaling, primal-weight updates and the
    fixed step eta = 0.9 / ||K~||: the candidate after `iters` iterations
    matches the oracle's to 1e-10 relative, and every check record (restart
    flag, candidate choice, omega, eta, KKT values) agrees."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    x, y, info, tr = prob.solve(tol=1e-13, max_iters=iters, trace_cap=4096, **FIXED)
    xo, yo, io, tro = oracle_mod.solve(lp, tol=1e-13, max_iters=iters, trace_cap=4096, **FIXED)
    assert info["status"] == io["status"] == L.LP_ITERATION_LIMIT
    assert info["iters"] == io["iters"] == iters
    assert info["restarts"] == io["restarts"]
    assert rel(x, xo) <= 1e-10, rel(x, xo)
    assert rel(y, yo) <= 1e-10, rel(y, yo)
    assert info["norm_K"] == pytest.approx(io["norm_K"], rel=1e-12)
    _check_trace(tr, tro)


@pytest.mark.parametrize("name", ["lp200x400", "ragged", "shuffled", "powerlaw"])
@pytest.mark.parametrize("iters", [1, 10, 32])
def test_fp64_adaptive_iterates_track_oracle(L, oracle_mod, name, iters):
    """With Algorithm 5 the map amplifies rounding differences exponentially
    (the oracle itself departs from its own run by 1e-3 after ~300 iterations
    when eta_0 moves by 1e-15, see test_adaptive_step_amplifies_rounding), so
    iterate tracking at 1e-10 is checked over the first 32 iterations, with a
    restart check every 16."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    x, y, info, tr = prob.solve(tol=1e-13, max_iters=iters, trace_cap=64, check_every=16)
    xo, yo, io, tro = oracle_mod.solve(lp, tol=1e-13, max_iters=iters, trace_cap=64,
                                       check_every=16)
    assert info["iters"] == io["iters"] == iters
    assert info["attempts"] == io["attempts"]
    assert rel(x, xo) <= 1e-10, rel(x, xo)
    assert rel(y, yo) <= 1e-10, rel(y, yo)
    _check_trace(tr, tro)


def _replay(oracle_mod, lp, rows, checks, y0=None):
    x0 = None if y0 is None else oracle_mod.start_point(lp)[0]
    return oracle_mod.solve_logged(lp, tol=1e-13, max_iters=1000, trace_cap=4096, replay=rows,
                                   replay_checks=checks, x0=x0, y0=y0)


@pytest.mark.parametrize("name", ["lp200x400", "ragged", "shuffled", "powerlaw"])
def test_fp64_adaptive_replay_1000_iterations(L, oracle_mod, name):
    """Parity of the adaptive path (Algorithm 5) over 1000 iterations by replay.

    The oracle takes the GPU run's discrete decisions (step sizes and accept /
    reject outcomes from its attempt log, restart and candidate choices from its
    trace) and computes everything else itself.  A replayed schedule can still
    amplify rounding differences where it accepts steps beyond 1/||K~||: the
    oracle replaying the same schedule from a start moved by 1e-12 (the order of
    the rounding differences that different summation orders accumulate over a
    few hundred steps) departs from its own replay, on the ragged and power-law
    LPs by more than 1e-6 in an attempt's terms after 120-190 attempts.  Up to that onset of the oracle's own divergence
    every quantity the GPU reports agrees with the oracle's replay within the
    rounding level (derived below) plus ten times the gap between the oracle's
    two replays, and every GPU decision is the oracle's own except where the
    oracle's quantities tie at that level.  Where no onset occurs within the
    1000 iterations, the final iterates agree to 1e-10 as well."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    x, y, info, tr = prob.solve(tol=1e-13, max_iters=1000, trace_cap=4096, attempt_cap=5000)
    log = info["attempt_log"]
    assert info["attempt_len"] == info["attempts"] == len(log) >= 1000
    rows = np.array([[a[f] for f in L.ATTEMPT_FIELDS] for a in log])
    checks = np.array([[t["restart"], t["cand_is_avg"]] for t in tr])
    xo, yo, io, tro, att = _replay(oracle_mod, lp, rows, checks)
    y0p = 1e-12 * np.random.default_rng(1).normal(size=lp.m)
    xp, yp, ip, trp, attp = _replay(oracle_mod, lp, rows, checks, y0=y0p)
    assert io["iters"] == info["iters"] == ip["iters"] == 1000
    assert io["attempts"] == info["attempts"] == ip["attempts"]
    assert len(tr) == len(tro) == len(trp)
    # onset of the oracle's own divergence under the replayed schedule
    def gap(o, p, f):
        return abs(p[f] - o[f]) / max(abs(o[f]), 1e-300)
    onset = next((i for i, (o, p) in enumerate(zip(att, attp))
                  if max(gap(o, p, "eta_bar"), gap(o, p, "dx2"), gap(o, p, "dy2")) > 1e-6),
                 len(att))
    assert onset >= 100, onset
    if onset == len(att):
        assert rel(x, xo) <= 1e-10, rel(x, xo)
        assert rel(y, yo) <= 1e-10, rel(y, yo)
    band = lambda o, p: 10.0 * abs(p - o)
    # rounding-level tolerances: the terms of an attempt are differences of
    # iterates (||dx||^2, ||dy||^2) and dy^T K dx; with iterates agreeing to
    # eps ||z||, eta_bar (a ratio of them) agrees to tol_terms below; KKT values
    # are residual norms of the iterates (relative eps ||K~|| ||z|| / KKT,
    # floored at 1e-6, the summation-order level of the gap's cancellation)
    eps = 1e-13
    _, R, Cs, _ = oracle_mod.ruiz(lp)
    znorm = np.sqrt(np.sum((xo / Cs) ** 2) + np.sum((yo / R) ** 2))
    nk = info["norm_K"]
    tied = 0
    last_attempt = log[onset - 1]["k"] if onset < len(log) else np.inf
    for a, b, c in zip(tr, tro, trp):
        for f in ("k", "attempts", "restart", "cand_is_avg"):
            assert a[f] == b[f], (f, a, b)
        if a["k"] > last_attempt:
            break
        assert abs(a["omega"] - b["omega"]) <= 1e-10 * b["omega"] + band(b["omega"], c["omega"])
        for f in ("kkt_cur", "kkt_cand", "rel_gap", "rel_pres", "rel_dres"):
            t = max(1e-6 * abs(b[f]), 4 * eps * nk * znorm, 1e-12) + band(b[f], c[f])
            assert abs(a[f] - b[f]) <= t, (f, a[f], b[f], c[f])
        # the GPU's decisions against the oracle's own
        if b["own_cand_is_avg"] != b["cand_is_avg"]:
            t = (1e-6 * b["kkt_cur"] + band(b["kkt_cur"], c["kkt_cur"])
                 + band(b["kkt_avg"], c["kkt_avg"]))
            assert abs(b["kkt_cur"] - b["kkt_avg"]) <= t, (a, b)
            tied += 1
        if b["own_restart"] != b["restart"]:
            cnd = b["kkt_cand"]
            t = 1e-6 * cnd + band(cnd, c["kkt_cand"]) + band(b["kkt_anchor"], c["kkt_anchor"])
            d = oracle_mod.DEFAULTS
            near = (abs(cnd - d["beta_sufficient"] * b["kkt_anchor"]) <= t
                    or abs(cnd - d["beta_necessary"] * b["kkt_anchor"]) <= t
                    or abs(cnd - b["kkt_prev"]) <= t + band(b["kkt_prev"], c["kkt_prev"]))
            assert near, (a, b)
            tied += 1
    rejected = 0
    for g, o, p in list(zip(log, att, attp))[:onset]:
        assert g["k"] == o["k"] and g["eta"] == o["eta"]
        dz = np.sqrt(o["dx2"] + o["dy2"])
        tol_terms = max(1e-12, 8 * eps * znorm * (1.0 / max(dz, 1e-300)
                                                  + nk * dz / max(abs(o["inter"]), 1e-300)))
        eb = tol_terms * o["eta_bar"] + band(o["eta_bar"], p["eta_bar"])
        # where eta_bar sits well above eta, eta' = (1 + (k+1)^-0.6) eta does not
        # depend on it and the step is accepted either way: compared loosely there
        if o["eta_bar"] >= 2 * g["eta"]:
            eb = max(eb, 1e-5 * o["eta_bar"])
        assert abs(g["eta_bar"] - o["eta_bar"]) <= eb, (g, o, p)
        if abs(g["eta"] - o["eta_bar"]) > eb:
            assert bool(g["accept"]) == (g["eta"] <= o["eta_bar"]), (g, o)
        elif bool(g["accept"]) != (g["eta"] <= o["eta_bar"]):
            tied += 1
        en = tol_terms * o["eta_next"] + band(o["eta_next"], p["eta_next"])
        assert abs(g["eta_next"] - o["eta_next"]) <= en, (g, o, p)
        rejected += int(not g["accept"])
    print(name, "onset", onset, "of", len(att), "rejected attempts", rejected,
          "decisions taken at a tie", tied)


# ---------------------------------------------------------------- to tolerance

@pytest.mark.parametrize("tol", [1e-4, 1e-8])
def test_fp64_fixed_step_solve_matches_oracle(L, oracle_mod, tol):
    """Fixed-step restarted PDHG to tolerance: same iteration count, same
    decisions, objective equal to the oracle's to 1e-6 relative."""
    lp = PROBS["lp200x400"]
    prob = L.Problem(lp)
    x, y, info, tr = prob.solve(tol=tol, max_iters=400000, trace_cap=16384, **FIXED)
    xo, yo, io, tro = oracle_mod.solve(lp, tol=tol, max_iters=400000, trace_cap=16384, **FIXED)
    assert info["status"] == L.LP_OPTIMAL == io["status"]
    assert info["iters"] == io["iters"]
    assert float(lp.c @ x) == pytest.approx(float(lp.c @ xo), rel=1e-6)
    _check_trace(tr, tro)


@pytest.mark.parametrize("tol", [1e-4, 1e-8])
def test_fp64_adaptive_solve_reaches_oracle_objective(L, oracle_mod, tol):
    """Adaptive restarted PDHG (the default) to tolerance: the oracle re-checks
    the returned point in FP64, and the objective agrees with the oracle's
    solution within the tolerance's gap bound (and to 1e-6 at 1e-8)."""
    lp = PROBS["lp200x400"]
    prob = L.Problem(lp)
    x, y, info, tr = prob.solve(tol=tol, max_iters=200000, trace_cap=8192)
    xo, yo, io, _ = oracle_mod.solve(lp, tol=tol, max_iters=200000)
    assert info["status"] == L.LP_OPTIMAL == io["status"]
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= tol * (1 + 1e-6)
    f, fo = float(lp.c @ x), float(lp.c @ xo)
    assert abs(f - fo) <= 4 * tol * (1 + abs(fo))
    if tol <= 1e-8:
        assert f == pytest.approx(lp.f_star, rel=1e-6)
        assert fo == pytest.approx(lp.f_star, rel=1e-6)


# ---------------------------------------------------------------- behaviour

def test_repeat_solves_are_bitwise_identical(L):
    lp = PROBS["ragged"]
    prob = L.Problem(lp)
    r1 = prob.solve(tol=1e-13, max_iters=300, trace_cap=64)
    r2 = prob.solve(tol=1e-13, max_iters=300, trace_cap=64)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])
    assert r1[3] == r2[3]


def test_host_and_device_inputs_agree(L):
    lp = PROBS["powerlaw"]
    a = L.Problem(lp, device_copy=True).solve(tol=1e-13, max_iters=200)
    b = L.Problem(lp, device_copy=False).solve(tol=1e-13, max_iters=200)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_device_output_buffers(L):
    lp = PROBS["lp200x400"]
    prob = L.Problem(lp)
    xh, yh, _, _ = prob.solve(tol=1e-6, max_iters=100000)
    xd, yd, _, _ = prob.solve(tol=1e-6, max_iters=100000, out_device=True)
    assert np.array_equal(xh, xd.cpu().numpy()) and np.array_equal(yh, yd.cpu().numpy())


def test_warm_start_at_optimum_stops_at_first_check(L):
    lp = PROBS["lp200x400"]
    prob = L.Problem(lp)
    x, y, info, tr = prob.solve(tol=1e-8, x0=lp.x_star, y0=lp.y_star, trace_cap=16)
    assert info["status"] == L.LP_OPTIMAL and info["iters"] == 0
    assert rel(x, lp.x_star) < 1e-12


def test_iteration_and_time_limits(L):
    lp = PROBS["ragged"]
    prob = L.Problem(lp)
    _, _, info, _ = prob.solve(tol=1e-14, max_iters=130)
    assert info["status"] == L.LP_ITERATION_LIMIT and info["iters"] == 130
    _, _, info, _ = prob.solve(tol=1e-14, max_iters=10**9, time_limit_s=1e-7)
    assert info["status"] == L.LP_TIME_LIMIT


def _desc_copy(lp, **changes):
    d = {f: getattr(lp, f) for f in ("m", "n", "row_ptr", "col_idx", "vals", "sense",
                                     "c", "q", "l", "u")}
    d.update(changes)
    return synth.LP(**d)


@pytest.mark.parametrize("bad", ["col", "nan", "bounds", "rowptr", "sense"])
def test_invalid_problems_are_rejected(L, bad):
    lp = PROBS["lp200x400"]
    if bad == "col":
        ci = lp.col_idx.copy(); ci[5] = lp.n
        b = _desc_copy(lp, col_idx=ci)
    elif bad == "nan":
        v = lp.vals.copy(); v[3] = np.nan
        b = _desc_copy(lp, vals=v)
    elif bad == "bounds":
        l = lp.l.copy(); l[2] = lp.u[2] + 1
        b = _desc_copy(lp, l=l)
    elif bad == "rowptr":
        rp = lp.row_ptr.copy(); rp[10], rp[11] = rp[11], rp[10] - 1
        b = _desc_copy(lp, row_ptr=rp)
    else:
        s = lp.sense.copy(); s[0] = 7
        b = _desc_copy(lp, sense=s)
    with pytest.raises(L.LpError) as e:
        L.Problem(b)
    assert e.value.status == L.LP_INVALID_ARGUMENT


def test_constraint_free_columns_and_free_variables(L, oracle_mod):
    """Free variables (l = -inf, u = +inf) and one-sided bounds: lambda's
    projection onto {0}, R^+, R^- on the device agrees with the oracle."""
    lp = synth.small_dense_lp()
    rng = np.random.default_rng(5)
    l, u = lp.l.copy(), lp.u.copy()
    interior = (lp.x_star > lp.l) & (lp.x_star < lp.u)
    idx = np.flatnonzero(interior)
    l[idx[: len(idx) // 3]] = -np.inf
    u[idx[len(idx) // 3: 2 * len(idx) // 3]] = np.inf
    both = idx[2 * len(idx) // 3:][:10]
    l[both], u[both] = -np.inf, np.inf
    lp2 = _desc_copy(lp, l=l, u=u)
    prob = L.Problem(lp2)
    x, y, info, tr = prob.solve(tol=1e-13, max_iters=500, trace_cap=64, **FIXED)
    xo, yo, io, tro = oracle_mod.solve(lp2, tol=1e-13, max_iters=500, trace_cap=64, **FIXED)
    assert rel(x, xo) <= 1e-10 and rel(y, yo) <= 1e-10
    _check_trace(tr, tro)


@pytest.mark.parametrize("name", ["ragged", "powerlaw"])
def test_autotuned_schedule_solves(L, oracle_mod, name):
    """With the schedule autotuner on, the solve reaches the same tolerance and
    objective (the task shapes change only the order of the row sums)."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    x, y, info, _ = prob.solve(tol=1e-7, autotune=1, max_iters=500000)
    assert info["status"] == L.LP_OPTIMAL
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-7 * (1 + 1e-6)
    # a second solve on the same handle reuses the tuned schedule: bitwise repeatable
    x2, y2, info2, _ = prob.solve(tol=1e-7, autotune=1, max_iters=500000)
    assert np.array_equal(x, x2) and np.array_equal(y, y2)
