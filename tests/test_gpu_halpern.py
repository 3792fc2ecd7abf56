"""GPU parity of restarted (reflected) Halpern PDHG against the oracle.

The Halpern map is nonexpansive, so FP64 rounding differences between the two
summation orders do not grow: over hundreds of iterations with restarts the
candidate matches the oracle's to 1e-9 relative and every check record (restart
decision, omega, KKT values) agrees.  To tolerance, the oracle re-evaluates the
returned point in FP64.
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
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


PROBS = {
    "lp200x400": synth.small_dense_lp(),
    "ragged": synth.ragged_lp(),
    "shuffled": synth.shuffle_sense(synth.small_dense_lp(), 3),
    "powerlaw": synth.power_law_lp(4000, 8000, 4, 600, seed=11),
}


def _check_trace(tr, tro, rtol=1e-8, omega_rtol=1e-10):
    assert len(tr) == len(tro)
    for a, b in zip(tr, tro):
        assert a["k"] == b["k"] and a["attempts"] == b["attempts"]
        assert a["restart"] == b["restart"], (a, b)
        assert a["cand_is_avg"] == b["cand_is_avg"] == 1.0
        assert a["eta"] == pytest.approx(b["eta"], rel=1e-10), ("eta", a["eta"], b["eta"])
        assert a["omega"] == pytest.approx(b["omega"], rel=omega_rtol), ("omega", a["omega"],
                                                                        b["omega"])
        for f in ("kkt_cur", "kkt_avg", "kkt_cand", "rel_gap", "rel_pres", "rel_dres"):
            assert a[f] == pytest.approx(b[f], rel=rtol, abs=1e-10), (f, a[f], b[f])


@pytest.mark.parametrize("rho", [1.0, 0.0, 0.5])
@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("iters", [1, 63, 64, 700])
def test_fp64_halpern_tracks_oracle(L, oracle_mod, name, iters, rho):
    """Iteration-limit runs (restarts and primal-weight updates on): the
    candidate T(z) at the last check, the restart count and every check record
    agree with the oracle."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    kw = dict(tol=1e-13, max_iters=iters, trace_cap=4096, halpern=1)
    x, y, info, tr = prob.solve(halpern_reflect=rho, **kw)
    xo, yo, io, tro = oracle_mod.solve(lp, reflect=rho, **kw)
    assert info["status"] == io["status"] == L.LP_ITERATION_LIMIT
    assert info["iters"] == io["iters"] == iters
    assert info["attempts"] == iters
    assert info["restarts"] == io["restarts"]
    assert rel(x, xo) <= 1e-9, rel(x, xo)
    assert rel(y, yo) <= 1e-9, rel(y, yo)
    _check_trace(tr, tro)


@pytest.mark.parametrize("tol", [1e-4, 1e-8])
def test_fp64_halpern_solve_matches_oracle(L, oracle_mod, tol):
    lp = PROBS["lp200x400"]
    prob = L.Problem(lp)
    x, y, info, tr = prob.solve(tol=tol, max_iters=400000, trace_cap=16384, halpern=1)
    xo, yo, io, tro = oracle_mod.solve(lp, tol=tol, max_iters=400000, trace_cap=16384, halpern=1)
    assert info["status"] == L.LP_OPTIMAL == io["status"]
    assert info["iters"] == io["iters"]
    assert float(lp.c @ x) == pytest.approx(float(lp.c @ xo), rel=1e-6)
    # thousands of iterations: Algorithm 4's omega is a ratio of differences of
    # restart points, which carry the two runs' accumulated summation-order
    # differences; compared at 1e-8 here (1e-10 in the 700-iteration tracking)
    _check_trace(tr, tro, rtol=1e-6, omega_rtol=1e-8)
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= tol * (1 + 1e-6)


@pytest.mark.parametrize("name,tol", [("ragged", 1e-7), ("shuffled", 1e-7), ("powerlaw", 1e-6)])
def test_mixed_halpern_solves(L, oracle_mod, name, tol):
    """FP32 Halpern iterations to 1e-5, then the FP64 polish (also Halpern) to
    the tolerance; the oracle re-checks the point."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    x, y, info, _ = prob.solve(tol=tol, max_iters=2000000, precision=L.LP_PREC_MIXED,
                               halpern=1)
    assert info["status"] == L.LP_OPTIMAL
    assert info["precision_used"] == L.LP_PREC_FP64
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= tol * (1 + 1e-6)
    if getattr(lp, "f_star", None) is not None:
        assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-5, abs=1e-6)


def test_fp32_phase_caps_reflection(L):
    """The FP32 phase of LP_PREC_MIXED runs with min(rho, 1/2): rho = 1 and
    rho = 1/2 give the same FP32 run (the same check records up to its last
    check), and it reaches the hand-over tolerance; the FP64 check then decides
    whether FP64 iterations follow."""
    lp = PROBS["ragged"]
    prob = L.Problem(lp)
    a = prob.solve(tol=1e-5, max_iters=400000, precision=L.LP_PREC_MIXED, halpern=1,
                   halpern_reflect=1.0, trace_cap=100000)
    b = prob.solve(tol=1e-5, max_iters=400000, precision=L.LP_PREC_MIXED, halpern=1,
                   halpern_reflect=0.5, trace_cap=100000)
    assert a[2]["status"] == b[2]["status"] == L.LP_OPTIMAL
    k32 = a[2]["iters"] - a[2]["fp64_iters"]
    assert k32 == b[2]["iters"] - b[2]["fp64_iters"]
    # records of the FP32 phase: up to its last check, at k32 (the FP64 start
    # check that follows has the same k)
    n32 = next(i for i, r in enumerate(a[3]) if r["k"] == k32) + 1
    assert a[3][:n32] == b[3][:n32]
    assert a[3][n32 - 1]["k"] == k32 and max(a[3][n32 - 1][f] for f in
                                            ("rel_gap", "rel_pres", "rel_dres")) <= 1e-5


def test_halpern_profile_step(L):
    """lp_profile_step times the Halpern step kernels after a Halpern solve."""
    prob = L.Problem(PROBS["powerlaw"])
    prob.solve(tol=1e-4, max_iters=128, precision=L.LP_PREC_MIXED, halpern=1)
    ms, by = prob.profile_step(L.LP_PREC_MIXED, reps=3)
    assert all(t > 0 for t in ms[:3]) and all(b > 0 for b in by[:3])


def test_halpern_repeat_solves_are_bitwise_identical(L):
    prob = L.Problem(PROBS["powerlaw"])
    r1 = prob.solve(tol=1e-13, max_iters=300, trace_cap=64, halpern=1)
    r2 = prob.solve(tol=1e-13, max_iters=300, trace_cap=64, halpern=1)
    np.testing.assert_array_equal(r1[0], r2[0])
    np.testing.assert_array_equal(r1[1], r2[1])


def test_halpern_then_pdhg_on_one_handle(L, oracle_mod):
    """Switching between the two loops on one handle rebuilds the loop graph."""
    lp = PROBS["lp200x400"]
    prob = L.Problem(lp)
    a = prob.solve(tol=1e-13, max_iters=200, halpern=1)
    b = prob.solve(tol=1e-13, max_iters=200, adaptive_step=0)
    ao = oracle_mod.solve(lp, tol=1e-13, max_iters=200, halpern=1)
    bo = oracle_mod.solve(lp, tol=1e-13, max_iters=200, adaptive_step=0)
    assert rel(a[0], ao[0]) <= 1e-9 and rel(b[0], bo[0]) <= 1e-9


def test_halpern_stop_between_checks_returns_last_candidate(L, oracle_mod):
    """A loop stopped by the time limit returns the candidate of the last check:
    its x and y belong together, so the oracle's FP64 termination quantities of
    the returned pair are the ones that check recorded.  Several limits are
    tried; whatever iteration each run stops at, the pair must match the last
    trace record, and at least one run must stop between two checks (iterations
    not a multiple of check_every), the case the candidate buffers exist for."""
    lp = PROBS["powerlaw"]
    prob = L.Problem(lp)
    between = 0
    for limit in (0.02, 0.05, 0.11, 0.23):
        x, y, info, tr = prob.solve(tol=1e-14, max_iters=10**9, time_limit_s=limit, halpern=1,
                                    trace_cap=100000)
        assert info["status"] == L.LP_TIME_LIMIT
        k = oracle_mod.kkt(lp, x, y)
        for f in ("rel_gap", "rel_pres", "rel_dres"):
            assert tr[-1][f] == info[f]
            assert k[f] == pytest.approx(info[f], rel=1e-6, abs=1e-12), (limit, f, k[f], info[f])
        between += int(info["iters"] % 64 != 0)
    assert between >= 1


def test_halpern_options_validated(L):
    prob = L.Problem(PROBS["lp200x400"])
    for bad in (dict(halpern=2), dict(halpern=1, halpern_reflect=1.5),
                dict(halpern=1, halpern_reflect=-0.1), dict(halpern=1, halpern_reflect=math.nan)):
        with pytest.raises(L.LpError):
            prob.solve(tol=1e-4, **bad)
    batch = L.Batch([PROBS["lp200x400"], PROBS["shuffled"]])
    with pytest.raises(L.LpError) as e:
        batch.solve(tol=1e-4, halpern=1)
    assert e.value.status == -5


def test_halpern_ignores_adaptive_and_infeasibility_options(L, oracle_mod):
    """adaptive_step and infeas_detect do not change a Halpern run."""
    lp = PROBS["ragged"]
    prob = L.Problem(lp)
    a = prob.solve(tol=1e-13, max_iters=300, halpern=1, adaptive_step=1, infeas_detect=1)
    b = prob.solve(tol=1e-13, max_iters=300, halpern=1, adaptive_step=0, infeas_detect=0)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
