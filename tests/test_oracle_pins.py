"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-worked
values (tests/golden), closed forms, brute force on tiny inputs, a library
routine (LAPACK SVD), planted optima whose KKT conditions hold by construction,
and invariants of the convergence proof (Appendix D).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _lp_from_case(d):
    return synth.from_dense(d["K"], d["sense"], d["c"], d["q"], d["l"], d["u"])


# ---------------------------------------------------------------- KKT terms

def test_kkt_hand_values(oracle_mod):
    """Section 2.3.2 termination quantities and Section 2.4.2 KKT_omega on
    hand-worked cases (free, lower-only and boxed variables; >= and = rows)."""
    d = _load("kkt_hand.json")
    lp = _lp_from_case(d)
    for case in d["cases"]:
        got = oracle_mod.kkt(lp, case["x"], case["y"], omega=d["omega"])
        for key in oracle_mod.KKT_FIELDS:
            assert got[key] == pytest.approx(case[key], rel=1e-13, abs=1e-14), key


def test_proj_lambda_brute_force(oracle_mod):
    """lambda = nearest point of Lambda_i (Section 2.2): brute force over the
    candidates {v, 0} restricted to each Lambda_i."""
    rng = np.random.default_rng(1)
    n = 400
    l = np.where(rng.random(n) < 0.5, -np.inf, rng.normal(size=n))
    u = np.where(rng.random(n) < 0.5, np.inf, np.abs(rng.normal(size=n)) + 5)
    v = rng.normal(size=n)
    lam = oracle_mod.proj_lambda(l, u, v)
    for j in range(n):
        lf, uf = np.isfinite(l[j]), np.isfinite(u[j])
        allowed = []
        for cand in (v[j], 0.0):
            ok = ((lf and uf) or (not lf and not uf and cand == 0.0) or
                  (not lf and uf and cand <= 0) or (lf and not uf and cand >= 0))
            if ok:
                allowed.append(cand)
        best = min(allowed, key=lambda t: abs(t - v[j]))
        assert lam[j] == best


def test_dual_objective_brute_force_corners(oracle_mod):
    """For finite boxes the dual function is q^T y + min over box corners of
    (c - K^T y)^T x (Appendix B); the oracle's q^T y + l^T lambda^+ + u^T lambda^-
    must equal that minimum, found by enumerating all 2^n corners."""
    rng = np.random.default_rng(2)
    for trial in range(5):
        m, n = 4, 7
        K = rng.normal(size=(m, n)) * (rng.random((m, n)) < 0.7)
        sense = rng.integers(0, 2, m)
        lp = synth.from_dense(K, sense, rng.normal(size=n), rng.normal(size=m),
                              rng.uniform(-2, 0, n), rng.uniform(0.5, 3, n))
        y = rng.normal(size=m)
        y[sense == 1] = np.abs(y[sense == 1])
        lam = lp.c - K.T @ y
        best = min(float(lam @ np.where(bits, lp.u, lp.l))
                   for bits in itertools.product([0, 1], repeat=n))
        got = oracle_mod.kkt(lp, np.zeros(n), y)["dobj"]
        assert got == pytest.approx(float(lp.q @ y) + best, rel=1e-12, abs=1e-12)


def test_weak_duality_random_points(oracle_mod):
    """Weak duality (Appendix B): dual objective <= optimum <= primal objective
    of any feasible point; equality at the planted optimum."""
    lp = synth.small_dense_lp()
    f_star = lp.f_star
    rng = np.random.default_rng(3)
    for _ in range(20):
        y = lp.y_star + rng.normal(size=lp.m) * 0.3
        y[lp.sense == 1] = np.maximum(y[lp.sense == 1], 0)
        assert oracle_mod.kkt(lp, lp.x_star, y)["dobj"] <= f_star + 1e-9
    k = oracle_mod.kkt(lp, lp.x_star, lp.y_star)
    assert k["pobj"] == pytest.approx(f_star, rel=1e-14)
    assert k["dobj"] == pytest.approx(f_star, rel=1e-12)


def test_planted_point_has_zero_kkt(oracle_mod):
    """The planted (x0, y0) satisfies the KKT conditions exactly, so all three
    relative errors of Section 2.3.2 vanish; moving off it makes them positive."""
    for lp in (synth.small_dense_lp(), synth.power_law_lp(3000, 6000, 4, 200, seed=5),
               synth.shuffle_sense(synth.small_dense_lp(), 7)):
        k = oracle_mod.kkt(lp, lp.x_star, lp.y_star)
        assert k["rel_gap"] < 1e-13 and k["rel_pres"] < 1e-13 and k["rel_dres"] < 1e-13
        assert k["kkt_omega"] < 1e-9
        k2 = oracle_mod.kkt(lp, lp.x_star * 1.01, lp.y_star)
        assert k2["rel_pres"] > 1e-6 or k2["rel_gap"] > 1e-6


# ---------------------------------------------------------------- PDHG step

def test_pdhg_steps_hand(oracle_mod):
    d = _load("pdhg_steps_hand.json")
    for case in d["cases"]:
        lp = _lp_from_case(case)
        x, y = np.array(case["x0"], float), np.array(case["y0"], float)
        for xs, ys in zip(case["xs"], case["ys"]):
            x, y = oracle_mod.pdhg_step(lp, x, y, case["tau"], case["sigma"])
            np.testing.assert_allclose(x, xs, rtol=0, atol=1e-15)
            np.testing.assert_allclose(y, ys, rtol=0, atol=1e-15)


def test_step_without_constraints_is_projected_gradient(oracle_mod):
    """With K = 0 the primal step is projected gradient descent on c^T x and the
    dual step is projected gradient ascent on q^T y (textbook special case)."""
    rng = np.random.default_rng(4)
    m, n = 30, 50
    lp = synth.from_dense(np.zeros((m, n)), rng.integers(0, 2, m), rng.normal(size=n),
                          rng.normal(size=m), rng.uniform(-1, 0, n), rng.uniform(0, 1, n))
    x = rng.normal(size=n)
    y = rng.normal(size=m)
    xn, yn = oracle_mod.pdhg_step(lp, x, y, 0.3, 0.7)
    np.testing.assert_array_equal(xn, np.minimum(np.maximum(x - 0.3 * lp.c, lp.l), lp.u))
    ey = y + 0.7 * lp.q
    ey[lp.sense == 1] = np.maximum(ey[lp.sense == 1], 0)
    np.testing.assert_array_equal(yn, ey)


def test_saddle_point_is_fixed_point(oracle_mod):
    """A saddle point is a fixed point of the PDHG map (Appendix D); a wrong
    sign or a transposed operand anywhere in the step moves it."""
    for lp in (synth.small_dense_lp(), synth.power_law_lp(2000, 4000, 4, 300, seed=9)):
        for tau, sigma in ((0.1, 0.2), (1.0, 0.05)):
            xn, yn = oracle_mod.pdhg_step(lp, lp.x_star, lp.y_star, tau, sigma)
            assert np.max(np.abs(xn - lp.x_star)) < 1e-12
            assert np.max(np.abs(yn - lp.y_star)) < 1e-12


def test_fixed_step_distance_to_saddle_nonincreasing(oracle_mod):
    """Appendix D boundedness: with tau sigma ||K||^2 < 1 the iterates stay in
    the ball around any saddle point in the PDHG metric
    ||z||_M^2 = ||x||^2/tau + 2 y^T K x + ||y||^2/sigma, and the distance never
    grows from one iterate to the next."""
    lp = synth.small_dense_lp()
    Kd = lp.dense()
    normK = np.linalg.norm(Kd, 2)
    eta = 0.9 / normK
    for omega in (0.3, 1.0, 4.0):
        tau, sigma = eta / omega, eta * omega
        xs, ys = oracle_mod.unrolled_forward(lp, tau, sigma, 400)
        dx = xs - lp.x_star
        dy = ys - lp.y_star
        d = (np.sum(dx * dx, 1) / tau + 2 * np.einsum("ti,ij,tj->t", dy, Kd, dx)
             + np.sum(dy * dy, 1) / sigma)
        assert np.all(d > 0)
        assert np.all(np.diff(d) <= 1e-10 * d[0])
        assert d[-1] < d[0]


# ---------------------------------------------------------------- setup steps

def test_power_iteration_matches_svd(oracle_mod):
    """Algorithm 2 converges to the largest singular value (LAPACK SVD)."""
    for seed, (m, n) in enumerate(((30, 50), (60, 20), (200, 400))):
        lp = synth.random_planted(m, n, density=0.2, seed=seed)
        s = np.linalg.svd(lp.dense(), compute_uv=False)[0]
        assert oracle_mod.power_norm(lp, 1000) == pytest.approx(s, rel=1e-8)


def test_ruiz_reaches_unit_norms_and_is_consistent(oracle_mod):
    """Algorithm 3: row and column infinity norms converge to 1; the scaled
    values equal diag(R) K diag(C) entrywise; an already equilibrated matrix
    takes no pass."""
    lp = synth.power_law_lp(2000, 3000, 4, 100, seed=11)
    lp.vals = lp.vals * np.exp(np.random.default_rng(0).normal(0, 2, lp.nnz))
    vs, R, Cc, passes = oracle_mod.ruiz(lp, iters=60, tol=1e-6)
    rows = lp.row_of_nnz()
    np.testing.assert_allclose(vs, R[rows] * lp.vals * Cc[lp.col_idx], rtol=1e-13)
    rn = np.zeros(lp.m)
    np.maximum.at(rn, rows, np.abs(vs))
    cn = np.zeros(lp.n)
    np.maximum.at(cn, lp.col_idx, np.abs(vs))
    assert np.max(np.abs(rn[rn > 0] - 1)) < 1e-3
    assert np.max(np.abs(cn[cn > 0] - 1)) < 1e-3
    perm = synth.from_dense(np.eye(5)[::-1] * -1.0, [1] * 5, np.ones(5), np.ones(5),
                            np.zeros(5), np.ones(5))
    assert oracle_mod.ruiz(perm, 10, 1e-6)[3] == 0


def test_scaling_leaves_the_optimum_unchanged(oracle_mod):
    """Section 2.4.1 change of variables: the unscaled objective at 1e-8 is
    the same with and without preconditioning (and equals the planted one)."""
    lp = synth.small_dense_lp()
    objs = []
    for ruiz_iters, pc in ((0, 0), (10, 0), (10, 1)):
        x, y, info, _ = oracle_mod.solve(lp, tol=1e-8, ruiz_iters=ruiz_iters,
                                         pock_chambolle=pc, max_iters=200000)
        assert info["status"] == 1
        objs.append(float(lp.c @ x))
    for o in objs:
        assert o == pytest.approx(lp.f_star, rel=1e-6)


# ---------------------------------------------------------------- full solve

def _vertex_enumeration(lp):
    """Exact LP optimum by enumerating vertices: every choice of n linearly
    independent active constraints (all equalities plus some inequality rows
    and bounds), solved, kept if feasible."""
    K = lp.dense()
    m, n = K.shape
    eq = [i for i in range(m) if lp.sense[i] == 0]
    ge = [i for i in range(m) if lp.sense[i] == 1]
    cands = [("r", i) for i in ge] + [("l", j) for j in range(n)] + [("u", j) for j in range(n)]
    best = math.inf
    need = n - len(eq)
    for pick in itertools.combinations(cands, need):
        A = [K[i] for i in eq]
        b = [lp.q[i] for i in eq]
        for kind, idx in pick:
            if kind == "r":
                A.append(K[idx]); b.append(lp.q[idx])
            else:
                e = np.zeros(n); e[idx] = 1.0
                A.append(e); b.append(lp.l[idx] if kind == "l" else lp.u[idx])
        A = np.array(A); b = np.array(b)
        if abs(np.linalg.det(A)) < 1e-10:
            continue
        x = np.linalg.solve(A, b)
        Kx = K @ x
        if (np.all(x >= lp.l - 1e-9) and np.all(x <= lp.u + 1e-9)
                and np.all(np.abs(Kx[eq] - lp.q[eq]) < 1e-9)
                and np.all(Kx[ge] >= lp.q[ge] - 1e-9)):
            best = min(best, float(lp.c @ x))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_solve_matches_vertex_enumeration(oracle_mod, seed):
    """The oracle's objective at 1e-9 relative KKT equals the exact optimum
    found by vertex enumeration (n <= 6), including LPs whose costs are not
    planted."""
    rng = np.random.default_rng(100 + seed)
    m, n = 4, 6
    K = rng.normal(size=(m, n))
    sense = np.array([1, 1, 1, 0]) if seed % 2 else np.array([1, 0, 1, 1])
    l = rng.uniform(-1, 0, n)
    u = rng.uniform(0.5, 2, n)
    x_feas = rng.uniform(l, u)
    q = K @ x_feas - np.where(sense == 1, rng.uniform(0, 1, m), 0.0)
    c = rng.normal(size=n)
    lp = synth.from_dense(K, sense, c, q, l, u)
    f_exact = _vertex_enumeration(lp)
    x, y, info, _ = oracle_mod.solve(lp, tol=1e-9, max_iters=500000)
    assert info["status"] == 1
    assert float(lp.c @ x) == pytest.approx(f_exact, rel=1e-6, abs=1e-7)


def test_solve_reaches_planted_optimum(oracle_mod):
    """Planted LPs: at 1e-8 the objective matches c^T x0 and the three relative
    errors recomputed from the returned point are below tolerance."""
    for lp in (synth.small_dense_lp(), synth.shuffle_sense(synth.small_dense_lp(), 3)):
        x, y, info, trace = oracle_mod.solve(lp, tol=1e-8, max_iters=300000)
        assert info["status"] == 1
        assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-6)
        k = oracle_mod.kkt(lp, x, y)
        assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-8
        assert trace[-1]["rel_gap"] == pytest.approx(k["rel_gap"], rel=1e-9, abs=1e-15)


def test_restart_records_follow_the_criteria(oracle_mod):
    """Every check record's restart flag agrees with the three criteria of
    Section 2.4.2 evaluated on the logged KKT values (beta 0.2 / 0.8 / 0.36)."""
    lp = synth.small_dense_lp()
    _, _, info, trace = oracle_mod.solve(lp, tol=1e-8, max_iters=300000)
    anchor = trace[0]["kkt_cand"]
    prev = math.inf
    epoch_start = 0
    for t in trace[1:]:
        kc = t["kkt_cand"]
        assert kc == min(t["kkt_cur"], t["kkt_avg"])
        assert t["cand_is_avg"] == (0.0 if t["kkt_cur"] < t["kkt_avg"] else 1.0)
        converged = max(t["rel_gap"], t["rel_pres"], t["rel_dres"]) <= 1e-8
        expect = (not converged) and (kc <= 0.2 * anchor or (kc <= 0.8 * anchor and kc > prev)
                                      or (t["k"] - epoch_start) > 0.36 * t["k"])
        assert bool(t["restart"]) == expect
        if t["restart"]:
            anchor, prev, epoch_start = kc, math.inf, t["k"]
        else:
            prev = kc
    assert info["restarts"] == sum(int(t["restart"]) for t in trace)


def test_fixed_step_solver_converges_without_enhancements(oracle_mod):
    """Plain Algorithm 1 (no scaling, restarts, adaptive step or weight updates)
    also reaches the planted optimum, only more slowly."""
    lp = synth.small_dense_lp()
    x, y, info, _ = oracle_mod.solve(lp, tol=1e-5, ruiz_iters=0, restarts=0, adaptive_step=0,
                                     primal_weight_update=0, max_iters=2_000_000)
    assert info["status"] == 1
    assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-4)


def test_iteration_limit_status(oracle_mod):
    lp = synth.small_dense_lp()
    _, _, info, trace = oracle_mod.solve(lp, tol=1e-12, max_iters=100)
    assert info["status"] == 4 and info["iters"] == 100
    assert trace[-1]["k"] == 100


# ---------------------------------------------------------------- adjoint

def test_unrolled_adjoint_matches_central_differences(oracle_mod):
    """Reverse-mode gradient of ||x_K - x_target||^2 through K fixed-step
    iterations equals central finite differences (h = 1e-6, FP64) for entries
    whose projection masks do not flip under +-h (at a flip the loss has a kink
    and the two one-sided derivatives differ)."""
    lp, xt = synth.adjoint_lp(50, 100, 8, seed=20250820)
    eta = 0.9 / oracle_mod.power_norm(lp, 200)
    omega = 1.0
    tau, sigma = eta / omega, eta * omega
    Kit = 200

    def loss(lp_):
        xs, _ = oracle_mod.unrolled_forward(lp_, tau, sigma, Kit)
        return float(np.sum((xs[-1] - xt) ** 2))

    xs, _ = oracle_mod.unrolled_forward(lp, tau, sigma, Kit)
    dc, dq, dv = oracle_mod.unrolled_adjoint(lp, tau, sigma, Kit, 2 * (xs[-1] - xt))
    h = 1e-6
    rng = np.random.default_rng(0)
    checked = 0

    def masks(lp_):
        xs_, ys_ = oracle_mod.unrolled_forward(lp_, tau, sigma, Kit)
        out = []
        for t in range(Kit):
            vx = xs_[t] - tau * (lp_.c - oracle_mod.spmv_t(lp_, ys_[t]))
            vy = ys_[t] + sigma * (lp_.q - oracle_mod.spmv(lp_, 2 * xs_[t + 1] - xs_[t]))
            out.append(np.concatenate([(lp_.l < vx) & (vx < lp_.u), (lp_.sense == 0) | (vy > 0)]))
        return np.array(out)

    m0 = masks(lp)
    for kind, grad, n_ in (("c", dc, lp.n), ("q", dq, lp.m), ("vals", dv, lp.nnz)):
        for idx in rng.choice(n_, 12, replace=False):
            lps = []
            for sgn in (+1, -1):
                cp = synth.LP(**{f.name: getattr(lp, f.name) for f in
                                 __import__("dataclasses").fields(lp)})
                arr = getattr(lp, kind).copy()
                arr[idx] += sgn * h
                setattr(cp, kind, arr)
                lps.append(cp)
            # a projection kink between the two evaluations makes the loss
            # non-differentiable there (one-sided derivatives differ): skip it
            if not all(np.array_equal(m0, masks(q_)) for q_ in lps):
                continue
            fd = (loss(lps[0]) - loss(lps[1])) / (2 * h)
            scale = max(abs(fd), abs(grad[idx]), 1e-3)
            assert abs(fd - grad[idx]) / scale < 1e-5, (kind, idx, fd, grad[idx])
            checked += 1
    assert checked >= 30


def test_adaptive_step_amplifies_rounding(oracle_mod):
    """Documents why iterate tracking with Algorithm 5 is checked over the first
    check period only: moving eta_0 by one part in 1e15 leaves fixed-step
    restarted PDHG within 1e-13 of its own run after 1000 iterations, while the
    adaptive step rule carries the same change to > 1e-7."""
    lp = synth.small_dense_lp()
    vs, R, Cc, _ = oracle_mod.ruiz(lp, 10, 1e-4)
    eta = 0.9 / oracle_mod.power_norm(lp, 100, vals=vs)
    out = {}
    for adaptive in (0, 1):
        xa = oracle_mod.solve(lp, tol=1e-13, max_iters=1000, eta0=eta, adaptive_step=adaptive)[0]
        xb = oracle_mod.solve(lp, tol=1e-13, max_iters=1000, eta0=eta * (1 + 1e-15),
                              adaptive_step=adaptive)[0]
        out[adaptive] = np.linalg.norm(xa - xb) / np.linalg.norm(xa)
    assert out[0] < 1e-13
    assert out[1] > 1e-7


# ---------------------------------------------------------------- Pock-Chambolle

def test_pock_chambolle_hand_values(oracle_mod):
    """The Pock-Chambolle pass for alpha in {0, 1/2, 1, 2} on a hand-worked 2 x 2
    matrix (tests/golden/pock_chambolle_hand.json): factors and scaled values."""
    d = _load("pock_chambolle_hand.json")
    K = np.array(d["K"], dtype=float)
    lp = synth.from_dense(K, [1, 1], [1.0, 1.0], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0])
    for case in d["cases"]:
        vs, R, Cc, passes = oracle_mod.ruiz(lp, 0, 1e-4, pock_chambolle=True,
                                            pc_alpha=case["alpha"])
        assert passes == 0
        np.testing.assert_allclose(R, case["R"], rtol=1e-14, err_msg=case["_work"])
        np.testing.assert_allclose(Cc, case["C"], rtol=1e-14, err_msg=case["_work"])
        want = (np.array(case["R"])[:, None] * K * np.array(case["C"])[None, :])[K != 0]
        np.testing.assert_allclose(vs, want, rtol=1e-14)


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0, 2.0])
def test_pock_chambolle_leaves_the_optimum_unchanged(oracle_mod, alpha):
    """Section 2.4.1 change of variables with the Pock-Chambolle pass after Ruiz:
    the unscaled objective at 1e-8 is the planted one for every alpha."""
    lp = synth.small_dense_lp()
    x, y, info, _ = oracle_mod.solve(lp, tol=1e-8, pock_chambolle=1, pc_alpha=alpha,
                                     max_iters=200000)
    assert info["status"] == 1 and info["pc_alpha"] == alpha
    assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-6)


@pytest.mark.parametrize("name", ["small_dense", "ragged"])
def test_pock_chambolle_choice(oracle_mod, name):
    """pock_chambolle = 2: each trial error is that of a separate solve with that
    alpha, the stated number of iterations, no tolerance and no infeasibility
    detection; the chosen alpha has the smallest; the tuned solve is the solve
    with the chosen alpha, bit for bit."""
    lp = {"small_dense": synth.small_dense_lp, "ragged": synth.ragged_lp}[name]()
    alpha, errs = oracle_mod.pc_tune(lp, check_every=32)
    for a, e in zip(oracle_mod.PC_GRID, errs):
        _, _, info, _ = oracle_mod.solve(lp, pock_chambolle=1, pc_alpha=a, max_iters=64, tol=0.0,
                                         infeas_detect=0, check_every=32)
        assert e == max(info["rel_gap"], info["rel_pres"], info["rel_dres"])
    assert alpha == oracle_mod.PC_GRID[int(np.argmin(errs))]
    xa, ya, ia, _ = oracle_mod.solve(lp, pock_chambolle=2, check_every=32)
    xb, yb, ib, _ = oracle_mod.solve(lp, pock_chambolle=1, pc_alpha=alpha, check_every=32)
    assert ia["pc_alpha"] == alpha
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(ya, yb)
