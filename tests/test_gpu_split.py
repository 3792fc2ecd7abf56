"""Rows of K or K^T cut into pieces across the SpMV's task lists (split rows).

When the longest-first task lists would be unbalanced (a few rows each worth
several chunks against a small mean), the host cuts those rows into pieces on
different warps; the warp that completes a row adds its pieces in a fixed order
and applies the epilogue, and the epilogue's reductions for that row go to a
fixed partial slot.  The ragged LP (10,000 x 6,000 with rows and columns of up
to ~5,000 nonzeros) is split on both sides in both precisions; the miniature
dispatch-shaped LP (2,801 x 60, columns of hundreds of nonzeros, gathered through
L1 in 380-nonzero chunks) adds the long-column shape, without splits.  Checked
here, through the C ABI against the FP64 oracle:

- the schedules do cut rows (lp_result.split_rows);
- FP64 iterates and check records over the first two check periods with
  Algorithm 5 (its terms of split rows from both launches, the power
  iteration's partials);
- the adjoint of unrolled steps (forward and reverse products on split rows);
- FP32 fixed steps track the oracle at the FP32 level, and mixed solves reach
  the tolerance by the oracle's own KKT evaluation;
- repeat solves are bitwise identical: which warp completes a split row changes
  from launch to launch, the sums must not.
The Halpern iterations on the ragged LP (its K launch's split-row partials are
read by the K^T launch) are tracked in test_gpu_halpern.py.
"""
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


PROBS = {
    "ragged": synth.ragged_lp(),
    "dispatch_mini": synth.dispatch_lp(n_gen=60, n_base=400, n_cont=6, lo=5, hi=40, seed=3),
}


@pytest.mark.parametrize("name,prec", [("ragged", 0), ("ragged", 1)])
def test_schedules_cut_rows(L, name, prec):
    prob = L.Problem(PROBS[name])
    _, _, info, _ = prob.solve(tol=1e-13, max_iters=8, precision=prec)
    assert info["split_rows"] > 0


@pytest.mark.parametrize("iters", [16, 32])
def test_fp64_adaptive_iterates_with_split_rows_track_oracle(L, oracle_mod, iters):
    """Algorithm 5 with restarts and primal-weight updates, checks every 16
    iterations: the iterates agree with the oracle's to 1e-10 and so do the
    check records.  (The adaptive map amplifies rounding differences
    exponentially, see test_gpu_solver.py: beyond the first check periods
    parity is shown by replay there, on this LP among others.)"""
    lp = PROBS["ragged"]
    prob = L.Problem(lp)
    x, y, info, tr = prob.solve(tol=1e-13, max_iters=iters, trace_cap=64, check_every=16)
    xo, yo, io, tro = oracle_mod.solve(lp, tol=1e-13, max_iters=iters, trace_cap=64,
                                       check_every=16)
    assert info["split_rows"] > 0
    assert info["iters"] == io["iters"] == iters
    assert info["attempts"] == io["attempts"]
    assert info["norm_K"] == pytest.approx(io["norm_K"], rel=1e-12)
    assert rel(x, xo) <= 1e-10, rel(x, xo)
    assert rel(y, yo) <= 1e-10, rel(y, yo)
    assert len(tr) == len(tro)
    for a, b in zip(tr, tro):
        assert a["k"] == b["k"] and a["restart"] == b["restart"]
        assert a["eta"] == pytest.approx(b["eta"], rel=1e-10)
        assert a["omega"] == pytest.approx(b["omega"], rel=1e-10)


def test_adjoint_with_split_rows_matches_oracle(L, oracle_mod):
    """Unrolled fixed steps and their adjoint (lp_grad, FP64) on the ragged LP."""
    from paper_2508_16806_gb300 import autograd as AG
    lp = PROBS["ragged"]
    eta, omega = 0.9 / oracle_mod.power_norm(lp, 200), 1.0
    prob = L.Problem(lp)
    steps = 40
    xK, yK, (tau, sigma) = AG.unroll(prob, steps, eta=eta, omega=omega)
    xs, ys = oracle_mod.unrolled_forward(lp, tau, sigma, steps)
    assert rel(xK, xs[-1]) < 1e-12 and rel(yK, ys[-1]) < 1e-12
    g = np.random.default_rng(4).normal(size=lp.n)
    dc, dq, dv, _, _ = AG.grad(prob, steps, 10, g, eta=eta, omega=omega)
    oc, oq, ov = oracle_mod.unrolled_adjoint(lp, tau, sigma, steps, g)
    assert rel(dc, oc) < 1e-10, rel(dc, oc)
    assert rel(dq, oq) < 1e-10, rel(dq, oq)
    assert rel(dv, ov) < 1e-10, rel(dv, ov)


@pytest.mark.parametrize("name", ["ragged", "dispatch_mini"])
def test_fp32_fixed_steps_track_oracle(L, oracle_mod, name):
    """20 fixed FP32 steps (no scaling, eta and omega given): the FP32 iterates
    agree with the FP64 oracle's to 1e-5 relative, a few hundred FP32 roundings
    of steps whose operators have norm below one."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    eta = 0.9 / oracle_mod.power_norm(lp, 200)
    steps = 20
    x, y, info, _ = prob.solve(tol=0.0, max_iters=steps, check_every=1000, ruiz_iters=0,
                               adaptive_step=0, restarts=0, primal_weight_update=0,
                               eta0=eta, omega0=1.0, precision=1, polish_switch_tol=0.0)
    assert info["iters"] == steps and info["fp64_iters"] == 0
    xo, yo = oracle_mod.start_point(lp)
    for _ in range(steps):
        xo, yo = oracle_mod.pdhg_step(lp, xo, yo, eta, eta)
    assert rel(x, xo) < 1e-5, rel(x, xo)
    assert rel(y, yo) < 1e-5, rel(y, yo)


@pytest.mark.parametrize("name,tol", [("ragged", 1e-6), ("dispatch_mini", 1e-5)])
def test_mixed_solve_with_split_rows_reaches_tolerance(L, oracle_mod, name, tol):
    lp = PROBS[name]
    prob = L.Problem(lp)
    x, y, info, _ = prob.solve(tol=tol, precision=1, max_iters=2_000_000)
    assert info["status"] == L.LP_OPTIMAL
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= tol * (1 + 1e-6)


@pytest.mark.parametrize("prec", [0, 1])
def test_repeat_solves_with_split_rows_are_bitwise_identical(L, prec):
    lp = PROBS["ragged"]
    prob = L.Problem(lp)
    runs = [prob.solve(tol=1e-13, max_iters=2000, precision=prec, polish_switch_tol=0.0)
            for _ in range(2)]
    prob2 = L.Problem(lp)
    runs.append(prob2.solve(tol=1e-13, max_iters=2000, precision=prec, polish_switch_tol=0.0))
    x0, y0, i0, _ = runs[0]
    for x, y, info, _ in runs[1:]:
        assert info["attempts"] == i0["attempts"]
        assert np.array_equal(x, x0) and np.array_equal(y, y0)
