"""Full-size workloads in the benchmark's launch configuration (mixed path to
1e-4), checked on what the FP64 oracle can compute at this size: one exact FP64
evaluation of the termination quantities (Section 2.3.2) of the returned point,
and, for the planted LP, the objective against the planted optimum."""
import time

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


def _check(L, oracle_mod, lp, tol, time_limit):
    prob = L.Problem(lp)
    t = time.time()
    x, y, info, tr = prob.solve(tol=tol, precision=L.LP_PREC_MIXED, time_limit_s=time_limit,
                                trace_cap=100000)
    dt = time.time() - t
    prob.close()
    assert info["status"] == L.LP_OPTIMAL, (info, dt)
    k = oracle_mod.kkt(lp, x, y)
    worst = max(k["rel_gap"], k["rel_pres"], k["rel_dres"])
    # the mixed path returns LP_OPTIMAL only after its FP64 check confirmed the
    # three relative errors: the oracle's own FP64 evaluation agrees to rounding
    assert worst <= tol * (1 + 1e-6), (k, info)
    # and the returned figures are that FP64 evaluation
    for key in ("rel_gap", "rel_pres", "rel_dres"):
        assert abs(info[key] - k[key]) <= 1e-9 * tol + 1e-6 * k[key], (key, info, k)
    return x, y, info, k


def test_powerlaw_1Mx2M_mixed_to_1e4(L, oracle_mod):
    lp = synth.power_law_lp()
    x, y, info, k = _check(L, oracle_mod, lp, 1e-4, 300)
    f = float(lp.c @ x)
    assert abs(f - lp.f_star) / (1 + abs(lp.f_star)) < 1e-3


def test_dispatch_615kx5k_mixed_to_1e4(L, oracle_mod):
    lp = synth.dispatch_lp()
    x, y, info, k = _check(L, oracle_mod, lp, 1e-4, 600)
    # the box is enforced in scaled FP32 coordinates: one FP32 rounding of x / C and back
    slack = 1e-6 * (1 + np.abs(lp.u))
    assert np.all(x >= lp.l - slack) and np.all(x <= lp.u + slack)


def test_batch_512_mixed_to_1e4(L, oracle_mod):
    """The 512-LP batch (m log-uniform on 500..50,000, n = 2m, 5-20 nonzeros per
    row): every LP reaches 1e-4; a sample is re-checked by the oracle in FP64."""
    lps = synth.batch_lps()
    batch = L.Batch(lps)
    out = batch.solve(tol=1e-4, precision=L.LP_PREC_MIXED, time_limit_s=600)
    batch.close()
    statuses = [info["status"] for _, _, info in out]
    assert all(s == L.LP_OPTIMAL for s in statuses), statuses
    rng = np.random.default_rng(0)
    for k in rng.choice(len(lps), 8, replace=False):
        x, y, info = out[k]
        kk = oracle_mod.kkt(lps[k], x, y)
        assert max(kk["rel_gap"], kk["rel_pres"], kk["rel_dres"]) <= 1e-4 * (1 + 1e-6)


def test_powerlaw_1Mx2M_halpern_mixed_to_1e4(L, oracle_mod):
    """Restarted Halpern PDHG on C1 in the bench leg's configuration (mixed path,
    FP32 phase with rho = 1/2): the oracle's FP64 evaluation of the returned
    point confirms 1e-4 and the objective matches the planted optimum."""
    lp = synth.power_law_lp()
    prob = L.Problem(lp)
    x, y, info, _ = prob.solve(tol=1e-4, precision=L.LP_PREC_MIXED, time_limit_s=300,
                               halpern=1)
    prob.close()
    assert info["status"] == L.LP_OPTIMAL, info
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-4 * (1 + 1e-6), k
    assert abs(float(lp.c @ x) - lp.f_star) / (1 + abs(lp.f_star)) < 1e-3


def test_powerlaw_1Mx2M_mixed_to_1e6(L, oracle_mod):
    """C1 to the tighter tolerance: the FP32 phase hands over at 1e-5 and the
    FP64 polish finishes; the oracle's FP64 evaluation confirms 1e-6."""
    lp = synth.power_law_lp()
    x, y, info, k = _check(L, oracle_mod, lp, 1e-6, 900)
    assert info["fp64_iters"] > 0 and info["precision_used"] == L.LP_PREC_FP64
    f = float(lp.c @ x)
    assert abs(f - lp.f_star) / (1 + abs(lp.f_star)) < 1e-5


def test_powerlaw_1Mx2M_fp64_to_1e4(L, oracle_mod):
    """The plain FP64 path on C1 (the comparison line of the benchmark), against
    the FP64 oracle's own run to 1e-4 on the same LP (oracle/reference_runs.json,
    written by oracle/run_to_tolerance.py): both stop at a 1e-4 point, so their
    objectives agree within the gap tolerance, and the iteration counts agree
    within a few check periods (Algorithm 5 amplifies rounding differences)."""
    import json
    import os
    lp = synth.power_law_lp()
    prob = L.Problem(lp)
    x, y, info, _ = prob.solve(tol=1e-4, precision=L.LP_PREC_FP64, time_limit_s=600)
    prob.close()
    assert info["status"] == L.LP_OPTIMAL, info
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-4 * (1 + 1e-6)
    assert abs(float(lp.c @ x) - lp.f_star) / (1 + abs(lp.f_star)) < 1e-3
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                        "reference_runs.json")
    runs = [r for r in json.load(open(path)) if r["tol"] == 1e-4 and r["nnz"] == lp.nnz]
    assert runs, "no oracle run to 1e-4 recorded for this LP"
    ref = runs[0]
    print("GPU FP64 iterations", info["iters"], "oracle", ref["iters"])
    assert abs(info["iters"] - ref["iters"]) <= 0.1 * ref["iters"]
    assert abs(info["pobj"] - ref["pobj"]) / (1 + abs(ref["pobj"])) <= 2e-4


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) /
                 max(np.linalg.norm(np.asarray(b)), 1e-300))


def test_adjoint_100kx200k_K500(L, oracle_mod):
    """C4 at full size: 500 unrolled fixed-step iterations, checkpoints every
    50.  The FP64 adjoint equals the oracle's FP64 unrolled adjoint; the FP32
    adjoint's distance to it is bounded (and printed)."""
    from paper_2508_16806_gb300 import autograd as AG
    lp, xt = synth.adjoint_lp()
    prob = L.Problem(lp)
    x64, _, (tau, sigma) = AG.unroll(prob, 500)
    g = 2.0 * (x64 - xt)
    d64 = AG.grad(prob, 500, 50, g)
    oc, oq, ov = oracle_mod.unrolled_adjoint(lp, tau, sigma, 500, g)
    for a, b in zip(d64[:3], (oc, oq, ov)):
        assert _rel(a, b) < 1e-9, _rel(a, b)
    d32 = AG.grad(prob, 500, 50, g, precision=L.LP_PREC_MIXED)
    errs = [_rel(a, b) for a, b in zip(d32[:3], d64[:3])]
    print("FP32 adjoint relative error (dc, dq, dvals):", errs)
    assert all(np.all(np.isfinite(a)) for a in d32[:3])
    assert max(errs) < 1e-2, errs


def test_adjoint_batch_of_64_at_m5000(L, oracle_mod):
    """C4's batch form: 64 instances at m = 5,000 (K = 500, checkpoints every
    50, FP32); two of them are compared with the FP64 adjoint."""
    from paper_2508_16806_gb300 import autograd as AG
    t = time.time()
    for k in range(64):
        lp, xt = synth.adjoint_lp(5000, 10000, 20, seed=20250820 + k)
        prob = L.Problem(lp)
        x32, _, _ = AG.unroll(prob, 500, precision=L.LP_PREC_MIXED)
        d32 = AG.grad(prob, 500, 50, 2.0 * (x32 - xt), precision=L.LP_PREC_MIXED)
        assert all(np.all(np.isfinite(a)) for a in d32[:3])
        if k < 2:
            d64 = AG.grad(prob, 500, 50, 2.0 * (x32 - xt))
            assert max(_rel(a, b) for a, b in zip(d32[:3], d64[:3])) < 1e-2
        prob.close()
    print("64 adjoints at m=5000:", time.time() - t, "s")
