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
    # the FP32 iterates were judged with FP32 products; the FP64 re-evaluation may
    # differ in the last digits of a 1e-4 quantity
    assert worst <= 1.5 * tol, (k, info)
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
        assert max(kk["rel_gap"], kk["rel_pres"], kk["rel_dres"]) <= 1.5e-4
