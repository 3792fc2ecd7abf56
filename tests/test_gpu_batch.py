"""Batched restarted PDHG (lp_batch_create / lp_batch_solve / lp_solve_batch):
every LP of a batch follows the same per-LP method as lp_solve, checked against
single solves, against the FP64 oracle's own runs and against its KKT
evaluation."""
import ctypes as C

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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def mixed_lps():
    rng = np.random.default_rng(3)
    return [synth.small_dense_lp(), synth.ragged_lp(),
            synth.power_law_lp(4000, 8000, 4, 600, seed=11),
            synth.shuffle_sense(synth.small_dense_lp(), 3),
            synth.random_planted(700, 1400, lengths=rng.integers(5, 21, 700), seed=5),
            synth.small_dense_lp(99)]


LPS = mixed_lps()


@pytest.mark.parametrize("iters", [1, 64, 1000])
def test_batch_tracks_single_solves_fixed_step(L, iters):
    """Fixed-step restarted PDHG: each LP of the batch reaches the same
    iterate (1e-10 relative) with the same decisions as its single solve."""
    batch = L.Batch(LPS)
    out = batch.solve(tol=1e-13, max_iters=iters, adaptive_step=0)
    for lp, (x, y, info) in zip(LPS, out):
        xs, ys, si, _ = L.Problem(lp).solve(tol=1e-13, max_iters=iters, adaptive_step=0)
        assert info["status"] == si["status"] == L.LP_ITERATION_LIMIT
        assert info["iters"] == si["iters"] == iters
        assert info["restarts"] == si["restarts"]
        assert info["norm_K"] == pytest.approx(si["norm_K"], rel=1e-12)
        assert rel(x, xs) <= 1e-10 and rel(y, ys) <= 1e-10
    batch.close()


@pytest.mark.parametrize("iters", [64, 1000])
def test_batch_tracks_oracle_fixed_step(L, oracle_mod, iters):
    """Fixed-step restarted PDHG: each LP of the batch matches the FP64 oracle's
    own run directly (iterates to 1e-10 relative, same restarts, the same
    Algorithm 2 norm to 1e-12)."""
    batch = L.Batch(LPS)
    out = batch.solve(tol=1e-13, max_iters=iters, adaptive_step=0)
    for lp, (x, y, info) in zip(LPS, out):
        xo, yo, io, _ = oracle_mod.solve(lp, tol=1e-13, max_iters=iters, adaptive_step=0,
                                         trace_cap=4)
        assert info["iters"] == io["iters"] == iters
        assert info["restarts"] == io["restarts"]
        assert info["norm_K"] == pytest.approx(io["norm_K"], rel=1e-12)
        assert rel(x, xo) <= 1e-10, rel(x, xo)
        assert rel(y, yo) <= 1e-10, rel(y, yo)
    batch.close()


def test_batch_adaptive_to_tolerance(L, oracle_mod):
    batch = L.Batch(LPS)
    out = batch.solve(tol=1e-6, max_iters=500000)
    for lp, (x, y, info) in zip(LPS, out):
        assert info["status"] == L.LP_OPTIMAL, info
        k = oracle_mod.kkt(lp, x, y)
        assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-6 * (1 + 1e-6)
        assert 0 < info["solve_s"]
    batch.close()


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_batch_mixed_precision(L, oracle_mod, tol):
    """The batched mixed path: FP32 phase, then the FP64 check (and FP64
    iterations where needed) of every LP declared optimal; the oracle's FP64
    evaluation of each returned point confirms the tolerance, and the reported
    errors are that FP64 evaluation."""
    lps = synth.batch_lps(count=24, m_lo=500, m_hi=5000)
    batch = L.Batch(lps)
    out = batch.solve(tol=tol, precision=L.LP_PREC_MIXED, max_iters=500000)
    for lp, (x, y, info) in zip(lps, out):
        assert info["status"] == L.LP_OPTIMAL, info
        k = oracle_mod.kkt(lp, x, y)
        assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= tol * (1 + 1e-6), (k, info)
        for f in ("rel_gap", "rel_pres", "rel_dres"):
            assert abs(info[f] - k[f]) <= 1e-9 * tol + 1e-6 * k[f], (f, info, k)
        assert abs(float(lp.c @ x) - lp.f_star) / (1 + abs(lp.f_star)) < 1e-2
        if tol < 1e-5:
            assert info["fp64_iters"] > 0 and info["precision_used"] == L.LP_PREC_FP64
    batch.close()


def test_lp_solve_batch_one_shot(L):
    probs = [L.Problem(lp) for lp in LPS[:3]]
    res = (L.LpResult * 3)()
    xs = [np.empty(p.n) for p in probs]
    for k, p in enumerate(probs):
        res[k].x = xs[k].ctypes.data
        res[k].memory_space = L.LP_MEM_HOST
    o = L.lp_opts_default(tol=1e-6)
    assert L.lp_solve_batch([p.handle for p in probs], o, res) == 0
    for k in range(3):
        assert res[k].status == L.LP_OPTIMAL
        xk, _, sk, _ = probs[k].solve(tol=1e-6)
        assert abs(float(LPS[k].c @ xs[k]) - float(LPS[k].c @ xk)) <= 1e-5 * (1 + abs(float(LPS[k].c @ xk)))


def test_batch_autotuned_schedules(L, oracle_mod):
    batch = L.Batch(LPS)
    out = batch.solve(tol=1e-6, max_iters=500000, autotune=1)
    for lp, (x, y, info) in zip(LPS, out):
        assert info["status"] == L.LP_OPTIMAL, info
        k = oracle_mod.kkt(lp, x, y)
        assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-6 * (1 + 1e-6)
    batch.close()
