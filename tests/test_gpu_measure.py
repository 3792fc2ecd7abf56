"""The measurement hooks of the C ABI (lp_profile_step, lp_profile_gather) that
bench.py's per-kernel figures and roofline rest on.

- lp_profile_step's algorithmic bytes per launch follow the stated model: the
  K-side product streams the values and column indices of K (nnz (s + 4)
  bytes), its int64 row pointers, gathers x' once and reads / writes the dual
  step's row vectors (7 s + 1 bytes per row); the K^T side likewise, plus the
  primal step's column vectors (fused in FP32: x', c, l, u and the x-sum read,
  x'' and the x-sum written; unfused in FP64, where k_primal reads x, K^T y, c,
  l, u and writes x').
- lp_profile_gather times both sides, refuses blocks per SM outside 1..8, a
  handle without a solve and a scratch too small for its per-thread sums, and
  leaves the solver's results unchanged.
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


@pytest.fixture(scope="module")
def medium():
    return synth.power_law_lp(40000, 80000, 4, 600, seed=3)


@pytest.mark.parametrize("prec", [0, 1])
def test_profile_step_byte_model(L, medium, prec):
    lp = medium
    prob = L.Problem(lp)
    prob.solve(tol=1e-4, precision=prec, max_iters=64)
    ms, by = prob.profile_step(prec, reps=3)
    s = 8 if prec == 0 else 4
    m, n, nnz = lp.m, lp.n, lp.nnz
    k_side = nnz * (s + 4) + (m + 1) * 8 + n * s + m * (7 * s + 1)
    kt_base = nnz * (s + 4) + (n + 1) * 8 + m * s + n * s
    if prec == 1:     # FP32: primal step fused into the K^T launch
        want = [0.0, k_side, kt_base + 7 * n * s]
    else:             # FP64: k_primal after every K^T launch
        want = [6 * n * s, k_side, kt_base + 3 * n * s]
    assert [float(b) for b in by[:3]] == [float(w) for w in want]
    assert ms[1] > 0 and ms[2] > 0
    prob.close()


def test_profile_gather_times_and_refusals(L, medium):
    lp = medium
    prob = L.Problem(lp)
    # no solve on this handle yet: refused
    with pytest.raises(L.LpError):
        prob.profile_gather(L.LP_PREC_MIXED, reps=2, blocks_per_sm=4)
    x1, y1, i1, _ = prob.solve(tol=1e-5, precision=L.LP_PREC_MIXED, max_iters=2000)
    for bad in (0, 9):
        with pytest.raises(L.LpError):
            prob.profile_gather(L.LP_PREC_MIXED, reps=2, blocks_per_sm=bad)
    ms = prob.profile_gather(L.LP_PREC_MIXED, reps=3, blocks_per_sm=4)
    assert len(ms) == 2 and ms[0] > 0 and ms[1] > 0
    # the solver's results do not depend on the probe having run
    x2, y2, i2, _ = prob.solve(tol=1e-5, precision=L.LP_PREC_MIXED, max_iters=2000)
    assert i2["iters"] == i1["iters"]
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
    prob.close()


def test_profile_gather_refuses_small_scratch(L):
    """A problem whose scratch cannot hold one sum per probe thread is refused
    (the 200 x 400 LP: 152 SMs x 8 blocks x 256 threads of FP32 sums)."""
    prob = L.Problem(synth.small_dense_lp())
    prob.solve(tol=1e-4, precision=L.LP_PREC_MIXED, max_iters=64)
    with pytest.raises(L.LpError):
        prob.profile_gather(L.LP_PREC_MIXED, reps=2, blocks_per_sm=8)
    prob.close()
