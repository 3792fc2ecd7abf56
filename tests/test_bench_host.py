"""Host-side logic of bench.py (no GPU): the fishnet round schedule matches the
draw count of Algorithm 7 in the oracle and in the C ABI, and the block-product
byte model scales with the number of points as its terms say."""
import numpy as np
import pytest

import bench
from paper_2508_16806_gb300 import synth


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16, 32, 64])
def test_fishnet_schedule_matches_draws(oracle_mod, P):
    sched = bench.fishnet_schedule(P)
    # repopulations happen at odd rounds with more than two points entering
    draws = sum((c // 2) ** 2 for i, c in enumerate(sched) if i % 2 == 1 and c > 2)
    assert draws == oracle_mod.fishnet_draws(P)
    from paper_2508_16806_gb300 import lp as L
    assert draws == L.lp_fishnet_draws(P)
    assert all(c >= 2 for c in sched) and (P == 1 or sched[0] == P)


def test_spmm_bytes_model():
    lp = synth.small_dense_lp()
    b1, b2 = bench.spmm_bytes(lp, 1), bench.spmm_bytes(lp, 2)
    # one more point adds one gathered value per nonzero on each side and the
    # epilogue's point-block traffic (2 n + 4 m values)
    assert b2 - b1 == 2 * lp.nnz * 4 + 4 * (2 * lp.n + 4 * lp.m)
    assert bench.spmm_bytes(lp, 32, 8) > bench.spmm_bytes(lp, 32, 4)


def test_oracle_timer_pieces_and_estimate(oracle_mod):
    """The CPU baseline's arithmetic: every measured piece is positive, the
    per-iteration time comes from the samples, and the time-to-tolerance
    estimate is Ruiz + 100 power iterations + N iterations + one check per 64."""
    lp = synth.small_dense_lp()
    ot = bench.OracleTimer(lp)
    ot.setup()
    for _ in range(3):
        assert ot.sample() > 0
    assert len(ot.t_iter) == 3 and ot.iter_s() > 0
    for attr in ("t_ruiz", "t_pow", "t_start", "t_check"):
        assert getattr(ot, attr) >= 0
    n = 640
    want = ot.t_ruiz + 100 * ot.t_pow + n * ot.iter_s() + (n / 64 + 1) * ot.t_check
    assert ot.estimate(n) == pytest.approx(want)
    assert ot.estimate(2 * n) > ot.estimate(n)
    assert "iterations/s" in ot.describe(n, "test")


def test_reference_iterations_match_by_size(oracle_mod):
    """A stored oracle run is used only for the LP it was made on; a small LP
    gets its iteration count from an oracle run to tolerance here."""
    lp = synth.small_dense_lp()
    iters, src = bench.reference_iterations(1e-4, lp)
    _, _, info, _ = oracle_mod.solve(lp, tol=1e-4, max_iters=2_000_000)
    assert iters == info["iters"] and "this process" in src
