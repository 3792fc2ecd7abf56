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
