"""GPU parity of Algorithm 6 (infeasibility detection, Section 2.4.5).

The CUDA check kernels evaluate the certificate tests on the last step's
differences of the stored scaled iterates and products; the oracle recomputes
them from the unscaled problem.  Both must classify the same problems the same
way (HiGHS gives the expected class in the oracle's own pins); with the fixed
step, where the two trajectories track each other, the detection lands within
one check period of the oracle's.
"""
import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

pytestmark = pytest.mark.gpu

CHECK = 64


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16806_gb300 import lp as L
    L.load()
    return L


INF = np.inf


def _cases():
    small = synth.small_dense_lp()
    ragged = synth.ragged_lp()
    return {
        "P2": (synth.from_dense([[1, 1], [1, -1]], [1, 1], [0, 0], [3, 0], [0, 0], [1, 1]), 2),
        "D2": (synth.from_dense([[1, -1], [1, 1]], [0, 1], [-1, 0], [0, 1], [0, 0], [INF, INF]), 3),
        "contradiction": (synth.contradictory_rows_lp(small), 2),
        "contradiction_gap0.1": (synth.contradictory_rows_lp(small, seed=5, gap=0.1), 2),
        "unbounded_col": (synth.unbounded_column_lp(small), 3),
        "unbounded_col9": (synth.unbounded_column_lp(small, seed=9), 3),
        "ragged_contradiction": (synth.contradictory_rows_lp(ragged, seed=3, width=40), 2),
        "ragged_unbounded": (synth.unbounded_column_lp(ragged, seed=4, width=30), 3),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_fixed_step_detection_matches_oracle(L, oracle_mod, name):
    lp, want = CASES[name]
    kw = dict(tol=1e-8, max_iters=60000, check_every=CHECK, adaptive_step=0, infeas_detect=1,
              infeas_tol=1e-6)
    _, _, oi, _ = oracle_mod.solve(lp, **kw)
    assert oi["status"] == want
    _, _, gi, _ = L.Problem(lp).solve(**kw)
    assert gi["status"] == want, gi
    assert abs(gi["iters"] - oi["iters"]) <= CHECK, (gi["iters"], oi["iters"])


@pytest.mark.parametrize("name", list(CASES))
def test_adaptive_detection(L, name):
    lp, want = CASES[name]
    _, _, gi, _ = L.Problem(lp).solve(tol=1e-8, max_iters=200000)
    assert gi["status"] == want, gi


@pytest.mark.parametrize("name", ["contradiction", "unbounded_col", "ragged_contradiction",
                                  "ragged_unbounded"])
def test_mixed_precision_detection(L, name):
    lp, want = CASES[name]
    _, _, gi, _ = L.Problem(lp).solve(tol=1e-8, max_iters=200000, precision=L.LP_PREC_MIXED)
    assert gi["status"] == want, gi


def test_detection_off_runs_to_limit(L):
    lp, _ = CASES["contradiction"]
    _, _, gi, _ = L.Problem(lp).solve(tol=1e-8, max_iters=3000, infeas_detect=0)
    assert gi["status"] == L.LP_ITERATION_LIMIT and gi["iters"] == 3000


def test_no_false_positive_on_feasible(L, oracle_mod):
    for lp in (synth.small_dense_lp(), synth.ragged_lp(),
               synth.power_law_lp(4000, 8000, 4, 600, seed=11)):
        x, y, gi, _ = L.Problem(lp).solve(tol=1e-7, max_iters=500000)
        assert gi["status"] == L.LP_OPTIMAL, gi
        k = oracle_mod.kkt(lp, x, y)
        assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-7 * (1 + 1e-6)


def test_batch_mixes_statuses(L):
    """A batch of feasible, primal- and dual-infeasible LPs: each LP stops on
    its own verdict and the others run on."""
    lps = [CASES["contradiction"][0], synth.small_dense_lp(), CASES["unbounded_col"][0],
           synth.ragged_lp(), CASES["ragged_contradiction"][0], CASES["P2"][0]]
    want = [2, 1, 3, 1, 2, 2]
    batch = L.Batch(lps)
    out = batch.solve(tol=1e-7, max_iters=200000)
    for k, (x, y, info) in enumerate(out):
        assert info["status"] == want[k], (k, info)
    batch.close()
