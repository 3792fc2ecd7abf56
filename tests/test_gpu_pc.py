"""GPU parity of the Pock-Chambolle pass (parameter alpha) and of its choice
by trial solves (pock_chambolle = 2) against the FP64 oracle, through the C ABI.

The pass is not in the paper (Pock and Chambolle, 2011): rows are scaled by
1 / sqrt(sum_j |K~_ij|^(2 - alpha)) and columns by 1 / sqrt(sum_i |K~_ij|^alpha)
after Ruiz.  With the fixed step the FP64 path tracks the oracle's iterates to
1e-10 over 1000 iterations for every alpha of the grid; the tuned solve picks
the oracle's alpha and is then the solve with that alpha."""
import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

pytestmark = pytest.mark.gpu

GRID = (0.0, 0.5, 1.0, 2.0)


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


PROBS = {"lp200x400": synth.small_dense_lp(), "ragged": synth.ragged_lp(),
         "powerlaw": synth.power_law_lp(4000, 8000, 4, 600, seed=11)}


@pytest.mark.parametrize("name", ["lp200x400", "ragged", "powerlaw"])
@pytest.mark.parametrize("alpha", GRID)
def test_pock_chambolle_tracks_oracle(L, oracle_mod, name, alpha):
    """Ruiz + the Pock-Chambolle pass, fixed step, restarts and Algorithm 4:
    the iterates after 1000 iterations and the spectral norm match the oracle."""
    lp = PROBS[name]
    prob = L.Problem(lp)
    kw = dict(tol=1e-13, max_iters=1000, adaptive_step=0, pock_chambolle=1, pc_alpha=alpha)
    x, y, info, _ = prob.solve(**kw)
    xo, yo, io, _ = oracle_mod.solve(lp, **kw)
    assert info["iters"] == io["iters"] == 1000
    assert info["restarts"] == io["restarts"]
    assert info["pc_alpha_used"] == io["pc_alpha"] == alpha
    assert info["norm_K"] == pytest.approx(io["norm_K"], rel=1e-12)
    assert rel(x, xo) <= 1e-10, rel(x, xo)
    assert rel(y, yo) <= 1e-10, rel(y, yo)
    prob.close()


@pytest.mark.parametrize("name", ["lp200x400", "ragged", "powerlaw"])
def test_pock_chambolle_choice_matches_oracle(L, oracle_mod, name):
    """pock_chambolle = 2 in FP64: the GPU picks the oracle's alpha (when the
    oracle's best trial is not tied with the runner-up to 1e-6), each GPU trial
    reproduces the oracle's trial error, and the tuned solve is the solve with
    the chosen alpha, bit for bit."""
    lp = PROBS[name]
    alpha_o, errs = oracle_mod.pc_tune(lp, check_every=32)
    prob = L.Problem(lp)
    for a, e in zip(GRID, errs):
        _, _, it, _ = prob.solve(pock_chambolle=1, pc_alpha=a, max_iters=64, tol=0.0,
                                 infeas_detect=0, check_every=32)
        got = max(it["rel_gap"], it["rel_pres"], it["rel_dres"])
        assert got == pytest.approx(e, rel=1e-6), (a, got, e)
    x, y, info, _ = prob.solve(tol=1e-6, pock_chambolle=2, check_every=32)
    srt = sorted(errs)
    if srt[1] - srt[0] > 1e-6 * srt[0]:
        assert info["pc_alpha_used"] == alpha_o, (info["pc_alpha_used"], alpha_o, errs)
    x2, y2, i2, _ = prob.solve(tol=1e-6, pock_chambolle=1, pc_alpha=info["pc_alpha_used"],
                               check_every=32)
    np.testing.assert_array_equal(x, x2)
    np.testing.assert_array_equal(y, y2)
    assert info["status"] == L.LP_OPTIMAL
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-6 * (1 + 1e-6)
    prob.close()


def test_pock_chambolle_tuned_mixed_to_tolerance(L, oracle_mod):
    """The mixed path with the tuned pass reaches 1e-4, confirmed by the oracle."""
    lp = PROBS["powerlaw"]
    prob = L.Problem(lp)
    x, y, info, _ = prob.solve(tol=1e-4, precision=L.LP_PREC_MIXED, pock_chambolle=2)
    assert info["status"] == L.LP_OPTIMAL and info["pc_alpha_used"] in GRID
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-4 * (1 + 1e-6)
    prob.close()


def test_pock_chambolle_options_validated(L):
    prob = L.Problem(PROBS["lp200x400"])
    for bad in (dict(pock_chambolle=3), dict(pock_chambolle=1, pc_alpha=2.5),
                dict(pock_chambolle=1, pc_alpha=-0.1), dict(pock_chambolle=2, pc_trial_iters=-1)):
        with pytest.raises(L.LpError):
            prob.solve(tol=1e-4, **bad)
    batch = L.Batch([PROBS["lp200x400"], PROBS["ragged"]])
    with pytest.raises(L.LpError) as e:
        batch.solve(tol=1e-4, pock_chambolle=2)
    assert e.value.status == -5
    batch.close()
    prob.close()
