"""GPU parity of Algorithm 7 (fishnet casting, Section 2.5) against the oracle.

The GPU advances all points together with block sparse products and takes the
cull decisions in FP64 like the oracle; with fixed-step PDHG the trajectories
track each other, so the per-round gaps and the surviving point agree to
rounding (1e-9 relative), and the surviving point is the same one.
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
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = {
    "lp200x400_P32_k20": (synth.small_dense_lp(), 32, 20),
    "ragged_P8_k10": (synth.ragged_lp(), 8, 10),
    "powerlaw_P64_k5": (synth.power_law_lp(4000, 8000, 4, 600, seed=11), 64, 5),
    "lp200x400_P16_k0": (synth.small_dense_lp(), 16, 0),
    "lp200x400_P2_k7": (synth.small_dense_lp(), 2, 7),
    "lp200x400_P1": (synth.small_dense_lp(), 1, 3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fishnet_matches_oracle(L, oracle_mod, name):
    lp, P, k = CASES[name]
    rng = np.random.default_rng(sum(map(ord, name)))
    G = rng.standard_normal((lp.n, P))
    Z = rng.standard_normal(max(oracle_mod.fishnet_draws(P), 1))
    ox, oy, og, orounds = oracle_mod.fishnet(lp, P, k, G, Z)
    gx, gy, gg, grounds = L.Problem(lp).fishnet(P, k, G, Z)
    assert grounds == orounds
    np.testing.assert_array_equal(np.isnan(gg), np.isnan(og))
    fin = np.isfinite(og)
    np.testing.assert_allclose(gg[fin], og[fin], rtol=1e-9, atol=1e-12)
    assert rel(gx, ox) <= 1e-9 and rel(gy, oy) <= 1e-9


@pytest.mark.parametrize("name", ["lp200x400_P32_k20", "ragged_P8_k10", "powerlaw_P64_k5"])
def test_fishnet_fp32_blocks_track_oracle(L, oracle_mod, name):
    """FP32 point blocks and products (FP64 gap reductions): the same rounds and
    survivors as the FP64 oracle on these draws, gaps and the surviving point
    within FP32 rounding of a fixed-step trajectory."""
    lp, P, k = CASES[name]
    rng = np.random.default_rng(sum(map(ord, name)))
    G = rng.standard_normal((lp.n, P))
    Z = rng.standard_normal(max(oracle_mod.fishnet_draws(P), 1))
    ox, oy, og, orounds = oracle_mod.fishnet(lp, P, k, G, Z)
    gx, gy, gg, grounds = L.Problem(lp).fishnet(P, k, G, Z, precision=L.LP_PREC_MIXED)
    assert grounds == orounds
    fin = np.isfinite(og)
    np.testing.assert_allclose(gg[fin], og[fin], rtol=1e-3, atol=1e-6)
    assert rel(gx, ox) <= 1e-3 and rel(gy, oy) <= 1e-3


def test_fishnet_device_inputs(L):
    torch = pytest.importorskip("torch")
    lp, P, k = CASES["ragged_P8_k10"]
    rng = np.random.default_rng(3)
    G = rng.standard_normal((lp.n, P))
    Z = rng.standard_normal(L.lp_fishnet_draws(P))
    prob = L.Problem(lp)
    hx, hy, _, _ = prob.fishnet(P, k, G, Z)
    Gd = torch.tensor(G, dtype=torch.float64, device="cuda")
    Zd = torch.tensor(Z, dtype=torch.float64, device="cuda")
    xd = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    yd = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    o = L.lp_opts_default()
    s = L.lp_fishnet(prob.handle, o, P, k, Gd.data_ptr(), Zd.data_ptr(), Z.size, xd.data_ptr(),
                     yd.data_ptr(), None, None, L.LP_MEM_DEVICE)
    assert s == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(xd.cpu().numpy(), hx)
    np.testing.assert_array_equal(yd.cpu().numpy(), hy)


def test_fishnet_rejects_bad_arguments(L):
    lp, _, _ = CASES["lp200x400_P32_k20"]
    prob = L.Problem(lp)
    G = np.zeros((lp.n, 32))
    with pytest.raises(L.LpError):
        prob.fishnet(32, 5, G, np.zeros(83))          # 84 draws needed
    with pytest.raises(L.LpError):
        prob.fishnet(3, 5, np.zeros((lp.n, 3)), [])   # not a power of two
    with pytest.raises(L.LpError):
        prob.fishnet(128, 5, np.zeros((lp.n, 128)), np.zeros(2000))


def test_fishnet_warm_start_solves(L, oracle_mod):
    lp = synth.ragged_lp()
    rng = np.random.default_rng(11)
    P = 32
    x0, y0, _, _ = L.Problem(lp).fishnet(P, 20, rng.standard_normal((lp.n, P)),
                                         rng.standard_normal(84))
    x, y, info, _ = L.Problem(lp).solve(tol=1e-6, x0=x0, y0=y0, max_iters=500000)
    assert info["status"] == L.LP_OPTIMAL
    k = oracle_mod.kkt(lp, x, y)
    assert max(k["rel_gap"], k["rel_pres"], k["rel_dres"]) <= 1e-6 * (1 + 1e-6)
