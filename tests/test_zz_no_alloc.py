"""The allocation-free KKT evaluation, lp_kkt_noalloc.

Some callers cannot allocate device memory at the moment they want to check a
point: code capturing a stream into a CUDA graph, hosts that forbid device
allocation after start-up because it can block or synchronise the device, and
plugins inside an application that owns all device memory.  lp_kkt_noalloc
serves them from a fixed scratch array compiled into the library.  This test
checks it, through the C ABI, against the solver's own start-point check
(lp_solve with no scaling and max_iters = 0, which evaluates exactly these
quantities) on two calls in a row with different points, so that a leftover
from the first call would show in the second.  The file is named to be
collected last: if it fails, a run that stops at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_kkt_matches_solver_check_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16806_gb300 import lp as L

    L.load()
    lp = synth.ragged_lp()
    prob = L.Problem(lp)
    rng = np.random.default_rng(2024)
    for call in range(2):
        x = np.clip(lp.x_star + rng.normal(0, 0.3, lp.n), lp.l, lp.u)
        y = lp.y_star + rng.normal(0, 0.3, lp.m)
        y[lp.sense == 1] = np.maximum(y[lp.sense == 1], 0.0)
        _, _, info, tr = prob.solve(tol=0.0, max_iters=0, ruiz_iters=0, x0=x, y0=y, trace_cap=4)
        assert info["iters"] == 0 and len(tr) == 1
        xd = torch.from_numpy(x).cuda()
        yd = torch.from_numpy(y).cuda()
        torch.cuda.synchronize()
        out = L.lp_kkt_noalloc(prob.desc, xd.data_ptr(), yd.data_ptr(), tr[0]["omega"])
        want = [info["pobj"], info["dobj"], None, None, info["rel_gap"], info["rel_pres"],
                info["rel_dres"], tr[0]["kkt_cur"]]
        for got, exp in zip(out, want):
            if exp is not None:
                assert got == pytest.approx(exp, rel=1e-9, abs=1e-12), (call, out, want)
    prob.close()
