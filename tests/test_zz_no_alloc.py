"""The allocation-free KKT evaluation, lp_kkt_noalloc.

Some callers cannot allocate device memory at the moment they want to check a
point: hosts that forbid device allocation after start-up because it can block
or synchronise the device, and plugins inside an application that owns all
device memory.  lp_kkt_noalloc serves them from a fixed scratch array compiled
into the library.  These tests call it through the C ABI and check:

- all eight outputs against the FP64 oracle's evaluation of the same point
  (Section 2.3.2 termination quantities and KKT_omega), on two calls in a row
  with different points, so that a leftover from the first call would show in
  the second;
- the same figures against the solver's own start-point check;
- the rejections: a problem larger than the fixed scratch, an out-of-range
  column index or row pointer (found on the device), and a stream that is being
  captured into a CUDA graph (refused before anything is launched); a good call
  after each rejection still gives the right answer.

The file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2508_16806_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("pobj", "dobj", "pres", "dres", "rel_gap", "rel_pres", "rel_dres", "kkt_omega")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16806_gb300 import lp as L
    L.load()
    lp = synth.ragged_lp()
    prob = L.Problem(lp)
    yield torch, L, lp, prob
    prob.close()


def _point(lp, rng):
    x = np.clip(lp.x_star + rng.normal(0, 0.3, lp.n), lp.l, lp.u)
    y = lp.y_star + rng.normal(0, 0.3, lp.m)
    y[lp.sense == 1] = np.maximum(y[lp.sense == 1], 0.0)
    return x, y


def _call(torch, L, desc, x, y, omega, stream=None):
    """Raw status and outputs of one call (no exception on a refusal)."""
    import ctypes as C
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    torch.cuda.synchronize()
    out = (C.c_double * 8)()
    s = L.load().lp_kkt_noalloc(C.byref(desc), xd.data_ptr(), yd.data_ptr(), omega,
                                C.cast(out, C.c_void_p), C.c_void_p(stream or 0))
    return s, list(out)


def _check_against_oracle(oracle_mod, lp, x, y, omega, got):
    want = oracle_mod.kkt(lp, x, y, omega=omega)
    for name, g in zip(FIELDS, got):
        assert g == pytest.approx(want[name], rel=1e-9, abs=1e-12), (name, g, want[name])


def test_noalloc_matches_oracle_on_two_calls(env, oracle_mod):
    torch, L, lp, prob = env
    rng = np.random.default_rng(2024)
    for call, omega in enumerate((1.0, 2.5)):
        x, y = _point(lp, rng)
        s, out = _call(torch, L, prob.desc, x, y, omega)
        assert s == 0, L.STATUS.get(s, s)
        _check_against_oracle(oracle_mod, lp, x, y, omega, out)


def test_noalloc_matches_solver_start_check(env):
    """The solver's start-point check (no scaling, max_iters = 0) evaluates the
    same quantities of the same point."""
    torch, L, lp, prob = env
    rng = np.random.default_rng(7)
    x, y = _point(lp, rng)
    _, _, info, tr = prob.solve(tol=0.0, max_iters=0, ruiz_iters=0, x0=x, y0=y, trace_cap=4)
    assert info["iters"] == 0 and len(tr) == 1
    s, out = _call(torch, L, prob.desc, x, y, tr[0]["omega"])
    assert s == 0
    want = [info["pobj"], info["dobj"], None, None, info["rel_gap"], info["rel_pres"],
            info["rel_dres"], tr[0]["kkt_cur"]]
    for got, exp in zip(out, want):
        if exp is not None:
            assert got == pytest.approx(exp, rel=1e-9, abs=1e-12), (out, want)


def test_noalloc_rejects_problem_above_scratch(env, oracle_mod):
    """m + n + 1800 above LP_KKT_NOALLOC_MAX_DOUBLES is refused on the host,
    before any array is read; a good call afterwards is unaffected."""
    torch, L, lp, prob = env
    limit = 1048576
    d = prob.desc
    big = L.LpDesc(limit // 2, limit // 2, d.nnz, d.row_ptr, d.col_idx, d.vals, d.sense, d.c,
                   d.q, d.l, d.u, d.memory_space, 0)
    x, y = _point(lp, np.random.default_rng(3))
    s, _ = _call(torch, L, big, x, y, 1.0)
    assert s == L.LP_INVALID_ARGUMENT
    s, out = _call(torch, L, prob.desc, x, y, 1.0)
    assert s == 0
    _check_against_oracle(oracle_mod, lp, x, y, 1.0, out)


@pytest.mark.parametrize("what", ["col_idx", "row_ptr"])
def test_noalloc_rejects_bad_index(env, oracle_mod, what):
    """An out-of-range column index, or a row pointer past nnz, is skipped by
    the device range checks and turns the call into LP_INVALID_ARGUMENT; the next
    good call (which clears the flag) gives the oracle's figures."""
    torch, L, lp, prob = env
    ci = np.ascontiguousarray(lp.col_idx, np.int32).copy()
    rp = np.ascontiguousarray(lp.row_ptr, np.int64).copy()
    if what == "col_idx":
        ci[len(ci) // 2] = lp.n + 7
    else:
        rp[1] = lp.nnz + 5
    ci_d = torch.from_numpy(ci).cuda()
    rp_d = torch.from_numpy(rp).cuda()
    d = prob.desc
    bad = L.LpDesc(d.m, d.n, d.nnz, rp_d.data_ptr(), ci_d.data_ptr(), d.vals, d.sense, d.c, d.q,
                   d.l, d.u, d.memory_space, 0)
    x, y = _point(lp, np.random.default_rng(5))
    s, _ = _call(torch, L, bad, x, y, 1.0)
    assert s == L.LP_INVALID_ARGUMENT
    s, out = _call(torch, L, prob.desc, x, y, 1.0)
    assert s == 0
    _check_against_oracle(oracle_mod, lp, x, y, 1.0, out)


def test_noalloc_refuses_capturing_stream(env, oracle_mod):
    """Called on a stream that is being captured, the entry point returns
    LP_NOT_SUPPORTED without launching anything, and the capture stays valid."""
    torch, L, lp, prob = env
    x, y = _point(lp, np.random.default_rng(11))
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    a = torch.zeros(4, device="cuda")
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    import ctypes as C
    out = (C.c_double * 8)()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        a.add_(1.0)
        s = L.load().lp_kkt_noalloc(C.byref(prob.desc), xd.data_ptr(), yd.data_ptr(), 1.0,
                                    C.cast(out, C.c_void_p),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert s == L.LP_NOT_SUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert float(a[0]) == 1.0
    s, out2 = _call(torch, L, prob.desc, x, y, 1.0)
    assert s == 0
    _check_against_oracle(oracle_mod, lp, x, y, 1.0, out2)
