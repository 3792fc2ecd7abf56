"""Python access to the FP64 CPU oracle (``pdhg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA solver never imports this
package, and this package imports nothing from the solver.

``build()`` compiles ``pdhg_oracle.c`` with gcc into ``liboracle.so`` next to
it (plain C, -O2, no architecture flags, so it builds the same on x86-64 and
aarch64).  Every wrapper below converts numpy arrays and calls the C function
of the same role; see the C file for the paper passages each follows.

Parity status: every function is pinned by the not-gpu tests.  Algorithm 4
and Algorithm 5 are pinned by hand-worked values (tests/golden/step_rules_hand.json)
both as functions and at their call sites inside ``solve``, by the invariant
that every accepted step size satisfies eta <= eta_bar, and by planted-mistake
tests that compile broken copies of the oracle and check that the pins fail.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdhg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc) if it is missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Lp(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("vals", C.c_void_p),
                ("sense", C.c_void_p), ("c", C.c_void_p), ("q", C.c_void_p),
                ("l", C.c_void_p), ("u", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int64), ("check_every", C.c_int32),
                ("ruiz_iters", C.c_int32), ("ruiz_tol", C.c_double),
                ("pock_chambolle", C.c_int32), ("power_iters", C.c_int32),
                ("adaptive_step", C.c_int32), ("primal_weight_update", C.c_int32),
                ("restarts", C.c_int32), ("eta_scale", C.c_double),
                ("beta_sufficient", C.c_double), ("beta_necessary", C.c_double),
                ("beta_artificial", C.c_double), ("eps_zero", C.c_double),
                ("x0", C.c_void_p), ("y0", C.c_void_p),
                ("omega0", C.c_double), ("eta0", C.c_double),
                ("infeas_detect", C.c_int32), ("pad", C.c_int32), ("infeas_tol", C.c_double),
                ("halpern", C.c_int32), ("pad2", C.c_int32), ("reflect", C.c_double),
                ("pc_alpha", C.c_double), ("pc_trial_iters", C.c_int32), ("pad3", C.c_int32),
                ("replay", C.c_void_p), ("replay_len", C.c_int64),
                ("replay_checks", C.c_void_p), ("replay_checks_len", C.c_int64)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("pad", C.c_int32), ("iters", C.c_int64),
                ("attempts", C.c_int64), ("restarts", C.c_int64),
                ("pobj", C.c_double), ("dobj", C.c_double), ("rel_gap", C.c_double),
                ("rel_pres", C.c_double), ("rel_dres", C.c_double),
                ("omega", C.c_double), ("eta", C.c_double), ("norm_K", C.c_double),
                ("pc_alpha", C.c_double)]


TRACE_FIELDS = ("k", "attempts", "restart", "cand_is_avg", "omega", "eta",
                "kkt_cur", "kkt_avg", "rel_gap", "rel_pres", "rel_dres", "kkt_cand",
                "fpr", "fpr0", "own_restart", "own_cand_is_avg", "kkt_anchor", "kkt_prev")

DEFAULTS = dict(tol=1e-4, max_iters=100000, check_every=64, ruiz_iters=10, ruiz_tol=1e-4,
                pock_chambolle=0, power_iters=100, adaptive_step=1, primal_weight_update=1,
                restarts=1, eta_scale=0.9, beta_sufficient=0.2, beta_necessary=0.8,
                beta_artificial=0.36, eps_zero=1e-6, omega0=0.0, eta0=0.0,
                infeas_detect=1, infeas_tol=1e-6, halpern=0, reflect=1.0, pc_alpha=1.0,
                pc_trial_iters=0)


def _bind(lib):
    """Declares the C signatures on a loaded oracle library."""
    if True:
        _lib = lib
        P = C.POINTER
        _lib.orc_spmv.argtypes = [P(_Lp), C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_spmv_t.argtypes = [P(_Lp), C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_ruiz.argtypes = [P(_Lp), C.c_int32, C.c_double, C.c_int32, C.c_double,
                                  C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_ruiz.restype = C.c_int
        _lib.orc_power_norm.argtypes = [P(_Lp), C.c_void_p, C.c_int32]
        _lib.orc_power_norm.restype = C.c_double
        _lib.orc_proj_lambda.argtypes = [C.c_int64] + [C.c_void_p] * 4
        _lib.orc_kkt.argtypes = [P(_Lp)] + [C.c_void_p] * 7 + [C.c_double, C.c_void_p]
        _lib.orc_pdhg_step.argtypes = [P(_Lp)] + [C.c_void_p] * 7 + [C.c_double, C.c_double,
                                                                     C.c_void_p, C.c_void_p]
        _lib.orc_solve.argtypes = [P(_Lp), P(_Opts), C.c_void_p, C.c_void_p, P(_Info),
                                   C.c_void_p, C.c_int64, P(C.c_int64)]
        _lib.orc_solve.restype = C.c_int
        _lib.orc_infeasibility.argtypes = [P(_Lp), C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                           C.c_void_p]
        _lib.orc_infeasibility.restype = C.c_int
        _lib.orc_fishnet.argtypes = [P(_Lp), P(_Opts), C.c_int32, C.c_int32, C.c_void_p,
                                     C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                     P(C.c_int32)]
        _lib.orc_fishnet.restype = C.c_int
        _lib.orc_pnorm2.argtypes = [P(_Lp)] + [C.c_void_p] * 3 + [C.c_double, C.c_double]
        _lib.orc_pnorm2.restype = C.c_double
        _lib.orc_halpern_step.argtypes = ([P(_Lp)] + [C.c_void_p] * 9 +
                                          [C.c_double, C.c_double, C.c_int64, C.c_double] +
                                          [C.c_void_p] * 4)
        _lib.orc_halpern_step.restype = C.c_double
        _lib.orc_unrolled_forward.argtypes = [P(_Lp), C.c_double, C.c_double, C.c_int32,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_unrolled_adjoint.argtypes = [P(_Lp), C.c_double, C.c_double, C.c_int32,
                                              C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_solve_logged.argtypes = [P(_Lp), P(_Opts), C.c_void_p, C.c_void_p, P(_Info),
                                          C.c_void_p, C.c_int64, P(C.c_int64), C.c_void_p,
                                          C.c_int64, P(C.c_int64)]
        _lib.orc_solve_logged.restype = C.c_int
        _lib.orc_primal_weight.argtypes = [C.c_double] * 4
        _lib.orc_primal_weight.restype = C.c_double
        _lib.orc_step_rule.argtypes = [C.c_double] * 5 + [C.c_int64, P(C.c_double),
                                                           P(C.c_double)]
        _lib.orc_step_rule.restype = C.c_int
        _lib.orc_pc_tune.argtypes = [P(_Lp), P(_Opts), C.c_void_p]
        _lib.orc_pc_tune.restype = C.c_double
    return lib


_override = None   # a library loaded by use_library (planted-mistake tests)


def _load():
    global _lib
    if _override is not None:
        return _override
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


class use_library:
    """Context manager: every wrapper of this module calls the oracle library
    at `path` (a separately compiled copy of pdhg_oracle.c) instead of the
    default one.  The planted-mistake tests use it to run the pins against
    deliberately broken copies of the oracle."""

    def __init__(self, path):
        self.lib = _bind(C.CDLL(path))

    def __enter__(self):
        global _override
        self.prev = _override
        _override = self.lib
        return self.lib

    def __exit__(self, *exc):
        global _override
        _override = self.prev
        return False


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class _Bound:
    """Holds contiguous copies of an LP's arrays and the C struct over them."""

    def __init__(self, lp, vals=None, c=None, q=None, l=None, u=None):
        self.rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
        self.v = _f64(lp.vals if vals is None else vals)
        self.s = np.ascontiguousarray(lp.sense, dtype=np.uint8)
        self.c = _f64(lp.c if c is None else c)
        self.q = _f64(lp.q if q is None else q)
        self.l = _f64(lp.l if l is None else l)
        self.u = _f64(lp.u if u is None else u)
        self.st = _Lp(lp.m, lp.n, _ptr(self.rp), _ptr(self.ci), _ptr(self.v), _ptr(self.s),
                      _ptr(self.c), _ptr(self.q), _ptr(self.l), _ptr(self.u))
        self.m, self.n = lp.m, lp.n


def spmv(lp, x, vals=None):
    b = _Bound(lp, vals)
    x = _f64(x)
    out = np.empty(lp.m)
    _load().orc_spmv(C.byref(b.st), _ptr(b.v), _ptr(x), _ptr(out))
    return out


def spmv_t(lp, y, vals=None):
    b = _Bound(lp, vals)
    y = _f64(y)
    out = np.empty(lp.n)
    _load().orc_spmv_t(C.byref(b.st), _ptr(b.v), _ptr(y), _ptr(out))
    return out


def ruiz(lp, iters=10, tol=1e-4, pock_chambolle=False, pc_alpha=1.0):
    """Algorithm 3 (and the Pock-Chambolle pass with parameter pc_alpha).
    Returns (scaled values, R, C, passes) with K~ = diag(R) K diag(C)."""
    b = _Bound(lp)
    vs = np.empty(lp.nnz)
    R = np.empty(lp.m)
    Cc = np.empty(lp.n)
    passes = _load().orc_ruiz(C.byref(b.st), iters, tol, int(pock_chambolle), float(pc_alpha),
                              _ptr(vs), _ptr(R), _ptr(Cc))
    return vs, R, Cc, passes


def power_norm(lp, iters=100, vals=None):
    """Algorithm 2."""
    b = _Bound(lp, vals)
    return float(_load().orc_power_norm(C.byref(b.st), _ptr(b.v), iters))


def proj_lambda(l, u, v):
    l, u, v = _f64(l), _f64(u), _f64(v)
    out = np.empty_like(v)
    _load().orc_proj_lambda(v.shape[0], _ptr(l), _ptr(u), _ptr(v), _ptr(out))
    return out


KKT_FIELDS = ("pobj", "dobj", "pres", "dres", "rel_gap", "rel_pres", "rel_dres", "kkt_omega")


def kkt(lp, x, y, omega=1.0, vals=None, c=None, q=None, l=None, u=None):
    """Termination quantities (Section 2.3.2) and KKT_omega (Section 2.4.2)."""
    b = _Bound(lp, vals, c, q, l, u)
    x, y = _f64(x), _f64(y)
    out = np.empty(8)
    _load().orc_kkt(C.byref(b.st), _ptr(b.v), _ptr(b.c), _ptr(b.q), _ptr(b.l), _ptr(b.u),
                    _ptr(x), _ptr(y), omega, _ptr(out))
    return dict(zip(KKT_FIELDS, out.tolist()))


def pdhg_step(lp, x, y, tau, sigma, vals=None, c=None, q=None, l=None, u=None):
    """One step of Algorithm 1 (theta = 1)."""
    b = _Bound(lp, vals, c, q, l, u)
    x, y = _f64(x), _f64(y)
    xn = np.empty(lp.n)
    yn = np.empty(lp.m)
    _load().orc_pdhg_step(C.byref(b.st), _ptr(b.v), _ptr(b.c), _ptr(b.q), _ptr(b.l),
                          _ptr(b.u), _ptr(x), _ptr(y), tau, sigma, _ptr(xn), _ptr(yn))
    return xn, yn


def pnorm2(lp, dx, dy, tau, sigma, vals=None):
    """||(dx, dy)||_P^2 = ||dx||^2 / tau + ||dy||^2 / sigma + 2 dy^T K dx."""
    b = _Bound(lp, vals)
    dx, dy = _f64(dx), _f64(dy)
    return float(_load().orc_pnorm2(C.byref(b.st), _ptr(b.v), _ptr(dx), _ptr(dy), tau, sigma))


def halpern_step(lp, x, y, xanc, yanc, tau, sigma, k, rho, vals=None, c=None, q=None, l=None,
                 u=None):
    """One inner step of restarted Halpern PDHG: returns (T(z), z_next, ||z - T(z)||_P)
    with T(z) = (xh, yh) and z_next = (xn, yn)."""
    b = _Bound(lp, vals, c, q, l, u)
    x, y, xa, ya = _f64(x), _f64(y), _f64(xanc), _f64(yanc)
    xh, yh, xn, yn = np.empty(lp.n), np.empty(lp.m), np.empty(lp.n), np.empty(lp.m)
    r = _load().orc_halpern_step(C.byref(b.st), _ptr(b.v), _ptr(b.c), _ptr(b.q), _ptr(b.l),
                                 _ptr(b.u), _ptr(x), _ptr(y), _ptr(xa), _ptr(ya), tau, sigma,
                                 int(k), float(rho), _ptr(xh), _ptr(yh), _ptr(xn), _ptr(yn))
    return (xh, yh), (xn, yn), float(r)


def _opts(o, x0a=None, y0a=None, replay=None, replay_checks=None):
    return _Opts(o["tol"], int(o["max_iters"]), int(o["check_every"]), int(o["ruiz_iters"]),
                 o["ruiz_tol"], int(o["pock_chambolle"]), int(o["power_iters"]),
                 int(o["adaptive_step"]), int(o["primal_weight_update"]), int(o["restarts"]),
                 o["eta_scale"], o["beta_sufficient"], o["beta_necessary"],
                 o["beta_artificial"], o["eps_zero"],
                 None if x0a is None else _ptr(x0a), None if y0a is None else _ptr(y0a),
                 o["omega0"], o["eta0"], int(o["infeas_detect"]), 0, o["infeas_tol"],
                 int(o["halpern"]), 0, float(o["reflect"]), float(o["pc_alpha"]),
                 int(o["pc_trial_iters"]), 0, None if replay is None else _ptr(replay),
                 0 if replay is None else int(replay.shape[0]),
                 None if replay_checks is None else _ptr(replay_checks),
                 0 if replay_checks is None else int(replay_checks.shape[0]))


def solve(lp, trace_cap=100000, x0=None, y0=None, **kw):
    """Restarted PDHG (halpern=1: the restarted Halpern variant with reflection
    ``reflect``).  Returns (x, y, info dict, trace list of dicts)."""
    o = dict(DEFAULTS)
    o.update(kw)
    b = _Bound(lp)
    x0a = None if x0 is None else _f64(x0)
    y0a = None if y0 is None else _f64(y0)
    opts = _opts(o, x0a, y0a)
    x = np.empty(lp.n)
    y = np.empty(lp.m)
    info = _Info()
    tr = np.zeros((trace_cap, len(TRACE_FIELDS)))
    tl = C.c_int64(0)
    _load().orc_solve(C.byref(b.st), C.byref(opts), _ptr(x), _ptr(y), C.byref(info),
                      _ptr(tr), trace_cap, C.byref(tl))
    d = {f: getattr(info, f) for f, _ in _Info._fields_ if f != "pad"}
    trace = [dict(zip(TRACE_FIELDS, r.tolist())) for r in tr[: min(tl.value, trace_cap)]]
    return x, y, d, trace


ATTEMPT_FIELDS = ("k", "eta", "eta_bar", "eta_next", "accept", "omega", "dx2", "dy2", "inter")


def solve_logged(lp, attempt_cap=100000, trace_cap=100000, x0=None, y0=None, replay=None,
                 replay_checks=None, **kw):
    """``solve`` plus one record per step attempt (ATTEMPT_FIELDS: accepted
    iterations before the attempt, the eta tried, Algorithm 5's eta_bar and
    eta', the outcome, omega and the three terms ||dx||^2, ||dy||^2, dy^T K dx on
    the scaled problem).  replay: attempt records of another run (an array of
    rows in ATTEMPT_FIELDS order) whose step sizes and outcomes this run takes
    (eta_bar and eta' are still its own).  replay_checks: per check of another
    run, (restart, candidate is the average); this run takes those decisions and
    logs its own in the trace (own_restart, own_cand_is_avg, with the KKT values
    its restart criteria compared: kkt_anchor, kkt_prev).
    Returns (x, y, info, trace, attempts)."""
    o = dict(DEFAULTS)
    o.update(kw)
    b = _Bound(lp)
    x0a = None if x0 is None else _f64(x0)
    y0a = None if y0 is None else _f64(y0)
    rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.float64)
    rch = (None if replay_checks is None
           else np.ascontiguousarray(replay_checks, dtype=np.float64).reshape(-1, 2))
    opts = _opts(o, x0a, y0a, rep, rch)
    x = np.empty(lp.n)
    y = np.empty(lp.m)
    info = _Info()
    tr = np.zeros((trace_cap, len(TRACE_FIELDS)))
    tl = C.c_int64(0)
    al = np.zeros((attempt_cap, len(ATTEMPT_FIELDS)))
    an = C.c_int64(0)
    _load().orc_solve_logged(C.byref(b.st), C.byref(opts), _ptr(x), _ptr(y), C.byref(info),
                             _ptr(tr), trace_cap, C.byref(tl), _ptr(al), attempt_cap,
                             C.byref(an))
    d = {f: getattr(info, f) for f, _ in _Info._fields_ if f != "pad"}
    trace = [dict(zip(TRACE_FIELDS, r.tolist())) for r in tr[: min(tl.value, trace_cap)]]
    attempts = [dict(zip(ATTEMPT_FIELDS, r.tolist())) for r in al[: min(an.value, attempt_cap)]]
    return x, y, d, trace, attempts


PC_GRID = (0.0, 0.5, 1.0, 2.0)


def pc_tune(lp, **kw):
    """The Pock-Chambolle alpha that pock_chambolle = 2 picks, and the relative
    KKT error of each trial (one per alpha of PC_GRID)."""
    o = dict(DEFAULTS)
    o.update(kw)
    b = _Bound(lp)
    errs = np.empty(len(PC_GRID))
    a = _load().orc_pc_tune(C.byref(b.st), C.byref(_opts(o)), _ptr(errs))
    return float(a), errs


def primal_weight(omega, dx, dy, eps_zero=1e-6):
    """Algorithm 4: the primal weight after a restart whose anchors moved by
    dx (primal) and dy (dual)."""
    return float(_load().orc_primal_weight(omega, dx, dy, eps_zero))


def step_rule(eta, omega, dx2, dy2, inter, accepted):
    """Algorithm 5 on one attempt: (accept, eta_bar, eta')."""
    eb = C.c_double(0.0)
    en = C.c_double(0.0)
    a = _load().orc_step_rule(eta, omega, dx2, dy2, inter, int(accepted), C.byref(eb),
                              C.byref(en))
    return bool(a), eb.value, en.value


def fishnet(lp, P, k_steps, G, Z, **kw):
    """Algorithm 7 (fishnet casting).  G: (n, P) standard-normal casting draws,
    Z: 1-D normal draws of the repopulations.  Returns (x0, y0, gaps, rounds):
    the unscaled warm start and, per round, the |duality gap| of each column
    before the cull (NaN where a round had fewer columns)."""
    o = dict(DEFAULTS)
    o.update(kw)
    b = _Bound(lp)
    G = _f64(G).reshape(lp.n, P)
    Z = _f64(np.asarray(Z, dtype=np.float64).ravel())
    x = np.empty(lp.n)
    y = np.empty(lp.m)
    gaps = np.full((2 * 8 + 2, P), np.nan)
    rounds = C.c_int32(0)
    st = _load().orc_fishnet(C.byref(b.st), C.byref(_opts(o)), P, k_steps, _ptr(G), _ptr(Z),
                             Z.shape[0], _ptr(x), _ptr(y), _ptr(gaps), C.byref(rounds))
    if st != 0:
        raise ValueError("orc_fishnet: invalid P or too few repopulation draws")
    return x, y, gaps[: rounds.value], rounds.value


def fishnet_draws(P):
    """Normal draws one fishnet run with P columns consumes in its repopulations."""
    total, cols, i = 0, P, 0
    while cols > 1:
        keep = cols // 2
        if i % 2 == 1 and cols > 2:
            total += keep * keep
            cols = 2 * keep
        else:
            cols = keep
        i += 1
    return total


def infeasibility(lp, dx, dy, dlam, tol):
    """Algorithm 6 on given differences: (status 0 / 2 / 3, terms dict)."""
    b = _Bound(lp)
    dx, dy, dl = _f64(dx), _f64(dy), _f64(dlam)
    terms = np.empty(8)
    st = _load().orc_infeasibility(C.byref(b.st), _ptr(dx), _ptr(dy), _ptr(dl), tol, _ptr(terms))
    names = ("adx", "gdx_min", "cdx", "v_dist", "ktdy_res", "dy_ineq_min", "psi")
    return st, dict(zip(names, terms[:7].tolist()))


def start_point(lp):
    """Unscaled default start: x = proj_X(0), y = 0."""
    return np.clip(np.zeros(lp.n), lp.l, lp.u), np.zeros(lp.m)


def unrolled_forward(lp, tau, sigma, K_iters, x0=None, y0=None):
    """Iterates 0..K_iters of fixed-step PDHG on the unscaled problem."""
    b = _Bound(lp)
    if x0 is None:
        x0, y0 = start_point(lp)
    x0, y0 = _f64(x0), _f64(y0)
    xs = np.empty((K_iters + 1, lp.n))
    ys = np.empty((K_iters + 1, lp.m))
    _load().orc_unrolled_forward(C.byref(b.st), tau, sigma, K_iters, _ptr(x0), _ptr(y0),
                                 _ptr(xs), _ptr(ys))
    return xs, ys


def unrolled_adjoint(lp, tau, sigma, K_iters, gxK, x0=None, y0=None):
    """Gradient of L(x_K) w.r.t. (c, q, nonzeros of K) given dL/dx_K."""
    b = _Bound(lp)
    if x0 is None:
        x0, y0 = start_point(lp)
    x0, y0, g = _f64(x0), _f64(y0), _f64(gxK)
    dc = np.empty(lp.n)
    dq = np.empty(lp.m)
    dv = np.empty(lp.nnz)
    _load().orc_unrolled_adjoint(C.byref(b.st), tau, sigma, K_iters, _ptr(x0), _ptr(y0),
                                 _ptr(g), _ptr(dc), _ptr(dq), _ptr(dv))
    return dc, dq, dv
