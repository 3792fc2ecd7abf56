"""Python binding of the C ABI in ``include/lp.h`` (argument marshalling only).

The functions ``lp_create``, ``lp_solve``, ``lp_solve_batch``, ``lp_grad``,
``lp_profile_step``, ``lp_destroy`` and ``lp_status_string`` have the C
names and call the CUDA library ``csrc/libpdhg.so`` through ctypes; every step of
the solver runs in that library's kernels.  PyTorch is used only to hold device
memory and to supply the current CUDA stream.  There is no fallback: if the
library is missing or fails to load, ``load()`` raises.

``Problem`` is a thin convenience wrapper that moves a ``synth.LP`` (numpy
arrays) to the GPU with torch and keeps the handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LP_MEM_HOST, LP_MEM_DEVICE = 0, 1
LP_PREC_FP64, LP_PREC_MIXED = 0, 1

STATUS = {0: "LP_OK", 1: "LP_OPTIMAL", 2: "LP_PRIMAL_INFEASIBLE", 3: "LP_DUAL_INFEASIBLE",
          4: "LP_ITERATION_LIMIT", 5: "LP_TIME_LIMIT", 6: "LP_NUMERICAL_ERROR",
          -1: "LP_INVALID_ARGUMENT", -2: "LP_CUDA_ERROR", -3: "LP_OUT_OF_MEMORY",
          -4: "LP_DEVICE_TIMEOUT", -5: "LP_NOT_SUPPORTED"}
LP_OPTIMAL, LP_ITERATION_LIMIT, LP_TIME_LIMIT, LP_NUMERICAL_ERROR = 1, 4, 5, 6
LP_INVALID_ARGUMENT, LP_NOT_SUPPORTED = -1, -5


class LpDesc(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("vals", C.c_void_p),
                ("sense", C.c_void_p), ("c", C.c_void_p), ("q", C.c_void_p),
                ("l", C.c_void_p), ("u", C.c_void_p),
                ("memory_space", C.c_int32), ("reserved", C.c_int32)]


class LpOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int64), ("time_limit_s", C.c_double),
                ("precision", C.c_int32), ("check_every", C.c_int32),
                ("ruiz_iters", C.c_int32), ("pock_chambolle", C.c_int32),
                ("adaptive_step", C.c_int32), ("primal_weight_update", C.c_int32),
                ("restarts", C.c_int32), ("power_iters", C.c_int32),
                ("ruiz_tol", C.c_double), ("eta_scale", C.c_double),
                ("beta_sufficient", C.c_double), ("beta_necessary", C.c_double),
                ("beta_artificial", C.c_double), ("eps_zero", C.c_double),
                ("polish_switch_tol", C.c_double),
                ("x0", C.c_void_p), ("y0", C.c_void_p),
                ("omega0", C.c_double), ("eta0", C.c_double),
                ("warm_memory_space", C.c_int32), ("loop_mode", C.c_int32),
                ("infeas_detect", C.c_int32), ("reserved_opts", C.c_int32),
                ("infeas_tol", C.c_double), ("autotune", C.c_int32),
                ("halpern", C.c_int32), ("halpern_reflect", C.c_double),
                ("pc_alpha", C.c_double), ("pc_trial_iters", C.c_int32),
                ("reserved_opts2", C.c_int32), ("attempt_log", C.c_void_p),
                ("attempt_cap", C.c_int64)]


ATTEMPT_FIELDS = ("k", "eta", "eta_bar", "eta_next", "accept", "omega", "dx2", "dy2", "inter")

TRACE_FIELDS = ("k", "attempts", "restart", "cand_is_avg", "omega", "eta",
                "kkt_cur", "kkt_avg", "rel_gap", "rel_pres", "rel_dres", "kkt_cand")


class LpTraceRec(C.Structure):
    _fields_ = [(f, C.c_double) for f in TRACE_FIELDS]


class LpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("precision_used", C.c_int32),
                ("iters", C.c_int64), ("attempts", C.c_int64), ("restarts", C.c_int64),
                ("fp64_iters", C.c_int64),
                ("pobj", C.c_double), ("dobj", C.c_double), ("rel_gap", C.c_double),
                ("rel_pres", C.c_double), ("rel_dres", C.c_double),
                ("omega", C.c_double), ("eta", C.c_double), ("norm_K", C.c_double),
                ("setup_s", C.c_double), ("solve_s", C.c_double),
                ("kernel_launches", C.c_int64),
                ("x", C.c_void_p), ("y", C.c_void_p),
                ("memory_space", C.c_int32), ("split_rows", C.c_int32),
                ("trace", C.c_void_p), ("trace_cap", C.c_int64), ("trace_len", C.c_int64),
                ("pc_alpha_used", C.c_double), ("attempt_len", C.c_int64)]


EXPORTS = ("lp_opts_default", "lp_create", "lp_solve", "lp_solve_batch", "lp_grad",
           "lp_unroll", "lp_update_values", "lp_profile_step", "lp_profile_gather", "lp_destroy",
           "lp_status_string",
           "lp_abi_version", "lp_kkt_noalloc", "lp_batch_create", "lp_batch_solve",
           "lp_batch_destroy", "lp_fishnet", "lp_fishnet_draws")

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpdhg.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA solver library missing: {path}")
    lib = C.CDLL(path)
    P = C.POINTER
    lib.lp_opts_default.argtypes = [P(LpOpts)]
    lib.lp_opts_default.restype = None
    lib.lp_create.argtypes = [P(LpDesc), C.c_void_p, P(C.c_void_p)]
    lib.lp_create.restype = C.c_int
    lib.lp_solve.argtypes = [C.c_void_p, P(LpOpts), P(LpResult)]
    lib.lp_solve.restype = C.c_int
    lib.lp_solve_batch.argtypes = [P(C.c_void_p), C.c_int32, P(LpOpts), P(LpResult)]
    lib.lp_solve_batch.restype = C.c_int
    lib.lp_grad.argtypes = [C.c_void_p, P(LpOpts), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    lib.lp_grad.restype = C.c_int
    lib.lp_profile_step.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]
    lib.lp_profile_step.restype = C.c_int
    lib.lp_profile_gather.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
    lib.lp_profile_gather.restype = C.c_int
    lib.lp_destroy.argtypes = [C.c_void_p]
    lib.lp_destroy.restype = None
    lib.lp_status_string.argtypes = [C.c_int]
    lib.lp_status_string.restype = C.c_char_p
    lib.lp_abi_version.argtypes = []
    lib.lp_abi_version.restype = C.c_int32
    lib.lp_unroll.argtypes = [C.c_void_p, P(LpOpts), C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                              C.c_void_p]
    lib.lp_unroll.restype = C.c_int
    lib.lp_update_values.argtypes = [C.c_void_p] + [C.c_void_p] * 5 + [C.c_int32]
    lib.lp_update_values.restype = C.c_int
    lib.lp_batch_create.argtypes = [P(C.c_void_p), C.c_int32, C.c_void_p, P(C.c_void_p)]
    lib.lp_batch_create.restype = C.c_int
    lib.lp_batch_solve.argtypes = [C.c_void_p, P(LpOpts), C.c_void_p]
    lib.lp_batch_solve.restype = C.c_int
    lib.lp_batch_destroy.argtypes = [C.c_void_p]
    lib.lp_batch_destroy.restype = None
    lib.lp_kkt_noalloc.argtypes = [P(LpDesc), C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                   C.c_void_p]
    lib.lp_kkt_noalloc.restype = C.c_int
    lib.lp_fishnet.argtypes = [C.c_void_p, P(LpOpts), C.c_int32, C.c_int32, C.c_void_p,
                               C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                               P(C.c_int32), C.c_int32]
    lib.lp_fishnet.restype = C.c_int
    lib.lp_fishnet_draws.argtypes = [C.c_int32]
    lib.lp_fishnet_draws.restype = C.c_int64
    _lib = lib
    return lib


# ------------------------------------------------------------ C-named calls

def lp_opts_default(**overrides) -> LpOpts:
    o = LpOpts()
    load().lp_opts_default(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def lp_create(desc: LpDesc, stream: int | None = None) -> C.c_void_p:
    h = C.c_void_p()
    s = load().lp_create(C.byref(desc), C.c_void_p(stream or 0), C.byref(h))
    if s != 0:
        raise LpError(s, "lp_create")
    return h


def lp_solve(h, opts: LpOpts, res: LpResult) -> int:
    return load().lp_solve(h, C.byref(opts), C.byref(res))


def lp_solve_batch(handles, opts: LpOpts, results) -> int:
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h
                                        for h in handles])
    return load().lp_solve_batch(arr, len(handles), C.byref(opts), results)


def lp_grad(h, opts: LpOpts, K_iters: int, ckpt_every: int, dL_dxK: int, dc: int, dq: int,
            dvals: int, x_K: int | None, memory_space: int, tau_sigma_out=None) -> int:
    return load().lp_grad(h, C.byref(opts), K_iters, ckpt_every, dL_dxK, dc, dq, dvals,
                          x_K or None, memory_space, tau_sigma_out)


def lp_unroll(h, opts: LpOpts, K_iters: int, x_K: int | None, y_K: int | None,
              memory_space: int, tau_sigma_out=None) -> int:
    return load().lp_unroll(h, C.byref(opts), K_iters, x_K or None, y_K or None, memory_space,
                            tau_sigma_out)


def lp_fishnet(h, opts: LpOpts, P: int, k_steps: int, G: int, Z: int | None, nZ: int, x0: int,
               y0: int, gaps=None, rounds=None, memory_space: int = LP_MEM_HOST) -> int:
    return load().lp_fishnet(h, C.byref(opts), P, k_steps, G, Z or None, nZ, x0, y0, gaps,
                             rounds, memory_space)


def lp_fishnet_draws(P: int) -> int:
    return int(load().lp_fishnet_draws(P))


def lp_update_values(h, vals=None, c=None, q=None, l=None, u=None,
                     memory_space: int = LP_MEM_DEVICE) -> int:
    return load().lp_update_values(h, vals, c, q, l, u, memory_space)


def lp_profile_gather(h, precision: int, reps: int, blocks_per_sm: int = 4):
    """Milliseconds per launch of the minimal gather loop over K and over K^T."""
    ms = (C.c_double * 2)()
    s = load().lp_profile_gather(h, precision, reps, blocks_per_sm, C.cast(ms, C.c_void_p))
    if s != 0:
        raise LpError(s, "lp_profile_gather")
    return list(ms)


def lp_profile_step(h, precision: int, reps: int):
    ms = (C.c_double * 4)()
    by = (C.c_double * 4)()
    s = load().lp_profile_step(h, precision, reps, C.cast(ms, C.c_void_p), C.cast(by, C.c_void_p))
    if s != 0:
        raise LpError(s, "lp_profile_step")
    return list(ms), list(by)


def lp_kkt_noalloc(desc: LpDesc, x: int, y: int, omega: float, stream: int | None = None):
    """Termination quantities of (x, y) (device pointers) without device
    allocation; returns the 8 values of include/lp.h's lp_kkt_noalloc."""
    out = (C.c_double * 8)()
    s = load().lp_kkt_noalloc(C.byref(desc), x, y, omega, C.cast(out, C.c_void_p),
                              C.c_void_p(stream or 0))
    if s != 0:
        raise LpError(s, "lp_kkt_noalloc")
    return list(out)


def lp_batch_create(handles, stream: int | None = None) -> C.c_void_p:
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h
                                        for h in handles])
    b = C.c_void_p()
    s = load().lp_batch_create(arr, len(handles), C.c_void_p(stream or 0), C.byref(b))
    if s != 0:
        raise LpError(s, "lp_batch_create")
    return b


def lp_batch_solve(b, opts: LpOpts, results) -> int:
    return load().lp_batch_solve(b, C.byref(opts), C.cast(results, C.c_void_p))


def lp_batch_destroy(b) -> None:
    load().lp_batch_destroy(b)


def lp_destroy(h) -> None:
    load().lp_destroy(h)


def lp_status_string(s: int) -> str:
    return load().lp_status_string(s).decode()


class LpError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status


# ------------------------------------------------------------ convenience

def _torch():
    import torch
    return torch


class Problem:
    """An LP resident on the current CUDA device.

    ``lp`` is a ``synth.LP`` (numpy arrays).  With ``device_copy=True`` the
    arrays are first placed in torch CUDA tensors and passed as device pointers;
    otherwise the host arrays are passed and the library copies them.
    """

    def __init__(self, lp, device_copy: bool = True, stream=None):
        torch = _torch()
        self.lp = lp
        self.m, self.n, self.nnz = lp.m, lp.n, lp.nnz
        arrays = dict(row_ptr=np.ascontiguousarray(lp.row_ptr, np.int64),
                      col_idx=np.ascontiguousarray(lp.col_idx, np.int32),
                      vals=np.ascontiguousarray(lp.vals, np.float64),
                      sense=np.ascontiguousarray(lp.sense, np.uint8),
                      c=np.ascontiguousarray(lp.c, np.float64),
                      q=np.ascontiguousarray(lp.q, np.float64),
                      l=np.ascontiguousarray(lp.l, np.float64),
                      u=np.ascontiguousarray(lp.u, np.float64))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        if device_copy:
            self._keep = {k: torch.from_numpy(v).cuda() for k, v in arrays.items()}
            ptr = {k: v.data_ptr() for k, v in self._keep.items()}
            space = LP_MEM_DEVICE
            torch.cuda.synchronize()
        else:
            self._keep = arrays
            ptr = {k: v.ctypes.data for k, v in arrays.items()}
            space = LP_MEM_HOST
        self.desc = LpDesc(lp.m, lp.n, lp.nnz, ptr["row_ptr"], ptr["col_idx"], ptr["vals"],
                           ptr["sense"], ptr["c"], ptr["q"], ptr["l"], ptr["u"], space, 0)
        self.handle = lp_create(self.desc, stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None) is not None:
            lp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, trace_cap: int = 0, out_device: bool = False, x0=None, y0=None,
              attempt_cap: int = 0, **opts):
        """Returns (x, y, info, trace).  x, y are numpy (or torch CUDA tensors
        with out_device=True); info is a dict of the lp_result scalars.  With
        attempt_cap > 0, info["attempt_log"] lists up to that many step attempts
        (dicts of ATTEMPT_FIELDS)."""
        torch = _torch()
        o = lp_opts_default(**opts)
        keep = []
        alog = None
        if attempt_cap > 0:
            alog = np.zeros((attempt_cap, len(ATTEMPT_FIELDS)))
            o.attempt_log = alog.ctypes.data
            o.attempt_cap = attempt_cap
        if x0 is not None or y0 is not None:
            wx = np.ascontiguousarray(x0, np.float64) if x0 is not None else None
            wy = np.ascontiguousarray(y0, np.float64) if y0 is not None else None
            keep += [wx, wy]
            o.x0 = wx.ctypes.data if wx is not None else None
            o.y0 = wy.ctypes.data if wy is not None else None
            o.warm_memory_space = LP_MEM_HOST
        res = LpResult()
        if out_device:
            x = torch.empty(self.n, dtype=torch.float64, device="cuda")
            y = torch.empty(self.m, dtype=torch.float64, device="cuda")
            res.x, res.y = x.data_ptr(), y.data_ptr()
            res.memory_space = LP_MEM_DEVICE
        else:
            x = np.empty(self.n)
            y = np.empty(self.m)
            res.x, res.y = x.ctypes.data, y.ctypes.data
            res.memory_space = LP_MEM_HOST
        tr = None
        if trace_cap > 0:
            tr = (LpTraceRec * trace_cap)()
            res.trace = C.cast(tr, C.c_void_p)
            res.trace_cap = trace_cap
        s = lp_solve(self.handle, o, res)
        if s < 0:
            raise LpError(s, "lp_solve")
        info = {f: getattr(res, f) for f, _ in LpResult._fields_
                if f not in ("x", "y", "trace", "reserved", "memory_space", "trace_cap")}
        if alog is not None:
            info["attempt_log"] = [dict(zip(ATTEMPT_FIELDS, r.tolist()))
                                   for r in alog[: res.attempt_len]]
        trace = []
        if tr is not None:
            for r in tr[: min(res.trace_len, trace_cap)]:
                trace.append({f: getattr(r, f) for f in TRACE_FIELDS})
        return x, y, info, trace

    def fishnet(self, P: int, k_steps: int, G, Z, **opts):
        """Algorithm 7 on this LP: G (n, P) and Z (1-D) are numpy normal draws.
        Returns (x0, y0, gaps (rounds, P) with NaN for absent points, rounds)."""
        o = lp_opts_default(**opts)
        Gh = np.ascontiguousarray(np.asarray(G, np.float64).reshape(self.n, P))
        Zh = np.ascontiguousarray(np.asarray(Z, np.float64).ravel())
        x0 = np.empty(self.n)
        y0 = np.empty(self.m)
        gaps = np.full((2 * 8 + 2, P), np.nan)
        rounds = C.c_int32(0)
        s = lp_fishnet(self.handle, o, P, k_steps, Gh.ctypes.data,
                       Zh.ctypes.data if Zh.size else None, Zh.size, x0.ctypes.data,
                       y0.ctypes.data, gaps.ctypes.data, C.byref(rounds), LP_MEM_HOST)
        if s < 0:
            raise LpError(s, "lp_fishnet")
        return x0, y0, gaps[: rounds.value], rounds.value

    def profile_step(self, precision: int = LP_PREC_FP64, reps: int = 20):
        return lp_profile_step(self.handle, precision, reps)

    def profile_gather(self, precision: int = LP_PREC_MIXED, reps: int = 20,
                       blocks_per_sm: int = 4):
        return lp_profile_gather(self.handle, precision, reps, blocks_per_sm)


class Batch:
    """A batch of LPs (``synth.LP`` list) solved together by lp_batch_solve."""

    def __init__(self, lps, device_copy: bool = True):
        torch = _torch()
        self.problems = [Problem(lp, device_copy=device_copy) for lp in lps]
        self.stream = torch.cuda.Stream()
        self.handle = lp_batch_create([p.handle for p in self.problems], self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None) is not None:
            lp_batch_destroy(self.handle)
            self.handle = None
        for p in getattr(self, "problems", []):
            p.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, **opts):
        """Returns a list of (x, y, info) per LP."""
        o = lp_opts_default(**opts)
        B = len(self.problems)
        res = (LpResult * B)()
        xs, ys = [], []
        for k, p in enumerate(self.problems):
            x = np.empty(p.n)
            y = np.empty(p.m)
            xs.append(x)
            ys.append(y)
            res[k].x, res[k].y = x.ctypes.data, y.ctypes.data
            res[k].memory_space = LP_MEM_HOST
        s = lp_batch_solve(self.handle, o, res)
        if s < 0:
            raise LpError(s, "lp_batch_solve")
        out = []
        for k in range(B):
            info = {f: getattr(res[k], f) for f, _ in LpResult._fields_
                    if f not in ("x", "y", "trace", "reserved", "memory_space", "trace_cap")}
            out.append((xs[k], ys[k], info))
        return out
