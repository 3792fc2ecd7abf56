"""torch.autograd.Function over unrolled fixed-step PDHG (argument marshalling only).

``UnrolledPDHG.apply(c, q, vals, problem, K, ckpt, precision, eta, omega)``
returns x_K, the primal iterate after K fixed-step PDHG iterations (Algorithm 1,
theta = 1, start x = proj_X(0), y = 0) of the LP held by ``problem`` with its cost
c, right-hand side q and nonzero values vals replaced by the given tensors.
Backward puts the forward's values back on the handle (another forward on the
same problem may have replaced them) and calls the CUDA library's hand-written
adjoint (lp_grad) for dL/dc, dL/dq and dL/dvals; step sizes are constants (eta,
omega given, or derived from the LP of that forward when None).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import lp as L


def _opts(precision, eta, omega):
    o = L.lp_opts_default(precision=precision)
    if eta:
        o.eta0 = float(eta)
    if omega:
        o.omega0 = float(omega)
    return o


def _f64(t):
    return t.detach().to(device="cuda", dtype=torch.float64).contiguous()


class UnrolledPDHG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, q, vals, problem, K, ckpt, precision=L.LP_PREC_FP64, eta=None,
                omega=None):
        c64, q64, v64 = _f64(c), _f64(q), _f64(vals)
        torch.cuda.current_stream().synchronize()
        s = L.lp_update_values(problem.handle, v64.data_ptr(), c64.data_ptr(), q64.data_ptr(),
                               None, None, L.LP_MEM_DEVICE)
        if s != 0:
            raise L.LpError(s, "lp_update_values")
        xK = torch.empty(problem.n, dtype=torch.float64, device="cuda")
        o = _opts(precision, eta, omega)
        s = L.lp_unroll(problem.handle, o, int(K), xK.data_ptr(), None, L.LP_MEM_DEVICE)
        if s != 0:
            raise L.LpError(s, "lp_unroll")
        ctx.problem, ctx.K, ctx.ckpt, ctx.opts = problem, int(K), int(ckpt), o
        ctx.dtypes = (c.dtype, q.dtype, vals.dtype)
        # the values this forward ran on: lp_grad recomputes the unrolled forward
        # from the handle's current values, which a later forward may have replaced
        ctx.values = (c64, q64, v64)
        return xK

    @staticmethod
    def backward(ctx, gx):
        p = ctx.problem
        g = _f64(gx)
        dc = torch.empty(p.n, dtype=torch.float64, device="cuda")
        dq = torch.empty(p.m, dtype=torch.float64, device="cuda")
        dv = torch.empty(max(p.nnz, 1), dtype=torch.float64, device="cuda")
        c64, q64, v64 = ctx.values
        torch.cuda.current_stream().synchronize()
        s = L.lp_update_values(p.handle, v64.data_ptr(), c64.data_ptr(), q64.data_ptr(), None,
                               None, L.LP_MEM_DEVICE)
        if s != 0:
            raise L.LpError(s, "lp_update_values")
        s = L.lp_grad(p.handle, ctx.opts, ctx.K, ctx.ckpt, g.data_ptr(), dc.data_ptr(),
                      dq.data_ptr(), dv.data_ptr(), None, L.LP_MEM_DEVICE)
        if s != 0:
            raise L.LpError(s, "lp_grad")
        tc, tq, tv = ctx.dtypes
        return (dc.to(tc), dq.to(tq), dv[: p.nnz].to(tv), None, None, None, None, None, None)


def unroll(problem, K, precision=L.LP_PREC_FP64, eta=None, omega=None):
    """x_K and y_K (numpy) of the LP as it is held by ``problem``."""
    import numpy as np
    x = np.empty(problem.n)
    y = np.empty(problem.m)
    ts = (C.c_double * 2)()
    s = L.lp_unroll(problem.handle, _opts(precision, eta, omega), int(K), x.ctypes.data,
                    y.ctypes.data, L.LP_MEM_HOST, C.cast(ts, C.c_void_p))
    if s != 0:
        raise L.LpError(s, "lp_unroll")
    return x, y, (ts[0], ts[1])


def grad(problem, K, ckpt, gxK, precision=L.LP_PREC_FP64, eta=None, omega=None):
    """(dc, dq, dvals, x_K, (tau, sigma)) as numpy arrays for dL/dx_K = gxK."""
    import numpy as np
    g = np.ascontiguousarray(gxK, dtype=np.float64)
    dc = np.empty(problem.n)
    dq = np.empty(problem.m)
    dv = np.empty(max(problem.nnz, 1))
    xK = np.empty(problem.n)
    ts = (C.c_double * 2)()
    s = L.lp_grad(problem.handle, _opts(precision, eta, omega), int(K), int(ckpt), g.ctypes.data,
                  dc.ctypes.data, dq.ctypes.data, dv.ctypes.data, xK.ctypes.data, L.LP_MEM_HOST,
                  C.cast(ts, C.c_void_p))
    if s != 0:
        raise L.LpError(s, "lp_grad")
    return dc, dq, dv[: problem.nnz], xK, (ts[0], ts[1])
