"""GPU adjoint of unrolled fixed-step PDHG (lp_grad) against the FP64 oracle's
unrolled adjoint and central finite differences, through the C ABI."""
import dataclasses

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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _steps(oracle_mod, lp):
    eta = 0.9 / oracle_mod.power_norm(lp, 200)
    return eta, 1.0


def masks(oracle_mod, lp, tau, sigma, K):
    """Projection masks of every unrolled step (FP64 oracle forward)."""
    xs, ys = oracle_mod.unrolled_forward(lp, tau, sigma, K)
    mx, my = [], []
    for t in range(K):
        vx = xs[t] - tau * (lp.c - oracle_mod.spmv_t(lp, ys[t]))
        mx.append((lp.l < vx) & (vx < lp.u))
        vy = ys[t] + sigma * (lp.q - oracle_mod.spmv(lp, 2 * xs[t + 1] - xs[t]))
        my.append((lp.sense == 0) | (vy > 0))
    return np.array(mx), np.array(my)


def perturbed(lp, kind, idx, delta):
    cp = synth.LP(**{f.name: getattr(lp, f.name) for f in dataclasses.fields(lp)})
    arr = getattr(lp, kind).copy()
    arr[idx] += delta
    setattr(cp, kind, arr)
    return cp


def kink_free(oracle_mod, lp, tau, sigma, K, kind, idx, h):
    """True when no projection mask of the trajectory changes under +-h, so the
    loss is differentiable there and central differences apply."""
    m0 = masks(oracle_mod, lp, tau, sigma, K)
    for sgn in (1, -1):
        m1 = masks(oracle_mod, perturbed(lp, kind, idx, sgn * h), tau, sigma, K)
        if not (np.array_equal(m0[0], m1[0]) and np.array_equal(m0[1], m1[1])):
            return False
    return True


def test_unroll_and_grad_match_oracle_fp64(L, oracle_mod):
    """m = 50, n = 100, K = 500 steps, checkpoint every 50: x_K and the gradient
    of ||x_K - x_target||^2 w.r.t. (c, q, nonzeros) agree with the oracle."""
    from paper_2508_16806_gb300 import autograd as AG
    lp, xt = synth.adjoint_lp(50, 100, 8, seed=20250820)
    eta, omega = _steps(oracle_mod, lp)
    prob = L.Problem(lp)
    xK, yK, (tau, sigma) = AG.unroll(prob, 500, eta=eta, omega=omega)
    assert tau == pytest.approx(eta / omega, rel=1e-15) and sigma == pytest.approx(eta * omega, rel=1e-15)
    xs, ys = oracle_mod.unrolled_forward(lp, tau, sigma, 500)
    assert rel(xK, xs[-1]) < 1e-12 and rel(yK, ys[-1]) < 1e-12
    g = 2.0 * (xK - xt)
    dc, dq, dv, xK2, _ = AG.grad(prob, 500, 50, g, eta=eta, omega=omega)
    assert np.array_equal(xK, xK2)
    oc, oq, ov = oracle_mod.unrolled_adjoint(lp, tau, sigma, 500, g)
    assert rel(dc, oc) < 1e-10, rel(dc, oc)
    assert rel(dq, oq) < 1e-10, rel(dq, oq)
    assert rel(dv, ov) < 1e-10, rel(dv, ov)


@pytest.mark.parametrize("K,ckpt", [(1, 1), (7, 3), (64, 64), (100, 50)])
def test_grad_checkpoint_schedules_agree(L, oracle_mod, K, ckpt):
    from paper_2508_16806_gb300 import autograd as AG
    lp, xt = synth.adjoint_lp(50, 100, 8, seed=3)
    eta, omega = _steps(oracle_mod, lp)
    prob = L.Problem(lp)
    xK, _, (tau, sigma) = AG.unroll(prob, K, eta=eta, omega=omega)
    g = 2.0 * (xK - xt)
    dc, dq, dv, _, _ = AG.grad(prob, K, ckpt, g, eta=eta, omega=omega)
    oc, oq, ov = oracle_mod.unrolled_adjoint(lp, tau, sigma, K, g)
    assert rel(dc, oc) < 1e-10 and rel(dq, oq) < 1e-10 and rel(dv, ov) < 1e-10


def test_grad_central_differences(L, oracle_mod):
    """Central finite differences (h = 1e-6, FP64) of the GPU's own unrolled
    forward agree with the GPU adjoint to 1e-5 relative."""
    from paper_2508_16806_gb300 import autograd as AG
    lp, xt = synth.adjoint_lp(50, 100, 8, seed=20250820)
    eta, omega = _steps(oracle_mod, lp)
    K = 200
    prob = L.Problem(lp)
    xK, _, _ = AG.unroll(prob, K, eta=eta, omega=omega)
    dc, dq, dv, _, _ = AG.grad(prob, K, 50, 2.0 * (xK - xt), eta=eta, omega=omega)
    h = 1e-6
    rng = np.random.default_rng(1)
    checked = 0
    for kind, grad, count in (("c", dc, lp.n), ("q", dq, lp.m), ("vals", dv, lp.nnz)):
        for idx in rng.choice(count, 10, replace=False):
            if not kink_free(oracle_mod, lp, eta / omega, eta * omega, K, kind, idx, h):
                continue
            checked += 1
            loss = []
            for sgn in (1, -1):
                arr = getattr(lp, kind).copy()
                arr[idx] += sgn * h
                kw = {kind: arr.ctypes.data}
                assert L.lp_update_values(prob.handle, memory_space=L.LP_MEM_HOST, **kw) == 0
                x2, _, _ = AG.unroll(prob, K, eta=eta, omega=omega)
                loss.append(float(np.sum((x2 - xt) ** 2)))
            base = getattr(lp, kind).copy()
            assert L.lp_update_values(prob.handle, memory_space=L.LP_MEM_HOST,
                                      **{kind: base.ctypes.data}) == 0
            fd = (loss[0] - loss[1]) / (2 * h)
            scale = max(abs(fd), abs(grad[idx]), 1e-3)
            # rounding of the two FP64 losses bounds the central difference's own
            # error by about 2 eps |L| / h (truncation, O(h^2), is far smaller)
            fd_noise = 4 * np.finfo(float).eps * max(abs(loss[0]), abs(loss[1])) / h
            assert abs(fd - grad[idx]) <= 1e-5 * scale + fd_noise, (kind, idx, fd, grad[idx])
    assert checked >= 20


def test_autograd_function(L, oracle_mod):
    import torch
    from paper_2508_16806_gb300.autograd import UnrolledPDHG
    from paper_2508_16806_gb300 import autograd as AG
    lp, xt = synth.adjoint_lp(50, 100, 8, seed=11)
    eta, omega = _steps(oracle_mod, lp)
    prob = L.Problem(lp)
    c = torch.tensor(lp.c, device="cuda", requires_grad=True)
    q = torch.tensor(lp.q, device="cuda", requires_grad=True)
    v = torch.tensor(lp.vals, device="cuda", requires_grad=True)
    xK = UnrolledPDHG.apply(c, q, v, prob, 120, 40, L.LP_PREC_FP64, eta, omega)
    loss = ((xK - torch.tensor(xt, device="cuda")) ** 2).sum()
    loss.backward()
    _, _, (tau, sigma) = AG.unroll(prob, 1, eta=eta, omega=omega)
    oc, oq, ov = oracle_mod.unrolled_adjoint(lp, tau, sigma, 120, 2.0 * (xK.detach().cpu().numpy() - xt))
    assert rel(c.grad.cpu().numpy(), oc) < 1e-10
    assert rel(q.grad.cpu().numpy(), oq) < 1e-10
    assert rel(v.grad.cpu().numpy(), ov) < 1e-10


def test_autograd_two_forwards_then_backward_of_first(L, oracle_mod):
    """Two forwards on one Problem with different values, then backward of the
    first: the gradient is that of the first LP (its values are put back on the
    handle), with step sizes derived from the first LP (eta, omega = None)."""
    import dataclasses
    import torch
    from paper_2508_16806_gb300.autograd import UnrolledPDHG
    lp, xt = synth.adjoint_lp(50, 100, 8, seed=12)
    rng = np.random.default_rng(99)
    lpb = synth.LP(**{f.name: getattr(lp, f.name) for f in dataclasses.fields(lp)})
    lpb.c = lp.c + rng.normal(0, 0.5, lp.n)
    lpb.vals = lp.vals * rng.uniform(0.5, 1.5, lp.nnz)
    prob = L.Problem(lp)
    dev = dict(device="cuda", dtype=torch.float64)
    ca = torch.tensor(lp.c, requires_grad=True, **dev)
    qa = torch.tensor(lp.q, requires_grad=True, **dev)
    va = torch.tensor(lp.vals, requires_grad=True, **dev)
    xa = UnrolledPDHG.apply(ca, qa, va, prob, 80, 20, L.LP_PREC_FP64, None, None)
    cb = torch.tensor(lpb.c, requires_grad=True, **dev)
    qb = torch.tensor(lpb.q, requires_grad=True, **dev)
    vb = torch.tensor(lpb.vals, requires_grad=True, **dev)
    xb = UnrolledPDHG.apply(cb, qb, vb, prob, 80, 20, L.LP_PREC_FP64, None, None)
    loss_a = ((xa - torch.tensor(xt, **dev)) ** 2).sum()
    loss_a.backward()
    # the first LP's own step sizes: eta_scale / ||K||_2 (Algorithm 2 on the
    # unscaled K, as lp_grad takes them) and ||c|| / ||q||
    eta = 0.9 / oracle_mod.power_norm(lp, 100)
    omega = np.linalg.norm(lp.c) / np.linalg.norm(lp.q)
    tau, sigma = eta / omega, eta * omega
    xs, _ = oracle_mod.unrolled_forward(lp, tau, sigma, 80)
    assert rel(xa.detach().cpu().numpy(), xs[-1]) < 1e-8
    oc, oq, ov = oracle_mod.unrolled_adjoint(lp, tau, sigma, 80, 2.0 * (xs[-1] - xt))
    assert rel(ca.grad.cpu().numpy(), oc) < 1e-8
    assert rel(qa.grad.cpu().numpy(), oq) < 1e-8
    assert rel(va.grad.cpu().numpy(), ov) < 1e-8
    assert xb.shape == xa.shape and cb.grad is None
    prob.close()


def test_fp32_gradient_close_to_fp64(L, oracle_mod):
    """The FP32 adjoint (FP64 accumulation of dc, dq, dvals) stays close to the
    FP64 one on an m = 5000 instance; the error is reported in the assertion."""
    from paper_2508_16806_gb300 import autograd as AG
    lp, xt = synth.adjoint_lp(5000, 10000, 20, seed=7)
    prob = L.Problem(lp)
    x64, _, (tau, sigma) = AG.unroll(prob, 100)
    g = 2.0 * (x64 - xt)
    d64 = AG.grad(prob, 100, 50, g)
    d32 = AG.grad(prob, 100, 50, g, precision=L.LP_PREC_MIXED)
    for a, b in zip(d32[:3], d64[:3]):
        assert np.all(np.isfinite(a))
        assert rel(a, b) < 1e-3, rel(a, b)
