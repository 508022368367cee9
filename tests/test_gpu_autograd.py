"""Gradients of L = sum_s ||x_s^T - target_s||^2 over T implicit hyperdiffusion
steps, from the adjoint (transposed-band) solves behind torch.autograd, against
the CPU oracle's adjoint and against central finite differences.

Tolerances: 1e-11 normwise against the oracle's gradients (both are FP64 but
reach them by different factorisations: the oracle factors A^T anew, the
library reuses A's factors, and the sums run in different orders); 1e-6 against
central differences with h = 1e-6.  The loss is quadratic in C0, so there the
central difference is exact up to round-off; in sigma its truncation error is
~(h/sigma)^2 (1e-6 relative for sigma ~ 5e-3), so the sigma check uses the
Richardson combination (4 D(h/2) - D(h)) / 3, whose truncation is O(h^4)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1807_07382_gb300 import build  # noqa: E402
from paper_1807_07382_gb300.autograd import hyperdiff_steps  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def make_case(batch, n, T):
    w = synth.adjoint_batch(batch=batch, n=n, steps=T)
    c0 = w.field0.reshape(batch, n)
    target = oracle.hyperdiff_steps(w.n, w.sigma * (1 + w.extra["perturb"]), w.field0, T).reshape(batch, n)
    return w, c0, target


def gpu_loss_grad(c0, sigma, target, T, k):
    c = torch.from_numpy(c0).cuda().requires_grad_(True)
    s = torch.from_numpy(sigma).cuda().requires_grad_(True)
    t = torch.from_numpy(target).cuda()
    x = hyperdiff_steps(c, s, T, checkpoint_every=k)
    loss = ((x - t) ** 2).sum()
    loss.backward()
    return float(loss.item()), c.grad.cpu().numpy(), s.grad.cpu().numpy()


def gpu_loss(c0, sigma, target, T):
    with torch.no_grad():
        x = hyperdiff_steps(torch.from_numpy(c0).cuda(), torch.from_numpy(sigma).cuda(), T, 10)
        return float(((x - torch.from_numpy(target).cuda()) ** 2).sum().item())


def nrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("batch,n,T,k", [(37, 64, 7, 3), (5, 300, 12, 12), (33, 1024, 20, 10)])
def test_gradients_match_oracle_adjoint(batch, n, T, k):
    w, c0, target = make_case(batch, n, T)
    loss_o, gc_o, gs_o = oracle.hyperdiff_loss_grad(w.sigma, T, c0, target)
    loss_g, gc_g, gs_g = gpu_loss_grad(c0, w.sigma, target, T, k)
    print("loss rel", abs(loss_g - loss_o) / loss_o, "dC0", nrel(gc_g, gc_o), "dsigma", nrel(gs_g, gs_o))
    assert abs(loss_g - loss_o) <= 1e-11 * loss_o
    assert nrel(gc_g, gc_o) <= 1e-11
    assert nrel(gs_g, gs_o) <= 1e-11


def test_gradients_match_central_differences():
    batch, n, T = 4, 128, 9
    w, c0, target = make_case(batch, n, T)
    _, gc, gs = gpu_loss_grad(c0, w.sigma, target, T, 4)
    h = 1e-6
    def central(s, step):
        sp, sm = w.sigma.copy(), w.sigma.copy()
        sp[s] += step
        sm[s] -= step
        return (gpu_loss(c0, sp, target, T) - gpu_loss(c0, sm, target, T)) / (2 * step)

    for s in range(batch):
        fd = (4.0 * central(s, h / 2) - central(s, h)) / 3.0
        assert gs[s] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for (s, i) in [(0, 0), (1, 63), (3, 127), (2, 5)]:
        cp, cm = c0.copy(), c0.copy()
        cp[s, i] += h
        cm[s, i] -= h
        fd = (gpu_loss(cp, w.sigma, target, T) - gpu_loss(cm, w.sigma, target, T)) / (2 * h)
        assert gc[s, i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_full_size_differentiation_workload():
    """4,096 systems of N=1024, T = 50, checkpoints every 10 steps.

    The adjoint pass is compared with the oracle's for the same cotangent
    lambda^T (1e-11).  End to end, lambda^T = 2 (x^T - target) is a ~1 %
    difference, so the ~1e-15 relative difference of the two forward
    trajectories is amplified in it; since ||A^{-T}|| <= 1, the dC0 difference is
    bounded by 2 max|x^T_gpu - x^T_oracle|, which is the end-to-end bar."""
    w, c0, target = make_case(4096, 1024, 50)
    loss_o, gc_o, gs_o = oracle.hyperdiff_loss_grad(w.sigma, 50, c0, target)
    c = torch.from_numpy(c0).cuda().requires_grad_(True)
    s = torch.from_numpy(w.sigma).cuda().requires_grad_(True)
    x = hyperdiff_steps(c, s, 50, checkpoint_every=10)
    xT_g = x.detach().cpu().numpy()
    xT_o = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, 50).reshape(4096, 1024)
    lam = 2.0 * (xT_o - target)
    x.backward(torch.from_numpy(lam).cuda())
    vc_o, vs_o = oracle.hyperdiff_vjp(w.sigma, 50, c0, lam)
    print("full vjp: dC0", nrel(c.grad.cpu().numpy(), vc_o), "dsigma", nrel(s.grad.cpu().numpy(), vs_o))
    assert nrel(c.grad.cpu().numpy(), vc_o) <= 1e-11
    assert nrel(s.grad.cpu().numpy(), vs_o) <= 1e-11
    loss_g, gc_g, gs_g = gpu_loss_grad(c0, w.sigma, target, 50, 10)
    dx = float(np.max(np.abs(xT_g - xT_o)))
    print("full: loss rel", abs(loss_g - loss_o) / loss_o, "dC0", nrel(gc_g, gc_o), "dsigma", nrel(gs_g, gs_o),
          "max|dxT|", dx)
    assert abs(loss_g - loss_o) <= 1e-11 * loss_o
    assert np.max(np.abs(gc_g - gc_o)) <= max(1e-11 * np.max(np.abs(gc_o)), 2.0 * 2.0 * dx)
    assert nrel(gs_g, gs_o) <= 1e-11


@pytest.mark.parametrize("batch,n,T,k", [(37, 64, 7, 3), (33, 1024, 20, 10)])
def test_f32_refine_gradients(batch, n, T, k):
    """The same gradients with FP32+refine solves (max_refine = 2); A = I + sigma D4 is
    symmetric, so the adjoint solves run through the FP32 kernel too.  Bars from the
    per-solve parity bar eps = 1e-12 (every FP32+refine solve meets it) and ||A^{-1}|| <= 1,
    so solve errors add over the steps: x^T within T eps; the vector-Jacobian product for the
    oracle's cotangent within 2 T eps (T adjoint solves on T recomputed states); the loss
    gradient within (amp + 2) T eps, where amp = max|x^T| / max|x^T - target| (~250 here) is
    how much the cotangent 2 (x^T - target) magnifies the error of x^T."""
    from paper_1807_07382_gb300 import PENT_F32_REFINE
    eps = 1e-12
    w, c0, target = make_case(batch, n, T)
    xT_o = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, T).reshape(batch, n)
    lam = 2.0 * (xT_o - target)
    c = torch.from_numpy(c0).cuda().requires_grad_(True)
    s = torch.from_numpy(w.sigma).cuda().requires_grad_(True)
    x = hyperdiff_steps(c, s, T, checkpoint_every=k, precision=PENT_F32_REFINE, max_refine=2)
    assert nrel(x.detach().cpu().numpy(), xT_o) <= T * eps
    x.backward(torch.from_numpy(lam).cuda())
    vc_o, vs_o = oracle.hyperdiff_vjp(w.sigma, T, c0, lam)
    assert nrel(c.grad.cpu().numpy(), vc_o) <= 2 * T * eps
    assert nrel(s.grad.cpu().numpy(), vs_o) <= 2 * T * eps
    amp = float(np.max(np.abs(xT_o)) / np.max(np.abs(xT_o - target)))
    _, gc_o, gs_o = oracle.hyperdiff_loss_grad(w.sigma, T, c0, target)
    c2 = torch.from_numpy(c0).cuda().requires_grad_(True)
    s2 = torch.from_numpy(w.sigma).cuda().requires_grad_(True)
    x2 = hyperdiff_steps(c2, s2, T, checkpoint_every=k, precision=PENT_F32_REFINE, max_refine=2)
    gc, gs = torch.autograd.grad(((x2 - torch.from_numpy(target).cuda()) ** 2).sum(), (c2, s2))
    print("f32 loss gradient: dC0", nrel(gc.cpu().numpy(), gc_o), "dsigma", nrel(gs.cpu().numpy(), gs_o), "amp", amp)
    assert nrel(gc.cpu().numpy(), gc_o) <= (amp + 2) * T * eps
    assert nrel(gs.cpu().numpy(), gs_o) <= (amp + 2) * T * eps
