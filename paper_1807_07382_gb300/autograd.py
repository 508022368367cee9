"""Differentiable implicit hyperdiffusion stepping through the library's kernels.

Forward: x^0 = C0, (I + sigma_s D4) x^k = x^{k-1} for k = 1..T (the implicit
step of the hyperdiffusion scheme, Sec. 2.2-2.3, with the factor-once /
solve-many use of Sec. 2.6).  Backward, by the discrete adjoint: with
lambda^T = dL/dx^T, for k = T..1

    mu^k = A^{-T} lambda^k                       (pent_adjoint_solve_batch)
    dL/dsigma_s -= (mu^k_s) . (D4 x^k_s)         (pent_hyperdiff_sigma_grad)
    lambda^{k-1} = mu^k

which follows from A x^k = x^{k-1} and dA/dsigma = D4; dL/dC0 = lambda^0.
States are kept only every `checkpoint_every` steps; the backward pass
recomputes each segment's states from its checkpoint with the forward solve
before walking it in reverse.  Every solve, adjoint solve and reduction runs
in the CUDA library; this module only orders the calls.
"""
from __future__ import annotations

import torch

from . import PENT_F32_REFINE, PENT_F64, Plan


class _Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c0, sigma, T: int, checkpoint_every: int, precision: int, max_refine: int):
        if c0.dtype != torch.float64 or sigma.dtype != torch.float64:
            raise TypeError("c0 and sigma must be float64")
        if not (c0.is_cuda and sigma.is_cuda):
            raise ValueError("c0 and sigma must be CUDA tensors")
        batch, n = c0.shape
        if sigma.shape != (batch,):
            raise ValueError("sigma must have shape (batch,)")
        k = max(1, int(checkpoint_every))
        if precision not in (PENT_F64, PENT_F32_REFINE):
            raise ValueError("precision must be PENT_F64 or PENT_F32_REFINE")
        plan = Plan(n, batch=batch, precision=precision, device=c0.device)
        sig = sigma.detach().contiguous()
        plan.factor_hyperdiff(sig)
        x = c0.detach().contiguous().clone()
        checkpoints = [x.clone()]
        for step in range(1, T + 1):
            plan.solve(x, x, max_refine=max_refine)
            if step % k == 0 and step < T:
                checkpoints.append(x.clone())
        ctx.plan = plan
        ctx.max_refine = max_refine
        ctx.sig = sig
        ctx.T = T
        ctx.k = k
        ctx.checkpoints = checkpoints
        return x.clone()

    @staticmethod
    def backward(ctx, grad_xT):
        plan, T, k = ctx.plan, ctx.T, ctx.k
        lam = grad_xT.detach().contiguous().clone()
        gsig = torch.zeros_like(ctx.sig)
        mu = torch.empty_like(lam)
        # segments [s0, s1): states x^{s0} .. x^{s1}; checkpoint j holds x^{j k}
        for j in range(len(ctx.checkpoints) - 1, -1, -1):
            s0 = j * k
            s1 = min(T, s0 + k)
            states = [ctx.checkpoints[j]]
            x = ctx.checkpoints[j].clone()
            for _ in range(s0, s1):
                plan.solve(x, x, max_refine=ctx.max_refine)
                states.append(x.clone())
            for step in range(s1, s0, -1):
                plan.adjoint_solve(lam, mu, max_refine=ctx.max_refine)
                plan.sigma_grad(mu, states[step - s0], gsig)
                lam, mu = mu, lam
        ctx.checkpoints = None
        return lam, gsig, None, None, None, None


def hyperdiff_steps(c0, sigma, T: int, checkpoint_every: int = 10, precision: int = PENT_F64, max_refine: int = 2):
    """x^T after T implicit hyperdiffusion steps from c0 (batch x n) with per-system
    sigma (batch,), differentiable w.r.t. c0 and sigma.  precision: PENT_F64, or
    PENT_F32_REFINE (FP32 solves refined against the float-float residual, up to
    max_refine steps each; A = I + sigma D4 is symmetric, so the adjoint solves run
    through the same kernel)."""
    return _Steps.apply(c0, sigma, int(T), int(checkpoint_every), int(precision), int(max_refine))
