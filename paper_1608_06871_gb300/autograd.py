"""torch.autograd wrapper of the misfit and its adjoint-state gradient (Theorem 3.2).

``misfit(c, solver, k, data, alphas, thetas)`` returns 0.5 ||F_k(c) - data||^2
for the real sine coefficients c (eq. sineseries).  The forward pass factors
the operator for c (hs_build) and runs hs_gradient_dev, which solves the
forward problems and one adjoint sweep over the receivers and contracts them
into the gradient without forming the Jacobian; backward returns that
gradient times the incoming scalar.  Factors are recomputed per call (per
frequency in a sweep), not kept across calls.

Arguments: c -- torch float64 (S1, S2); data -- CUDA float64 (M, P, 2);
alphas, thetas -- CUDA float64 (M,), (P,).  The gradient kernels run on
torch's current stream of data's device, so inputs produced there just
before the call are read after they are written.
"""
from __future__ import annotations

import torch

from . import hs_build, hs_gradient_dev


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, solver, k, data, alphas, thetas):
        hs_build(solver.ctx, c.detach().to("cpu", torch.float64).numpy(), float(k))
        grad = torch.empty(c.shape, dtype=torch.float64, device=data.device)
        mis = torch.empty(1, dtype=torch.float64, device=data.device)
        # enqueued on torch's current stream of that device: the adjoint-state
        # kernels start only after the kernels and copies that produced data,
        # alphas and thetas, and torch reads grad and mis in stream order
        # (torch's default stream has handle 0, which the C ABI reads as "the
        # context's own stream": pass cudaStreamLegacy, handle 1, instead)
        stream = torch.cuda.current_stream(data.device).cuda_stream or 1
        hs_gradient_dev(solver.ctx, data, alphas, thetas, grad, mis, stream=stream)
        ctx.save_for_backward(grad.to(c.device))
        return mis[0].to(c.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None, None


def misfit(c, solver, k, data, alphas, thetas):
    return _Misfit.apply(c, solver, k, data, alphas, thetas)
