"""torch.autograd wrapper of the rational pseudofermion action

    S(phi, U) = sum_s c_s Re(phi^dag (A[U] + sigma_s)^{-1} phi),

A[U] = m^2 - D[U]^2 the staggered operator. The forward pass solves every
shift with msc_solve (one Krylov sequence, CG-M) and evaluates S with
msc_quad_form; the backward pass returns dS/dphi and the link force dS/dU
from msc_quad_form_grad (hand-written CUDA kernels: D x_s passes and an
outer-product stencil over links), in torch's convention for complex leaves.
With recompute=True the solutions are not kept between forward and backward
but solved again from the saved phi and links, trading one solve for
S x n complex values of memory.
"""
from __future__ import annotations

import torch

from . import (MSC_FP64, MSC_MIXED, default_context, msc_op_destroy,
               msc_op_staggered, msc_quad_form, msc_quad_form_grad, solve)


def _solve_all(h, phi, links, dims, nc, mass, sigma, tol, precision):
    op = msc_op_staggered(h, nc, dims, links.detach().contiguous(), mass)
    x, info = solve(h, op, phi.detach().contiguous(), sigma, tol=tol, precision=precision)
    return op, x, info


class MultiShiftQuadForm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, links, sigma, c, dims, nc, mass, tol=1e-10, precision=MSC_MIXED,
                recompute=False):
        dev = phi.device.index or 0
        h = default_context(dev)
        sig = torch.as_tensor(sigma, dtype=torch.float64).cpu().numpy()
        cc = torch.as_tensor(c, dtype=torch.float64).cpu().numpy()
        op, x, info = _solve_all(h, phi, links, dims, nc, mass, sig, tol, precision)
        try:
            val = msc_quad_form(h, op, phi.detach().contiguous(), len(sig), cc, x)
        finally:
            msc_op_destroy(op)
        ctx.meta = (h, tuple(dims), nc, mass, sig, cc, tol, precision, recompute)
        ctx.info = info
        if recompute:
            ctx.save_for_backward(phi.detach(), links.detach())
        else:
            ctx.save_for_backward(x, links.detach())
        return torch.tensor(val, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, g):
        h, dims, nc, mass, sig, cc, tol, precision, recompute = ctx.meta
        a, links = ctx.saved_tensors
        op = msc_op_staggered(h, nc, dims, links.contiguous(), mass)
        try:
            if recompute:
                x, _ = solve(h, op, a.contiguous(), sig, tol=tol, precision=precision)
            else:
                x = a
            dphi = torch.empty(x.shape[-1], dtype=torch.complex128, device=x.device)
            dU = torch.empty_like(links)
            msc_quad_form_grad(h, op, len(sig), cc, x.contiguous(), dphi, dU)
        finally:
            msc_op_destroy(op)
        gs = g.to(torch.float64)
        return (gs * dphi if ctx.needs_input_grad[0] else None,
                gs * dU if ctx.needs_input_grad[1] else None,
                None, None, None, None, None, None, None, None)


def quad_form(phi, links, sigma, c, dims, nc, mass, tol=1e-10, precision=MSC_MIXED,
              recompute=False):
    """S = sum_s c_s Re(phi^dag (A + sigma_s)^{-1} phi), differentiable in phi
    (complex128 [V*nc], CUDA) and links (complex128 [4][V][nc][nc], CUDA)."""
    return MultiShiftQuadForm.apply(phi, links, sigma, c, dims, nc, mass, tol, precision, recompute)


__all__ = ["MultiShiftQuadForm", "quad_form", "MSC_FP64", "MSC_MIXED"]
