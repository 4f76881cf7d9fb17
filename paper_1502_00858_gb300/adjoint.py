"""Adjoint of the augmented Lagrangian behind torch.autograd.Function.

Forward runs the library's residual/gradient sweep (calib_eval) on the GPU and returns
L_i(J, Z, Y) per agent (Eq. sumtrace2) for the context's data and consensus state; the same
pass yields grad_i(L_i, J) of Eq. gradL, the gradient w.r.t. the inner product
h(xi, eta) = trace(xi^H eta + eta^H xi) of Eq. inprod. PyTorch's gradient of a real loss
with respect to a complex tensor is dL/dRe + i dL/dIm, which is twice that gradient; backward
returns 2 * grad_h scaled by the incoming gradient. Marshalling only: no arithmetic of the
method runs in Python.
"""
from __future__ import annotations

import torch

from . import capi


class ADMMLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, J: torch.Tensor, calibrator) -> torch.Tensor:
        if not (J.is_cuda and J.dtype == torch.complex64):
            raise TypeError("J must be a complex64 CUDA tensor of shape [A, K, N, 2, 2]")
        Jc = J.detach().contiguous()
        if tuple(Jc.shape) != tuple(calibrator.jones_shape):
            raise ValueError(f"J has shape {tuple(Jc.shape)}, expected {calibrator.jones_shape}")
        A = calibrator.A
        L = torch.empty(A, dtype=torch.float64, device=J.device)
        g = torch.empty(A, dtype=torch.float64, device=J.device)
        grad = torch.empty_like(Jc)
        torch.cuda.current_stream(J.device).synchronize()  # J is complete before the library stream reads it
        capi.calib_eval(calibrator.ctx, torch.view_as_real(Jc), L, g, torch.view_as_real(grad))
        capi.calib_sync(calibrator.ctx)
        ctx.save_for_backward(grad)
        return L

    @staticmethod
    def backward(ctx, grad_L: torch.Tensor):
        (grad_h,) = ctx.saved_tensors
        scale = grad_L.to(torch.float32).reshape(-1, 1, 1, 1, 1)
        return 2.0 * scale * grad_h, None


def admm_loss(J: torch.Tensor, calibrator) -> torch.Tensor:
    """Per-agent augmented Lagrangian L_i(J_i, Z, Y_i), differentiable with respect to J."""
    return ADMMLoss.apply(J, calibrator)
