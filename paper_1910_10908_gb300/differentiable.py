"""Differentiable tFFR and a least-squares image solver, on the library's kernels.

With E the non-uniform Fourier matrix (E[n, j] = exp(-2 pi i lam_n . x_j)) and
D = diag(D_n) the frame weights, the library's calls are

    adjoint:             f = E^H D y     (the tFFR image, Eq. (fstraight) with alpha_n = D_n)
    adjoint_unweighted:  f = E^H y
    forward:             y = D E f       (apply_weights=True)   or   E f   (apply_weights=False)

so each serves as another's backward pass.  PyTorch's convention for a real
loss L of complex tensors is that a tensor's gradient is dL/d(conj z) (up to
the factor 2 shared by every tensor), hence for f = E^H D y:

    grad_y = D E grad_f                       (the forward twin with weights)
    grad_D = Re(conj(E grad_f) * y)           (real weights, USER mode: tffr_weight_grad)

and for y = D E f, grad_f = E^H D grad_y; for y = E f, grad_f = E^H grad_y.
Every product, and every step of the conjugate-gradient solver, runs in the
library's CUDA kernels; this module orders the calls and converts dtypes.
"""

from __future__ import annotations

import torch

from . import Plan


def _c64(t: torch.Tensor) -> torch.Tensor:
    return t if t.dtype == torch.complex64 else t.to(torch.complex64)


def _set_user_weights(plan: Plan, D):
    if D is not None:
        plan.weights(mode="user", user_D=D.detach().float().contiguous(), count=False)


class _Adjoint(torch.autograd.Function):
    """f = E^H D y (D: the plan's weights, or the given user weights)."""

    @staticmethod
    def forward(ctx, values, D, plan: Plan):
        _set_user_weights(plan, D)
        v = _c64(values).contiguous()
        f = plan.adjoint(v)
        ctx.plan = plan
        ctx.values_dtype = values.dtype
        ctx.save_for_backward(v, D)
        return f

    @staticmethod
    def backward(ctx, grad_f):
        plan = ctx.plan
        v, D = ctx.saved_tensors
        g = _c64(grad_f).contiguous()
        grad_y = grad_D = None
        _set_user_weights(plan, D)
        if ctx.needs_input_grad[0]:
            grad_y = plan.forward(g, apply_weights=True).to(ctx.values_dtype)
        if D is not None and ctx.needs_input_grad[1]:
            grad_D = plan.weight_grad(g, v).to(D.dtype)
        return grad_y, grad_D, None


class _Forward(torch.autograd.Function):
    """y = D E f (apply_weights) or E f."""

    @staticmethod
    def forward(ctx, image, plan: Plan, apply_weights: bool):
        ctx.plan, ctx.apply_weights = plan, apply_weights
        ctx.dtype = image.dtype
        return plan.forward(_c64(image).contiguous(), apply_weights=apply_weights)

    @staticmethod
    def backward(ctx, grad_y):
        plan = ctx.plan
        g = _c64(grad_y).contiguous()
        if ctx.apply_weights:
            grad_f = plan.adjoint(g)                      # (D E)^H = E^H D
        else:
            grad_f = plan.adjoint_unweighted(g)           # E^H
        return grad_f.to(ctx.dtype), None, None


def tffr_image(plan: Plan, values: torch.Tensor, D: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable f = E^H D y.  With D (real, [N]) the plan switches to USER
    weights and D receives a gradient; without it the plan's current weights
    (set by plan.weights) are used and only the values are differentiated."""
    return _Adjoint.apply(values, D, plan)


def tffr_samples(plan: Plan, image: torch.Tensor, apply_weights: bool = True) -> torch.Tensor:
    """Differentiable y = D E f (or E f with apply_weights=False) with the plan's current weights."""
    return _Forward.apply(image, plan, apply_weights)


def cg_normal(plan: Plan, values: torch.Tensor, iters: int = 20, toeplitz: bool = False):
    """Conjugate gradients on the weighted normal equations E^H D E f = E^H D y, from f = 0.

    The minimiser of || D^(1/2) (E f - y) ||^2 over images f.  E^H D E is one
    forward twin without weights and one adjoint (which applies D), or, with
    toeplitz=True, the plan's Toeplitz normal operator (three line-FFT passes on
    the 2M grid, independent of the number of samples; built here by
    plan.normal_setup()).  The whole iteration (operator, dot products, vector
    updates) runs in the library (tffr_cg).  Returns (f, residual norms
    ||b - N f_k|| for k = 0..iters).  FP32 kernels: the residual levels off near
    1e-6 of ||b||.
    """
    if toeplitz:
        plan.normal_setup()
    return plan.cg(_c64(values).contiguous(), iters=iters, toeplitz=toeplitz)
