"""Differentiable tFFR and a least-squares image solver, on the library's kernels.

With E the non-uniform Fourier matrix (E[n, j] = exp(-2 pi i lam_n . x_j)) and
D = diag(D_n) the frame weights, the library's two calls are

    adjoint:  f = E^H D y        (the tFFR image, Eq. (fstraight) with alpha_n = D_n)
    forward:  y = D E f          (apply_weights=True)   or   E f   (apply_weights=False)

so each is the other's Hermitian transpose and serves as its backward pass.
PyTorch's convention for a real loss L of complex tensors is that a tensor's
gradient is dL/d(conj z) (up to the factor 2 shared by every tensor), hence for
f = E^H D y:

    grad_y = D E grad_f                       (the forward twin with weights)
    grad_D = Re(conj(E grad_f) * y)           (real weights, USER mode)

Every product runs in the CUDA kernels; this module only orders the calls.
"""

from __future__ import annotations

import torch

from . import Plan


def _c64(t: torch.Tensor) -> torch.Tensor:
    return t if t.dtype == torch.complex64 else t.to(torch.complex64)


class _Adjoint(torch.autograd.Function):
    """f = E^H D y (D: the plan's weights, or the given user weights)."""

    @staticmethod
    def forward(ctx, values, D, plan: Plan):
        if D is not None:
            plan.weights(mode="user", user_D=D.detach().float().contiguous(), count=False)
        f = plan.adjoint(_c64(values).contiguous())
        ctx.plan = plan
        ctx.save_for_backward(values, D)
        return f

    @staticmethod
    def backward(ctx, grad_f):
        plan = ctx.plan
        values, D = ctx.saved_tensors
        g = grad_f.contiguous().to(torch.complex64)
        grad_y = grad_D = None
        if D is not None:
            plan.weights(mode="user", user_D=D.detach().float().contiguous(), count=False)
        if ctx.needs_input_grad[0]:
            grad_y = plan.forward(g, apply_weights=True).to(values.dtype)
        if D is not None and ctx.needs_input_grad[1]:
            Eg = plan.forward(g, apply_weights=False).to(torch.complex128)
            grad_D = (Eg.conj() * values.to(torch.complex128)).real.to(D.dtype)
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
        g = grad_y.contiguous().to(torch.complex64)
        if ctx.apply_weights:
            grad_f = plan.adjoint(g)                      # (D E)^H = E^H D
        else:
            # E^H alone: the adjoint with unit weights, then the plan's weights back
            raise NotImplementedError("backward of the unweighted forward needs unit weights; "
                                      "use apply_weights=True or a unit-weight plan")
        return grad_f.to(ctx.dtype), None, None


def tffr_image(plan: Plan, values: torch.Tensor, D: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable f = E^H D y.  With D (real, [N]) the plan switches to USER
    weights and D receives a gradient; without it the plan's current weights
    (set by plan.weights) are used and only the values are differentiated."""
    return _Adjoint.apply(values, D, plan)


def tffr_samples(plan: Plan, image: torch.Tensor) -> torch.Tensor:
    """Differentiable y = D E f with the plan's current weights."""
    return _Forward.apply(image, plan, True)


def cg_normal(plan: Plan, values: torch.Tensor, iters: int = 20, tol: float = 0.0,
              x0: torch.Tensor | None = None, toeplitz: bool = False):
    """Conjugate gradients on the weighted normal equations E^H D E f = E^H D y.

    The minimiser of || D^(1/2) (E f - y) ||^2 over images f.  N f = E^H D E f
    is one forward twin without weights and one adjoint (which applies D), or,
    with toeplitz=True, the plan's Toeplitz normal operator (three line-FFT
    passes on the 2M grid, independent of the number of samples; built here by
    plan.normal_setup()).  Returns (f, residual norms ||b - N f_k|| for
    k = 0..iters).  FP32 kernels: the residual levels off near 1e-6 of ||b||.
    """
    if toeplitz:
        plan.normal_setup()

        def normal(f):
            return plan.normal(f.contiguous())
    else:
        def normal(f):
            return plan.adjoint(plan.forward(f.contiguous(), apply_weights=False))

    b = plan.adjoint(_c64(values).contiguous())
    x = torch.zeros_like(b) if x0 is None else x0.to(torch.complex64).clone()
    r = b - normal(x) if x0 is not None else b.clone()
    p = r.clone()
    rr = torch.vdot(r.flatten(), r.flatten()).real
    hist = [float(rr.sqrt())]
    bnorm = float(torch.linalg.vector_norm(b))
    for _ in range(iters):
        Ap = normal(p)
        alpha = rr / torch.vdot(p.flatten(), Ap.flatten()).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = torch.vdot(r.flatten(), r.flatten()).real
        hist.append(float(rr_new.sqrt()))
        if tol > 0 and hist[-1] <= tol * bnorm:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, hist
