"""Differentiable tFFR (autograd through the adjoint and the forward twin) and
the conjugate-gradient solver of the weighted normal equations, on the GPU.

Gradients are checked against central finite differences along 64 random
directions (the maps are linear, so the differences are exact up to FP32
rounding); the solver against the least-squares solution computed in FP64
from the explicit matrix E[n, j] = exp(-2 pi i lam_n . x_j) on a small grid.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import random_points, stolt_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def fd_check(L, x, grad, dirs, eps, real=False):
    """max over directions of |FD - Re(<grad, d>)| / scale."""
    g = np.random.default_rng(5)
    worst, scale = 0.0, 0.0
    for _ in range(dirs):
        if real:
            d = torch.from_numpy(g.standard_normal(x.shape[0])).to(x.device, x.dtype)
        else:
            d = torch.from_numpy(g.standard_normal(x.shape[0]) + 1j * g.standard_normal(x.shape[0])).to(
                x.device, x.dtype)
        fd = (L(x + eps * d) - L(x - eps * d)) / (2 * eps)
        an = float((torch.conj(grad) * d).real.sum()) if not real else float((grad * d).sum())
        worst = max(worst, abs(fd - an))
        scale = max(scale, abs(an))
    return worst / scale


def test_adjoint_gradients_for_values_and_user_weights():
    from paper_1910_10908_gb300 import Plan
    from paper_1910_10908_gb300.differentiable import tffr_image
    lx, ly, _ = stolt_points(48, 96, 64)
    N = lx.shape[0]
    g = np.random.default_rng(1)
    y0 = dev((g.standard_normal(N) + 1j * g.standard_normal(N)).astype(np.complex128))
    D0 = dev(oracle.tffr_weights(lx, 64)).float()
    c = dev((g.standard_normal((64, 64)) + 1j * g.standard_normal((64, 64))).astype(np.complex64))
    with Plan(64) as plan:
        plan.set_points(dev(lx), dev(ly))

        def loss(y, D):
            return float((torch.conj(c) * tffr_image(plan, y, D)).real.sum().double())

        y = y0.clone().requires_grad_(True)
        D = D0.clone().requires_grad_(True)
        L = (torch.conj(c) * tffr_image(plan, y, D)).real.sum()
        L.backward()
        assert fd_check(lambda yy: loss(yy, D0), y0, y.grad, 64, 1e-2) < 1e-4
        assert fd_check(lambda DD: loss(y0, DD), D0, D.grad, 64, 1e-2, real=True) < 1e-4


def test_forward_twin_gradient_is_the_adjoint():
    from paper_1910_10908_gb300 import Plan
    from paper_1910_10908_gb300.differentiable import tffr_samples
    lx, ly, _ = random_points(3000, 32, seed=4, extent=0.5)
    g = np.random.default_rng(2)
    f0 = dev((g.standard_normal((32, 32)) + 1j * g.standard_normal((32, 32))).astype(np.complex64))
    c = dev((g.standard_normal(3000) + 1j * g.standard_normal(3000)).astype(np.complex64))
    with Plan(32, width=8) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(tau=1.0, count=False)
        f = f0.clone().requires_grad_(True)
        (torch.conj(c) * tffr_samples(plan, f)).real.sum().backward()

        def loss(ff):
            return float((torch.conj(c) * tffr_samples(plan, ff.reshape(32, 32))).real.sum())

        assert fd_check(loss, f0.flatten(), f.grad.flatten(), 64, 1e-2) < 1e-4


def test_cg_reaches_the_weighted_least_squares_image():
    """On a jittered, twice-oversampled grid of frequencies (cond(E^H D E) ~ 5, so the
    comparison measures the solver and not the conditioning) 25 CG steps reach the FP64
    least-squares image to FP32 accuracy."""
    from paper_1910_10908_gb300 import Plan
    from paper_1910_10908_gb300.differentiable import cg_normal
    M = 16
    g = np.random.default_rng(3)
    k = np.arange(-M, M) / 2.0
    KX, KY = np.meshgrid(k, k)
    lx = KX.ravel() + g.uniform(-0.2, 0.2, KX.size)
    ly = KY.ravel() + g.uniform(-0.2, 0.2, KY.size)
    N = lx.shape[0]
    f_true = g.standard_normal((M, M)) + 1j * g.standard_normal((M, M))
    x = (np.arange(M) - M / 2) / M
    E = np.exp(-2j * np.pi * (lx[:, None, None] * x[None, None, :] + ly[:, None, None] * x[None, :, None]))
    E = E.reshape(N, M * M)                     # column j = jy * M + jx
    y = E @ f_true.reshape(-1) + 0.01 * (g.standard_normal(N) + 1j * g.standard_normal(N))
    D = oracle.tffr_weights(lx, M)
    f_ls = np.linalg.lstsq(np.sqrt(D)[:, None] * E, np.sqrt(D) * y, rcond=None)[0].reshape(M, M)
    with Plan(M, width=8) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(count=False)
        f, hist = cg_normal(plan, dev(y.astype(np.complex64)), iters=25)
    f = f.cpu().numpy().astype(np.complex128)
    assert hist[-1] < 1e-5 * hist[0]
    assert np.linalg.norm(f - f_ls) / np.linalg.norm(f_ls) < 1e-4
