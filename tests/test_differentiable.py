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


def test_unweighted_forward_gradient_is_the_unweighted_adjoint():
    """y = E f (no weights): its backward is E^H (tffr_adjoint_unweighted)."""
    from paper_1910_10908_gb300 import Plan
    from paper_1910_10908_gb300.differentiable import tffr_samples
    lx, ly, _ = stolt_points(40, 96, 32)
    N = lx.shape[0]
    g = np.random.default_rng(12)
    f0 = dev((g.standard_normal((32, 32)) + 1j * g.standard_normal((32, 32))).astype(np.complex64))
    c = dev((g.standard_normal(N) + 1j * g.standard_normal(N)).astype(np.complex64))
    with Plan(32, width=8) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(tau=1.02, count=False)            # weights that must not enter this map
        f = f0.clone().requires_grad_(True)
        (torch.conj(c) * tffr_samples(plan, f, apply_weights=False)).real.sum().backward()

        def loss(ff):
            return float((torch.conj(c) * tffr_samples(plan, ff.reshape(32, 32), apply_weights=False)).real.sum())

        assert fd_check(loss, f0.flatten(), f.grad.flatten(), 64, 1e-2) < 1e-4
        # and E^H c itself against the FP64 sum with alpha_n = 1
        img = plan.adjoint_unweighted(c).cpu().numpy().astype(np.complex128)
    ref = oracle.adjoint_image(lx, ly, c.cpu().numpy(), None, 32, 32)
    assert np.linalg.norm(img - ref) / np.linalg.norm(ref) <= 1e-5


def _stripmap_2048():
    from synth import make_workload
    return make_workload("stripmap_2048")


def test_gradients_against_the_fp64_oracle_at_the_2048_configuration():
    """Differentiable tFFR at its own configuration (1024 pulses x 2048 frequencies,
    2,089,290 samples -> 2048^2 image): for L = Re <c, E^H D y>, the gradients
    grad_y = D E c and grad_D = Re(conj(E c) y) from the hand-written backward against
    the FP64 oracle's forward sum, at sampled samples (the first, the last and random
    ones), for the plan's tFFR weights and for user weights.  The backward is the forward
    twin of a white image c, whose energy reaches the image edges, where the width-6 kernel
    sits at ~1.1e-5: width 8 here, as in the other white-input parity tests."""
    from paper_1910_10908_gb300 import Plan
    from paper_1910_10908_gb300.differentiable import tffr_image
    wl = _stripmap_2048()
    M, N = wl.M, wl.N
    g = np.random.default_rng(13)
    c_np = (g.standard_normal((M, M)) + 1j * g.standard_normal((M, M))).astype(np.complex64)
    D_np = oracle.tffr_weights(wl.lam_x, M, tau=1.02)          # zeros included
    idx = np.concatenate([[0, N - 1], g.integers(0, N, 94)])
    Ec = oracle.forward_samples(wl.lam_x, wl.lam_y, c_np, None, idx=idx)
    with Plan(M, width=8) as plan:
        plan.set_points(dev(wl.lam_x), dev(wl.lam_y))
        plan.weights(tau=1.02, count=False)
        y = dev(wl.values).requires_grad_(True)
        D = dev(D_np).float().requires_grad_(True)
        c = dev(c_np)
        (torch.conj(c) * tffr_image(plan, y, D)).real.sum().backward()
        gy = y.grad.cpu().numpy().astype(np.complex128)
        gD = D.grad.cpu().numpy().astype(np.float64)
        # the plan's own weights (no D argument): the same grad_y
        y2 = dev(wl.values).requires_grad_(True)
        plan.weights(tau=1.02, count=False)
        (torch.conj(c) * tffr_image(plan, y2)).real.sum().backward()
        gy2 = y2.grad.cpu().numpy().astype(np.complex128)
    ref_y = D_np[idx] * Ec
    ref_D = (np.conj(Ec) * wl.values[idx].astype(np.complex128)).real
    assert np.linalg.norm(gy[idx] - ref_y) / np.linalg.norm(ref_y) <= 1e-5
    assert np.linalg.norm(gy2[idx] - ref_y) / np.linalg.norm(ref_y) <= 1e-5
    assert np.linalg.norm(gD[idx] - ref_D) / np.linalg.norm(ref_D) <= 1e-5


def test_finite_differences_on_64_directions_at_the_2048_configuration():
    """The maps are linear, so central differences along 64 random directions equal the
    directional derivatives up to FP32 rounding and the small mismatch between the
    approximate adjoint and its forward twin, for the sample values and the weights.  The
    deviation is measured against the largest directional derivative (a random direction
    can make one derivative arbitrarily small)."""
    from paper_1910_10908_gb300 import Plan
    from paper_1910_10908_gb300.differentiable import tffr_image
    wl = _stripmap_2048()
    M, N = wl.M, wl.N
    gen = torch.Generator(device="cuda").manual_seed(14)
    with Plan(M) as plan:
        plan.set_points(dev(wl.lam_x), dev(wl.lam_y))
        y0 = dev(wl.values)
        D0 = dev(oracle.tffr_weights(wl.lam_x, M)).float()
        c = torch.randn((M, M), dtype=torch.complex64, device="cuda", generator=gen)

        def loss(y, D):
            with torch.no_grad():
                return float((torch.conj(c) * tffr_image(plan, y, D)).to(torch.complex128).real.sum())

        y = y0.clone().requires_grad_(True)
        D = D0.clone().requires_grad_(True)
        (torch.conj(c) * tffr_image(plan, y, D)).real.sum().backward()
        dev_y = dev_D = scale_y = scale_D = 0.0
        for _ in range(64):
            dy = torch.randn(N, dtype=torch.complex64, device="cuda", generator=gen)
            dD = torch.randn(N, dtype=torch.float32, device="cuda", generator=gen)
            fd_y = (loss(y0 + dy, D0) - loss(y0 - dy, D0)) / 2.0
            an_y = float((torch.conj(y.grad).to(torch.complex128) * dy).real.sum())
            fd_D = (loss(y0, D0 + dD) - loss(y0, D0 - dD)) / 2.0
            an_D = float((D.grad.double() * dD.double()).sum())
            dev_y, scale_y = max(dev_y, abs(fd_y - an_y)), max(scale_y, abs(an_y))
            dev_D, scale_D = max(dev_D, abs(fd_D - an_D)), max(scale_D, abs(an_D))
    assert dev_y < 1e-4 * scale_y and dev_D < 1e-4 * scale_D, (dev_y / scale_y, dev_D / scale_D)


def test_twenty_iterations_of_toeplitz_cg_at_the_2048_configuration():
    """20 CG iterations on E^H D E f = E^H D y at 2048^2 (2,089,290 samples): the residual
    falls, and the Toeplitz operator gives the image of the forward + adjoint operator."""
    from paper_1910_10908_gb300 import Plan
    wl = _stripmap_2048()
    with Plan(wl.M) as plan:
        plan.set_points(dev(wl.lam_x), dev(wl.lam_y))
        plan.weights(count=False)
        y = dev(wl.values)
        b = plan.adjoint(y).clone()
        plan.normal_setup()
        f_t, hist_t = plan.cg(y, iters=20, toeplitz=True)
        f_t = f_t.clone()
        f_s, hist_s = plan.cg(y, iters=20, toeplitz=False)
        # the first CG residual is b = E^H D y itself
        assert abs(hist_t[0] - float(torch.linalg.vector_norm(b))) <= 1e-5 * hist_t[0]
        rel = float(torch.linalg.vector_norm(f_t - f_s) / torch.linalg.vector_norm(f_s))
        # the true residual of the result, with the forward + adjoint operator
        Nf = plan.adjoint(plan.forward(f_t, apply_weights=False))
        true_res = float(torch.linalg.vector_norm(b - Nf))
    assert len(hist_t) == 21 and hist_t[-1] < 0.05 * hist_t[0], hist_t
    assert hist_s[-1] < 0.05 * hist_s[0], hist_s
    assert rel < 1e-3, rel
    assert true_res < 0.1 * hist_t[0], (true_res, hist_t[0])
