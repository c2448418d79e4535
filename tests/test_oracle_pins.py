"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: numerical quadrature of the
defining integrals, Poisson summation, a limit with a textbook answer, dense
matrices built by quadrature from the definitions of Psi and W, numpy's
inverse FFT for the uniform-grid special case, Parseval, the Dirichlet-kernel
closed form of a point scatterer, and adjointness of two separately written
loops.  A last group plants mistakes in copies of the oracle's formulas and
checks that the pins catch them.
"""

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import weights as ow
from synth import stolt_points

A = 0.01


def quad_transform(xi, a, sign):
    """int_{-1/2}^{1/2} exp(sign * a |t|) exp(-2 pi i xi t) dt by adaptive quadrature."""
    f = lambda t: np.exp(sign * a * abs(t))
    re = 2.0 * integrate.quad(f, 0.0, 0.5, weight="cos", wvar=2 * np.pi * xi, epsabs=1e-14, epsrel=1e-13)[0]
    # the odd (sine) part of an even function integrates to zero over a symmetric interval
    im_l = integrate.quad(f, -0.5, 0.0, weight="sin", wvar=2 * np.pi * xi, epsabs=1e-14)[0]
    im_r = integrate.quad(f, 0.0, 0.5, weight="sin", wvar=2 * np.pi * xi, epsabs=1e-14)[0]
    return re, -(im_l + im_r)


@pytest.mark.parametrize("xi", [0.0, 0.3, -0.77, 1.0, 2.7, 17.25, 1000.4])
def test_w_hat_matches_quadrature(xi):
    re, im = quad_transform(xi, A, -1.0)
    assert abs(ow.w_hat(xi, A) - re) < 1e-12
    assert abs(im) < 1e-12


@pytest.mark.parametrize("eta", [0.0, 0.5, -1.3, 2.0, 3.9, 250.1])
def test_psi_hat_matches_quadrature(eta):
    re, _ = quad_transform(eta, A, +1.0)
    assert abs(ow.psi_hat(eta, A) - re) < 1e-12


def test_a_to_zero_gives_sinc():
    xi = np.array([0.0, 0.25, 0.5, 1.5, 2.9])
    assert np.allclose(ow.w_hat(xi, 1e-8), np.sinc(xi), atol=1e-7)
    assert np.allclose(ow.psi_hat(xi, 1e-8), np.sinc(xi), atol=1e-7)


def test_untruncated_diagonal_is_partition_of_unity():
    """Poisson summation: sum_j psi(d - j) w_hat(j - d) = (w 1 * w^-1 1)(0) = 1.

    The convolution of exp(-a|t|) and exp(+a|t|) (both cut to [-1/2, 1/2])
    equals 1 at t = 0 and 0 at every other integer, so the full sum over the
    integer grid is 1 for every offset d; the truncated sums approach it like 1/J.
    """
    rng = np.random.default_rng(3)
    d = rng.uniform(0, 1, 16)
    errs = []
    for J in (250, 2000, 16000):
        j = np.arange(-J, J + 1)[:, None]
        s = np.sum(ow.psi_hat(d[None, :] - j, A) * ow.w_hat(j - d[None, :], A), axis=0)
        errs.append(np.max(np.abs(s - 1.0)))
    assert errs[2] < 2e-5
    assert errs[0] > errs[1] > errs[2]


def test_truncated_diagonal_sinc_squared_limit():
    """a -> 0: G(d) -> sum_{|d-j|<q} sinc^2(d - j), a textbook sum; G(1/2) at q=3 is 0.9331."""
    d = np.array([0.1, 0.37, 0.5, 0.81]) + 5.0
    G = ow.diag_psi_w(d, 64, q=3.0, a=1e-7)
    ref = []
    for v in d:
        j = np.arange(np.floor(v) - 4, np.floor(v) + 6)
        j = j[np.abs(v - j) < 3.0]
        ref.append(np.sum(np.sinc(v - j) ** 2))
    assert np.allclose(G, ref, atol=1e-6)
    half = 2 * (4 / np.pi**2) * (1 + 1 / 9 + 1 / 25)
    assert abs(ow.diag_psi_w(np.array([0.5]), 64, q=3.0, a=1e-7)[0] - half) < 1e-6


def _dense_psi_w_by_quadrature(lam, ell, a):
    """Psi (P x M) and W (M x P) from their defining integrals, complex quadrature."""
    P, M = lam.shape[0], ell.shape[0]
    Psi = np.zeros((P, M), complex)
    W = np.zeros((M, P), complex)
    inv_w = lambda t: np.exp(a * abs(t))
    w = lambda t: np.exp(-a * abs(t))
    for p in range(P):
        for m in range(M):
            # <e^{2 pi i lam t}, e^{2 pi i ell t}/w> = int e^{2 pi i (lam - ell) t} / w(t) dt
            om = 2 * np.pi * (lam[p] - ell[m])
            re = integrate.quad(lambda t: inv_w(t) * np.cos(om * t), -0.5, 0.5, epsabs=1e-13, limit=200)[0]
            im = integrate.quad(lambda t: inv_w(t) * np.sin(om * t), -0.5, 0.5, epsabs=1e-13, limit=200)[0]
            Psi[p, m] = re + 1j * im
            # w_hat(ell - lam) = int w(t) e^{-2 pi i (ell - lam) t} dt
            om2 = 2 * np.pi * (ell[m] - lam[p])
            re = integrate.quad(lambda t: w(t) * np.cos(om2 * t), -0.5, 0.5, epsabs=1e-13, limit=200)[0]
            im = -integrate.quad(lambda t: w(t) * np.sin(om2 * t), -0.5, 0.5, epsabs=1e-13, limit=200)[0]
            W[m, p] = re + 1j * im
    return Psi, W


def test_diagonal_from_dense_matrices_built_by_quadrature():
    """Build Psi and banded W from their definitions; diag(Psi W) and R_tau(pinv) match."""
    M = 16
    rng = np.random.default_rng(7)
    lam = np.sort(rng.uniform(-6.5, 6.5, 6))
    lam[0] = -7.2  # within q of the grid edge l = -8: truncation by the finite grid
    ell = np.arange(-M // 2, M // 2, dtype=float)
    Psi, W = _dense_psi_w_by_quadrature(lam, ell, A)
    band = np.abs(lam[:, None] - ell[None, :]) < 3.0     # |lam_p - l_m| < q
    Psi_b = np.where(band, Psi, 0)
    W_b = np.where(band.T, W, 0)
    G = np.diag(Psi_b @ W_b)
    assert np.max(np.abs(G.imag)) < 1e-12
    assert np.allclose(ow.diag_psi_w(lam, M), G.real, rtol=0, atol=1e-11)
    D_ref = np.diag(np.linalg.pinv(np.diag(G.real)))
    for tau in (0.97, 1.02, 1.05):
        D_ref_t = np.where(D_ref >= tau, D_ref, 0.0)
        assert np.allclose(ow.tffr_weights(lam, M, tau=tau), D_ref_t, atol=1e-11)


def _quad2_nodes(n=48):
    """2-D Gauss-Legendre nodes and weights on [-1/2, 1/2]^2, split at t = 0 on each axis
    (the window exp(-a|t|) has a kink there): n points per half-axis."""
    x, w = np.polynomial.legendre.leggauss(n)
    t = np.concatenate([-0.25 + 0.25 * x, 0.25 + 0.25 * x])     # [-1/2, 0] and [0, 1/2]
    wt = np.concatenate([0.25 * w, 0.25 * w])
    TX, TY = np.meshgrid(t, t, indexing="ij")
    return TX, TY, np.outer(wt, wt)


def test_separable_weights_from_dense_2d_matrices_built_by_quadrature():
    """The separable variant on a tensor-product frame: the 2-D window is w(tx) w(ty), and
    Psi[p, m] = <e^{2 pi i lam_p . t}, e^{2 pi i l_m . t} / w2(t)>, W[m, p] = w2_hat(l_m - lam_p)
    are built by 2-D quadrature over [-1/2, 1/2]^2 on an Mx x My grid with Mx != My, banded by
    |lam_x - l_x| < q and |lam_y - l_y| < q (both grid edges truncate).  diag(Psi W),
    R_tau(pinv) with the threshold on the product, match the oracle's separable branch; a
    mistake that uses lam_x or Mx for both factors, or thresholds each factor, would not."""
    Mx, My, q = 8, 4, 3.0
    lam_x = np.array([-3.6, 0.5, 2.25, 3.9, 0.0])
    lam_y = np.array([0.3, -1.5, 1.7, -0.02, 0.5])
    lx_grid = np.arange(-Mx // 2, Mx // 2, dtype=float)
    ly_grid = np.arange(-My // 2, My // 2, dtype=float)
    TX, TY, WQ = _quad2_nodes()
    w2 = np.exp(-A * np.abs(TX)) * np.exp(-A * np.abs(TY))
    G = np.zeros(lam_x.shape[0], complex)
    for p in range(lam_x.shape[0]):
        for lx_m in lx_grid:
            for ly_m in ly_grid:
                if not (abs(lam_x[p] - lx_m) < q and abs(lam_y[p] - ly_m) < q):
                    continue
                ph = 2j * np.pi * ((lam_x[p] - lx_m) * TX + (lam_y[p] - ly_m) * TY)
                psi = np.sum(WQ * np.exp(ph) / w2)          # <e^{2 pi i lam.t}, e^{2 pi i l.t}/w2>
                wh = np.sum(WQ * w2 * np.exp(ph))           # w2_hat(l - lam) = int w2 e^{-2 pi i (l - lam).t}
                G[p] += psi * wh
    assert np.max(np.abs(G.imag)) < 1e-12
    Gx = ow.diag_psi_w(lam_x, Mx, q, A)
    Gy = ow.diag_psi_w(lam_y, My, q, A)
    assert np.allclose(Gx * Gy, G.real, rtol=0, atol=1e-11)
    D_ref = np.diag(np.linalg.pinv(np.diag(G.real)))
    decided_differently = False
    for tau in (0.97, 1.02, 1.1):
        D_sep = ow.tffr_weights(lam_x, Mx, tau=tau, q=q, lam_y=lam_y, My=My, separable=True)
        assert np.allclose(D_sep, np.where(D_ref >= tau, D_ref, 0.0), atol=1e-11)
        per_factor = np.where((1 / Gx >= tau) & (1 / Gy >= tau), D_ref, 0.0)
        decided_differently |= not np.allclose(D_sep, per_factor)
    assert decided_differently                     # the product decision is what is tested
    # the y edge matters: the same samples on a wide y grid give other weights
    assert not np.allclose(Gy, ow.diag_psi_w(lam_y, 64, q, A), rtol=0, atol=1e-6)
    assert not np.allclose(Gx * Gy, Gx * ow.diag_psi_w(lam_y, Mx, q, A), rtol=0, atol=1e-6)
    assert not np.allclose(Gx * Gy, Gx * ow.diag_psi_w(lam_x, My, q, A), rtol=0, atol=1e-6)


def test_weight_range_for_paper_parameters():
    """With a = 0.01, q = 3: G in [0.933, 1.0000022], so D in [1, 1.072] (tau = 0.97 keeps all)."""
    d = np.linspace(-0.5, 0.5, 2001) + 3.0
    D = ow.tffr_weights(d, 64)
    assert D.min() >= 0.9999978 and D.max() <= 1.0718
    assert np.all(D > 0)


def _uniform_grid(M):
    k = np.arange(-M // 2, M // 2, dtype=float)
    ky, kx = np.meshgrid(k, k, indexing="ij")
    return kx.ravel(), ky.ravel()


def test_uniform_grid_is_inverse_dft():
    """Integer lam covering all M^2 modes, alpha = 1: Eq. (fstraight) is the unnormalised 2-D IDFT."""
    M = 16
    lx, ly = _uniform_grid(M)
    rng = np.random.default_rng(11)
    F = rng.standard_normal(M * M) + 1j * rng.standard_normal(M * M)
    f = oracle.adjoint_image(lx, ly, F, None, M, M)
    A_ = np.zeros((M, M), complex)
    kx, ky = lx.astype(int), ly.astype(int)
    A_[ky % M, kx % M] = F * (-1.0) ** (kx + ky)
    ref = np.fft.ifft2(A_) * M * M
    assert np.max(np.abs(f - ref)) < 1e-11 * np.max(np.abs(ref))
    # Parseval
    assert abs(np.sum(np.abs(f) ** 2) - M * M * np.sum(np.abs(F) ** 2)) < 1e-10 * M * M * np.sum(np.abs(F) ** 2)


def test_point_scatterer_on_a_pixel():
    """fhat_n = exp(-2 pi i lam_n . x0) with x0 a pixel: f(x0) = sum_n D_n exactly, and it is the peak."""
    M = 64
    lx, ly, _ = stolt_points(64, 64, M)
    D = ow.tffr_weights(lx, M)
    jx0, jy0 = 41, 19
    x0 = (jx0 - M // 2) / M
    y0 = (jy0 - M // 2) / M
    th = lx * x0 + ly * y0
    fhat = np.exp(-2j * np.pi * (th - np.floor(th)))
    img = oracle.adjoint_image(lx, ly, fhat, D, M, M)
    assert abs(img[jy0, jx0] - D.sum()) < 1e-12 * D.sum()
    assert np.unravel_index(np.argmax(np.abs(img)), img.shape) == (jy0, jx0)


def test_point_scatterer_off_pixel_is_dirichlet_product():
    """Uniform grid, alpha = 1, target at x0 off the pixel grid: product of Dirichlet kernels

    sum_{k=-M/2}^{M/2-1} e^{2 pi i k u} = e^{-i pi u} sin(pi M u) / sin(pi u).
    """
    M = 16
    lx, ly = _uniform_grid(M)
    x0, y0 = 0.1234, -0.271
    fhat = np.exp(-2j * np.pi * (lx * x0 + ly * y0))
    img = oracle.adjoint_image(lx, ly, fhat, None, M, M)
    x = (np.arange(M) - M // 2) / M

    def dk(u):
        return np.exp(-1j * np.pi * u) * np.sin(np.pi * M * u) / np.sin(np.pi * u)
    ref = dk(x[:, None] - y0) * dk(x[None, :] - x0)
    assert np.max(np.abs(img - ref)) < 1e-10 * np.max(np.abs(ref))


def test_adjointness_of_the_two_sums():
    """<A^H D y, f> = <y, D A f> for the adjoint and forward loops (written separately)."""
    rng = np.random.default_rng(5)
    Mx, My, N = 12, 10, 300
    lx = rng.uniform(-0.45 * Mx, 0.45 * Mx, N)
    ly = rng.uniform(-0.45 * My, 0.45 * My, N)
    D = ow.tffr_weights(lx, Mx, tau=1.02)
    y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    f = rng.standard_normal((My, Mx)) + 1j * rng.standard_normal((My, Mx))
    lhs = np.vdot(f, oracle.adjoint_image(lx, ly, y, D, Mx, My))   # sum conj(f) A^H D y
    rhs = np.vdot(oracle.forward_samples(lx, ly, f, D), y)         # sum conj(D A f) y
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    assert 0 < np.count_nonzero(D) < N


def test_crop_matches_full_image():
    M = 32
    lx, ly, _ = stolt_points(32, 48, M)
    rng = np.random.default_rng(2)
    y = rng.standard_normal(lx.shape[0]) + 1j * rng.standard_normal(lx.shape[0])
    full = oracle.adjoint_image(lx, ly, y, None, M, M)
    crop = oracle.adjoint_image(lx, ly, y, None, M, M, crop=(5, 9, 7, 11))
    assert np.array_equal(crop, full[9:20, 5:12])


# ---- planted mistakes: copies of the formulas with one error each must fail a pin ----

def _w_hat_sign_flip(xi, a=A):
    num = a + np.exp(-a / 2.0) * (-a * np.cos(np.pi * xi) - 2.0 * np.pi * xi * np.sin(np.pi * xi))
    return 2.0 * num / (a * a + 4.0 * np.pi ** 2 * xi * xi)


def _psi_hat_dropped_term(eta, a=A):
    num = np.exp(a / 2.0) * (a * np.cos(np.pi * eta) + 2.0 * np.pi * eta * np.sin(np.pi * eta))
    return 2.0 * num / (a * a + 4.0 * np.pi ** 2 * eta * eta)


def test_planted_mistakes_are_caught():
    re, _ = quad_transform(1.7, A, -1.0)
    assert abs(_w_hat_sign_flip(1.7) - re) > 1e-3
    re, _ = quad_transform(0.4, A, +1.0)
    assert abs(_psi_hat_dropped_term(0.4) - re) > 1e-3
    # a transposed operand in the diagonal (w_hat(lam - l) in place of w_hat(l - lam)) is
    # invisible for an even w_hat, but an index shift by one grid point is not:
    d = np.array([0.3])
    j = np.arange(-2, 4)
    good = np.sum(ow.psi_hat(d - j) * ow.w_hat(j - d))
    shifted = np.sum(ow.psi_hat(d - j) * ow.w_hat(j + 1 - d))
    assert abs(good - shifted) > 0.1
