"""tFFR frame weights D_n in FP64 (oracle; test infrastructure only).

Steps, in the order of Algorithm 1 (per azimuth slice, on the range axis):

1. The window w(x) = exp(-a |x - 1/2|), a = 0.01 (Section IV, Baselines), taken
   on the centred domain t = x - 1/2 in [-1/2, 1/2] so that its transforms are
   real and even.
2. W = [w_hat(l_m - lam_p)], the window transform (Eq. (bound) and Algorithm 1):
       w_hat(xi) = int_{-1/2}^{1/2} exp(-a|t|) exp(-2 pi i xi t) dt
                 = 2 [a + e^{-a/2} (-a cos(pi xi) + 2 pi xi sin(pi xi))] / (a^2 + 4 pi^2 xi^2)
3. Psi = [<exp(2 pi i lam_p t), exp(2 pi i l_m t) / w(t)>] (Eq. (Psi)), "found
   analytically" (Section III.C):
       Psi_pm = psi(lam_p - l_m),
       psi(eta) = int_{-1/2}^{1/2} exp(+a|t|) exp(2 pi i eta t) dt
                = 2 [-a + e^{a/2} (a cos(pi eta) + 2 pi eta sin(pi eta))] / (a^2 + 4 pi^2 eta^2)
4. Only the diagonal of the sample-by-sample product Psi W is kept (the
   complexity paragraph of Section III.B), with W banded by the truncation
   |lam_p - l_m| < q of Eq. (Anu):
       G_p = sum_{m : |lam_p - l_m| < q, l_m on the grid} psi(lam_p - l_m) w_hat(l_m - lam_p)
5. D = R_tau(diag(G)^+): D_p = 1 / G_p (0 where G_p = 0), then the threshold
   R_tau(x) = x if x >= tau else 0 (Section III.B), tau = 0.97 by default.

The grid l_m is the image's integer Fourier grid, m in [-M/2, M/2).
"""

from __future__ import annotations

import numpy as np

A_DEFAULT = 0.01
Q_DEFAULT = 3.0
TAU_DEFAULT = 0.97


def w_hat(xi, a: float = A_DEFAULT):
    """Fourier transform of the window exp(-a|t|) on [-1/2, 1/2] (closed form)."""
    xi = np.asarray(xi, dtype=np.float64)
    num = a + np.exp(-a / 2.0) * (-a * np.cos(np.pi * xi) + 2.0 * np.pi * xi * np.sin(np.pi * xi))
    return 2.0 * num / (a * a + 4.0 * np.pi ** 2 * xi * xi)


def psi_hat(eta, a: float = A_DEFAULT):
    """Fourier transform of the reciprocal window exp(+a|t|) on [-1/2, 1/2] (closed form)."""
    eta = np.asarray(eta, dtype=np.float64)
    num = -a + np.exp(a / 2.0) * (a * np.cos(np.pi * eta) + 2.0 * np.pi * eta * np.sin(np.pi * eta))
    return 2.0 * num / (a * a + 4.0 * np.pi ** 2 * eta * eta)


def diag_psi_w(lam, M: int, q: float = Q_DEFAULT, a: float = A_DEFAULT):
    """G_p = diagonal of Psi W for samples at frequencies ``lam`` (grid units)."""
    lam = np.asarray(lam, dtype=np.float64)
    G = np.zeros_like(lam)
    base = np.floor(lam)
    span = int(np.ceil(q)) + 1
    for off in range(-span, span + 1):
        l_m = base + off
        on_grid = (l_m >= -(M // 2)) & (l_m < M - M // 2)
        near = np.abs(lam - l_m) < q
        use = on_grid & near
        term = psi_hat(lam - l_m, a) * w_hat(l_m - lam, a)
        G += np.where(use, term, 0.0)
    return G


def threshold(x, tau: float):
    """R_tau(x) = x if x >= tau, else 0."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(x >= tau, x, 0.0)


def pinv_diag(G):
    G = np.asarray(G, dtype=np.float64)
    out = np.zeros_like(G)
    nz = G != 0.0
    out[nz] = 1.0 / G[nz]
    return out


def tffr_weights(lam_x, Mx: int, *, tau: float = TAU_DEFAULT, q: float = Q_DEFAULT,
                 a: float = A_DEFAULT, lam_y=None, My: int | None = None,
                 separable: bool = False):
    """tFFR weights D_n (range axis only by default; optional separable product).

    Range-only (default): D_n = R_tau(1 / G(lam_x[n])).
    Separable variant:    D_n = R_tau(1 / (G(lam_x[n]) G(lam_y[n]))).
    """
    Gx = diag_psi_w(lam_x, Mx, q, a)
    if separable:
        Gy = diag_psi_w(lam_y, My, q, a)
        return threshold(pinv_diag(Gx * Gy), tau)
    return threshold(pinv_diag(Gx), tau)
