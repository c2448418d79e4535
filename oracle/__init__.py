"""FP64 CPU oracle for the tFFR adjoint and its forward twin.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path
(``paper_1910_10908_gb300``) never imports, links or calls anything here, and
this package shares no code with it.

What it computes (each function cites the passage it follows):

* ``weights.tffr_weights`` -- D_n = R_tau(diag(Psi W)^+) per sample, range axis
  (Algorithm 1; Eqs. (Psi), (bound); R_tau of Section III.B; a = 0.01,
  tau = 0.97 of Section IV).  Closed forms of the window transforms.
* ``adjoint_pixels`` / ``adjoint_image`` -- the weighted inverse-Fourier sum of
  Eq. (fstraight) with alpha_n = D_n, evaluated term by term in FP64 (C, OpenMP).
* ``forward_samples`` -- its adjoint, y_n = D_n sum_j f_j exp(-2 pi i lam_n . x_j).

Pins (tests/test_oracle_pins.py): quadrature of the window transforms, the
partition-of-unity identity of the untruncated Psi W diagonal, the sinc^2 limit
a -> 0, dense Psi and W built by quadrature from their definitions, the
uniform-grid case against numpy's inverse FFT, Parseval, the point-scatterer
closed form (Dirichlet kernels), and adjointness of the two sums.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import weights  # noqa: F401
from .weights import tffr_weights, diag_psi_w, w_hat, psi_hat  # noqa: F401

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        from .build import build
        path = build()
        lib = ctypes.CDLL(path)
        c_i64, c_int = ctypes.c_int64, ctypes.c_int
        p = ctypes.c_void_p
        lib.oracle_adjoint_pixels.argtypes = [c_i64, p, p, p, p, c_int, c_int, c_i64, p, p, p, c_int]
        lib.oracle_adjoint_pixels.restype = None
        lib.oracle_forward_samples.argtypes = [c_i64, p, p, p, p, c_int, c_int, c_i64, p, p, c_int]
        lib.oracle_forward_samples.restype = None
        lib.oracle_threads.restype = c_int
        _LIB = lib
    return _LIB


def threads() -> int:
    return int(_lib().oracle_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def adjoint_pixels(lam_x, lam_y, y, D, Mx: int, My: int, jx, jy, nthreads: int = 0):
    """Eq. (fstraight) at pixels (jx[k], jy[k]); D=None means alpha_n = 1."""
    lam_x, lam_y, y = _f64(lam_x), _f64(lam_y), _c128(y)
    Dv = None if D is None else _f64(D)
    jx = np.ascontiguousarray(jx, dtype=np.int32)
    jy = np.ascontiguousarray(jy, dtype=np.int32)
    out = np.zeros(jx.shape[0], dtype=np.complex128)
    _lib().oracle_adjoint_pixels(lam_x.shape[0], _ptr(lam_x), _ptr(lam_y), _ptr(y), _ptr(Dv),
                                 int(Mx), int(My), jx.shape[0], _ptr(jx), _ptr(jy), _ptr(out),
                                 int(nthreads))
    return out


def adjoint_image(lam_x, lam_y, y, D, Mx: int, My: int, crop=None, nthreads: int = 0):
    """Whole image [My, Mx] (or the crop (jx0, jy0, nx, ny)) of Eq. (fstraight)."""
    if crop is None:
        crop = (0, 0, Mx, My)
    jx0, jy0, nx, ny = crop
    gy, gx = np.meshgrid(np.arange(jy0, jy0 + ny), np.arange(jx0, jx0 + nx), indexing="ij")
    out = adjoint_pixels(lam_x, lam_y, y, D, Mx, My, gx.ravel(), gy.ravel(), nthreads)
    return out.reshape(ny, nx)


def forward_samples(lam_x, lam_y, img, D, idx=None, nthreads: int = 0):
    """y_n = D_n sum_j f_j exp(-2 pi i lam_n . x_j) at samples ``idx`` (all if None)."""
    lam_x, lam_y = _f64(lam_x), _f64(lam_y)
    img = _c128(img)
    My, Mx = img.shape
    Dv = None if D is None else _f64(D)
    if idx is None:
        nidx, ip = lam_x.shape[0], None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        nidx, ip = idx.shape[0], idx
    out = np.zeros(nidx, dtype=np.complex128)
    _lib().oracle_forward_samples(lam_x.shape[0], _ptr(lam_x), _ptr(lam_y), _ptr(img), _ptr(Dv),
                                  int(Mx), int(My), nidx, _ptr(ip), _ptr(out), int(nthreads))
    return out
