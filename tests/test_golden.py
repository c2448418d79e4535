"""The oracle against its stored values in tests/golden/ (written by
tests/golden/make_golden.py, which calls only oracle/): any change to the
oracle's arithmetic shows up here.  CPU only."""

import importlib.util
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_weights_match_the_stored_values():
    lam, G, D97, D102 = np.loadtxt(os.path.join(GOLDEN, "weights_M64.txt"), unpack=True)
    M = _maker().M
    np.testing.assert_allclose(oracle.diag_psi_w(lam, M), G, rtol=1e-13, atol=0)
    np.testing.assert_allclose(oracle.tffr_weights(lam, M, tau=0.97), D97, rtol=1e-13, atol=0)
    np.testing.assert_allclose(oracle.tffr_weights(lam, M, tau=1.02), D102, rtol=1e-13, atol=0)
    assert np.count_nonzero(D102 == 0) > 0 and np.count_nonzero(D97 == 0) == 0   # both sides of tau


def test_tiny_adjoint_matches_the_stored_values():
    jx, jy, re, im = np.loadtxt(os.path.join(GOLDEN, "adjoint_tiny.txt"), unpack=True)
    lam_x, lam_y, y, _, _ = _maker().tiny_inputs()
    D = oracle.tffr_weights(lam_x, 8)
    got = oracle.adjoint_pixels(lam_x, lam_y, y, D, 8, 8, jx.astype(np.int64), jy.astype(np.int64))
    np.testing.assert_allclose(got, re + 1j * im, rtol=1e-12, atol=1e-12)


def test_stored_stripmap_4096_crop_is_the_oracle_direct_sum():
    """The stored 256 x 256 centre crop of the 16.7M-sample workload (the reference of the
    GPU crop test and of the bench's accuracy) against the direct FP64 sum recomputed here
    at its corners, edge midpoints and centre."""
    mg = _maker()
    crop = np.load(os.path.join(GOLDEN, mg.CROP_FILE))
    assert crop.shape == (mg.CROP, mg.CROP) and crop.dtype == np.complex128
    from synth import make_workload
    wl = make_workload(mg.CROP_WORKLOAD)
    jx0, jy0, nx, ny = mg.crop_box(wl.M)
    ix = np.array([0, nx - 1, 0, nx - 1, nx // 2, 0, nx - 1, nx // 2, nx // 2])
    iy = np.array([0, 0, ny - 1, ny - 1, 0, ny // 2, ny // 2, ny - 1, ny // 2])
    D = oracle.tffr_weights(wl.lam_x, wl.M)
    got = oracle.adjoint_pixels(wl.lam_x, wl.lam_y, wl.values, D, wl.M, wl.M, jx0 + ix, jy0 + iy)
    np.testing.assert_allclose(got, crop[iy, ix], rtol=1e-12, atol=1e-9 * np.abs(crop).max())
