"""Writes the stored oracle values of tests/golden/ (run from the repository
root: ``python tests/golden/make_golden.py``).  Calls only ``oracle/``.

The paper prints no worked example with numbers, so these files are the
oracle's own FP64 values on small fixed inputs, kept so that any later change
to the oracle's arithmetic shows up as a test failure
(``tests/test_golden.py``).  The independent pins of the oracle are in
``tests/test_oracle_pins.py``.
"""

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

M = 64
CROP = 256
CROP_WORKLOAD = "stripmap_4096"
CROP_FILE = "stripmap_4096_crop256.npy"


def crop_box(Mimg: int, side: int = CROP):
    """The centre crop: pixels j in [M/2 - side/2, M/2 + side/2) on both axes, as (jx0, jy0, nx, ny)."""
    j0 = Mimg // 2 - side // 2
    return (j0, j0, side, side)


def weight_points():
    """Offsets on the image grid that cover the regimes of G: on a grid point,
    halfway, near the truncation breakpoints, and within q of both grid edges."""
    d = np.array([0.0, 0.1, 0.25, 0.4, 0.5, 0.6, 0.75, 0.9, 0.999])
    centre = np.concatenate([d, -d[1:]]) + 3.0
    edges = np.array([-M / 2, -M / 2 + 0.3, -M / 2 + 1.7, -M / 2 + 2.9, M / 2 - 3.1, M / 2 - 1.5, M / 2 - 0.2])
    return np.concatenate([centre, edges])


def tiny_inputs():
    """Twelve samples and eight pixels on an 8 x 8 image, fixed by formula."""
    n = np.arange(12)
    lam_x = -3.7 + 0.61 * n
    lam_y = 2.9 - 0.53 * n
    y = np.cos(0.7 * n) + 1j * np.sin(1.3 * n + 0.2)
    jx = np.array([0, 1, 3, 4, 4, 5, 7, 2])
    jy = np.array([0, 6, 2, 4, 3, 7, 1, 5])
    return lam_x, lam_y, y, jx, jy


def write_crop():
    """The 256 x 256 centre crop of the weighted adjoint (Eq. (fstraight), alpha_n = D_n,
    tau = 0.97) of the 16,714,266-sample, 4096 x 4096 stripmap workload, by the direct FP64
    sum: 65,536 pixels x 16.7M terms (about 85 minutes on 8 cores)."""
    from synth import make_workload
    wl = make_workload(CROP_WORKLOAD)
    D = oracle.tffr_weights(wl.lam_x, wl.M)
    img = oracle.adjoint_image(wl.lam_x, wl.lam_y, wl.values, D, wl.M, wl.M, crop=crop_box(wl.M))
    np.save(os.path.join(HERE, CROP_FILE), img.astype(np.complex128))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--crop", action="store_true", help="also write the stripmap_4096 centre crop (slow)")
    args = ap.parse_args()
    lam = weight_points()
    G = oracle.diag_psi_w(lam, M)
    D97 = oracle.tffr_weights(lam, M, tau=0.97)
    D102 = oracle.tffr_weights(lam, M, tau=1.02)
    with open(os.path.join(HERE, "weights_M64.txt"), "w") as f:
        f.write("# tFFR weights on a 64-point image grid, a = 0.01, q = 3 (Sec. IV parameters):\n")
        f.write("# G = diag(Psi W) by the closed forms of Eq. (Psi), D = R_tau(1 / G) (Sec. III.B),\n")
        f.write("# written by tests/golden/make_golden.py from oracle/.\n")
        f.write("# lam_x  G  D(tau=0.97)  D(tau=1.02)\n")
        for row in zip(lam, G, D97, D102):
            f.write("%.17g %.17g %.17g %.17g\n" % row)
    lam_x, lam_y, y, jx, jy = tiny_inputs()
    D = oracle.tffr_weights(lam_x, 8)
    f_px = oracle.adjoint_pixels(lam_x, lam_y, y, D, 8, 8, jx, jy)
    with open(os.path.join(HERE, "adjoint_tiny.txt"), "w") as f:
        f.write("# Weighted adjoint of Eq. (fstraight), alpha_n = D_n (tau = 0.97), on an 8 x 8 image,\n")
        f.write("# at the pixels below, for the twelve samples of tiny_inputs() in make_golden.py;\n")
        f.write("# written by tests/golden/make_golden.py from oracle/.\n")
        f.write("# jx  jy  re  im\n")
        for row in zip(jx, jy, f_px.real, f_px.imag):
            f.write("%d %d %.17g %.17g\n" % row)
    if args.crop:
        write_crop()


if __name__ == "__main__":
    main()
