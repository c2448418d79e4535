"""Structure of the synthetic stripmap inputs (the generator, not the method)."""

import numpy as np
import pytest

from synth import stolt_points, make_workload, C0


@pytest.mark.parametrize("P,F,M,N", [(64, 64, 64, 4096), (512, 1024, 1024, 522320),
                                     (1024, 2048, 2048, 2089290)])
def test_sample_counts_and_rows(P, F, M, N):
    lx, ly, rp = stolt_points(P, F, M)
    assert lx.shape[0] == N and rp[-1] == N
    assert np.all(np.abs(lx) <= 0.45 * M + 1e-9) and np.all(np.abs(ly) <= 0.45 * M + 1e-9)
    for p in range(rp.shape[0] - 1):
        s, e = rp[p], rp[p + 1]
        assert np.all(ly[s:e] == ly[s])            # azimuth is uniform: one k_y per pulse
        assert np.all(np.diff(lx[s:e]) > 0)        # k_x grows with k along a pulse


def test_stolt_relation_before_the_affine_map():
    """k_x^2 + k_u^2 = 4 k^2 for each kept pair (the Stolt mapping of Section II.A)."""
    fc, bw, P, F = 10e9, 300e6, 64, 64
    f = fc - bw / 2 + np.arange(F) * bw / F
    k = 2 * np.pi * f / C0
    du = C0 / fc / 4
    ku = 2 * np.pi * (np.arange(P) - (P - 1) / 2) / (P * du)
    lx, ly, rp = stolt_points(P, F, 64)
    kx = np.sqrt(4 * k[None, :] ** 2 - ku[:, None] ** 2)
    # the affine map is monotone per axis: recover it from the extremes and invert
    sx = (kx.max() - kx.min()) / (0.9 * 64)
    kx_rec = lx * sx + 0.5 * (kx.max() + kx.min())
    assert np.allclose(kx_rec.reshape(P, F) ** 2 + ku[:, None] ** 2, 4 * k[None, :] ** 2, rtol=1e-12)


def test_workload_is_deterministic():
    a = make_workload("tiny_64")
    b = make_workload("tiny_64")
    assert np.array_equal(a.values, b.values) and a.values.dtype == np.complex128
    assert a.N == 4096


def test_edge_rows_lie_in_the_edge_band():
    """Every sample of edge_rows is within 4 image cells of the left or right grid edge, rows
    alternate sides, and each row shares one lam_y (bit-equal) with lam_x sorted along it."""
    import numpy as np
    from synth import edge_rows
    M, rows, per = 256, 10, 50
    lx, ly, v = edge_rows(M, rows, per, seed=3)
    assert lx.shape == ly.shape == v.shape == (rows * per,)
    j0 = np.floor(lx)
    assert np.all((j0 - 4 < -(M // 2)) | (j0 + 4 >= M - M // 2))
    assert np.all((lx >= -M / 2) & (lx < M / 2))
    for r in range(rows):
        x, y = lx[r * per:(r + 1) * per], ly[r * per:(r + 1) * per]
        assert np.all(y == y[0]) and np.all(np.diff(x) >= 0)
        assert (x[0] < 0) == (r % 2 == 0)
