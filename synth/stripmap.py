"""Synthetic stripmap-SAR Fourier data after range-migration (Stolt) mapping.

Geometry (Section II.A, Fig. 2): a platform on a straight azimuth track sends
a linear FM band; after the azimuth FFT and matched filter each sample sits at
spatial wavenumber (k_x, k_y) = (sqrt(4k^2 - k_u^2), k_u).  Range (x) is
non-uniform, azimuth (y) is uniform: every pulse row shares one k_y.

Parameters of the synthetic radar: carrier fc = 10 GHz, bandwidth B = 300 MHz,
azimuth spacing lambda_c / 4.  The wavenumber bounding box is mapped affinely
onto grid units (cycles per image extent) so that it fills ``fill`` = 0.9 of
the M x M image's Fourier grid on each axis, centred on zero.  Pairs with
4k^2 <= k_u^2 (evanescent) are dropped.

Scene model: K point targets with complex N(0,1) reflectivity at seeded
uniform positions in [-0.4, 0.4]^2 (image units, the image spans [-1/2, 1/2)),
plus speckle (a 64 x 64 lattice of weak scatterers with circular-Gaussian
reflectivity CN(0, sigma^2)), plus additive circular white noise at a given
SNR per sample.  A target at x_i contributes exp(-2 pi i lambda_n . x_i) to
sample n: the measurement model, written out directly.

Everything is FP64 with numpy; the sample values are rounded to the requested
complex dtype at the end.  Seeds: ``numpy.random.SeedSequence(191010908 + idx)``.
"""

from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

C0 = 299_792_458.0

_SEED_BASE = 191010908


@dataclass
class StripmapWorkload:
    name: str
    M: int                     # image side (square M x M image)
    lam_x: np.ndarray          # float64 [N], range frequency, grid units
    lam_y: np.ndarray          # float64 [N], azimuth frequency, grid units
    values: np.ndarray         # complex [N], sample values, [pulse][freq] order
    row_ptr: np.ndarray        # int64 [P+1], pulse-row boundaries in sample order
    n_pulses: int
    n_freq: int
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.lam_x.shape[0])


def stolt_points(n_pulses: int, n_freq: int, M: int, fc: float = 10e9,
                 bw: float = 300e6, fill: float = 0.9):
    """Stolt-mapped sample coordinates in grid units, [pulse][freq] order.

    Returns (lam_x, lam_y, row_ptr).  Rows are pulses with at least one
    propagating sample; lam_y is bit-identical within a row.
    """
    lam_c = C0 / fc
    du = lam_c / 4.0
    f = fc - bw / 2.0 + np.arange(n_freq, dtype=np.float64) * (bw / n_freq)
    k = 2.0 * np.pi * f / C0
    ku = 2.0 * np.pi * (np.arange(n_pulses, dtype=np.float64) - (n_pulses - 1) / 2.0) / (n_pulses * du)
    k2 = 4.0 * k[None, :] ** 2 - ku[:, None] ** 2
    keep = k2 > 0.0
    kx = np.sqrt(k2[keep])
    ky = np.broadcast_to(ku[:, None], k2.shape)[keep]
    counts = keep.sum(axis=1)
    row_ptr = np.concatenate([[0], np.cumsum(counts[counts > 0])]).astype(np.int64)

    def to_grid(v):
        lo, hi = v.min(), v.max()
        mid = 0.5 * (lo + hi)
        span = hi - lo if hi > lo else 1.0
        return (v - mid) * (fill * M / span)

    lam_x = np.ascontiguousarray(to_grid(kx))
    lam_y = np.ascontiguousarray(to_grid(ky))
    return lam_x, lam_y, row_ptr


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _chunks(n: int, size: int):
    return [(s, min(n, s + size)) for s in range(0, n, size)]


def _plane_waves(lam_x, lam_y, pos, amp, out):
    """out += sum_i amp_i * exp(-2 pi i (lam_x x_i + lam_y y_i)), FP64."""
    def work(rng):
        s, e = rng
        lx, ly = lam_x[s:e], lam_y[s:e]
        acc = np.zeros(e - s, dtype=np.complex128)
        for (xi, yi), ai in zip(pos, amp):
            th = lx * xi + ly * yi
            th = th - np.floor(th)
            acc += ai * (np.cos(2 * np.pi * th) - 1j * np.sin(2 * np.pi * th))
        out[s:e] += acc
    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(work, _chunks(lam_x.shape[0], 1 << 18)))


def _speckle_lattice(lam_x, lam_y, row_ptr, amp, extent, out):
    """Speckle from a K x K lattice of scatterers with reflectivity ``amp[a, b]``.

    Scatterer (a, b) sits at (X_a, Y_b) on a uniform lattice over
    [-extent, extent]^2.  Because every pulse row shares lam_y, the sum splits:
    T[p, a] = sum_b amp[a, b] exp(-2 pi i lam_y,p Y_b), then per sample a
    polynomial in z = exp(-2 pi i lam_x dX) evaluated by Horner's rule.
    """
    K = amp.shape[0]
    dX = 2.0 * extent / K
    X0 = -extent + 0.5 * dX
    Y = X0 + dX * np.arange(K)
    P = row_ptr.shape[0] - 1
    ly_rows = lam_y[row_ptr[:-1]]
    ph = np.outer(ly_rows, Y)
    ph -= np.floor(ph)
    Ey = np.exp(-2j * np.pi * ph)                 # [P, K]
    T = Ey @ amp.T                                # [P, K_a]
    row_of = np.repeat(np.arange(P), np.diff(row_ptr))

    def work(rng):
        s, e = rng
        lx = lam_x[s:e]
        th = lx * dX
        th -= np.floor(th)
        z = np.exp(-2j * np.pi * th)
        th0 = lx * X0
        th0 -= np.floor(th0)
        r = row_of[s:e]
        acc = T[r, K - 1].copy()
        for a in range(K - 2, -1, -1):
            acc *= z
            acc += T[r, a]
        out[s:e] += acc * np.exp(-2j * np.pi * th0)
    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(work, _chunks(lam_x.shape[0], 1 << 18)))


def scene_samples(lam_x, lam_y, row_ptr, *, n_targets: int, speckle_sigma: float,
                  snr_db, seed: int, target_extent: float = 0.4,
                  speckle_lattice: int = 64):
    """FP64 complex sample values of the synthetic scene (see module docstring)."""
    ss = np.random.SeedSequence(seed)
    s_pos, s_amp, s_spk, s_noise = ss.spawn(4)
    g_pos = np.random.default_rng(s_pos)
    g_amp = np.random.default_rng(s_amp)
    pos = g_pos.uniform(-target_extent, target_extent, size=(n_targets, 2))
    amp = (g_amp.standard_normal(n_targets) + 1j * g_amp.standard_normal(n_targets)) / np.sqrt(2.0)
    out = np.zeros(lam_x.shape[0], dtype=np.complex128)
    _plane_waves(lam_x, lam_y, pos, amp, out)
    if speckle_sigma > 0.0:
        g = np.random.default_rng(s_spk)
        K = speckle_lattice
        spk = speckle_sigma * (g.standard_normal((K, K)) + 1j * g.standard_normal((K, K))) / np.sqrt(2.0)
        _speckle_lattice(lam_x, lam_y, row_ptr, spk, 0.45, out)
    if snr_db is not None:
        g = np.random.default_rng(s_noise)
        p_sig = float(np.mean(np.abs(out) ** 2))
        sig_n = np.sqrt(p_sig / (10.0 ** (snr_db / 10.0)))
        n = out.shape[0]
        out += sig_n * (g.standard_normal(n) + 1j * g.standard_normal(n)) / np.sqrt(2.0)
    return out, {"targets": pos, "amplitudes": amp}


# name -> (n_pulses, n_freq, M, n_targets, speckle sigma, snr dB, value dtype)
WORKLOADS = {
    "tiny_64": (64, 64, 64, 5, 0.0, None, np.complex128),
    "stripmap_1024": (512, 1024, 1024, 50, 0.1, 20.0, np.complex64),
    "stripmap_4096": (4096, 4096, 4096, 50, 0.1, 20.0, np.complex64),
    "stripmap_2048": (1024, 2048, 2048, 50, 0.1, 20.0, np.complex64),
}
_WORKLOAD_INDEX = {"tiny_64": 0, "stripmap_1024": 1, "stripmap_4096": 2, "stripmap_2048": 3}


def make_workload(name: str, *, values: bool = True) -> StripmapWorkload:
    """Build one of the named stripmap workloads (coordinates + seeded scene)."""
    n_p, n_f, M, n_t, spk, snr, dt = WORKLOADS[name]
    lam_x, lam_y, row_ptr = stolt_points(n_p, n_f, M)
    meta = {"n_targets": n_t, "speckle_sigma": spk, "snr_db": snr}
    if values:
        v, extra = scene_samples(lam_x, lam_y, row_ptr, n_targets=n_t, speckle_sigma=spk,
                                 snr_db=snr, seed=_SEED_BASE + _WORKLOAD_INDEX[name])
        meta.update(extra)
        v = v.astype(dt)
    else:
        v = np.zeros(0, dtype=dt)
    return StripmapWorkload(name, M, lam_x, lam_y, v, row_ptr, n_p, n_f, meta)


def random_points(N: int, M: int, seed: int, extent: float = 0.45, dtype=np.complex64):
    """Unstructured points: uniform lam in [-extent M, extent M)^2, CN(0,1) values."""
    g = np.random.default_rng(np.random.SeedSequence(seed))
    lam_x = g.uniform(-extent * M, extent * M, N)
    lam_y = g.uniform(-extent * M, extent * M, N)
    v = ((g.standard_normal(N) + 1j * g.standard_normal(N)) / np.sqrt(2.0)).astype(dtype)
    return lam_x, lam_y, v


def patch_batch(n_patches: int = 64, seed: int = 191010908 + 5, sides=(256, 512, 1024),
                pulses=(128, 1024), freqs=(256, 2048)):
    """Uneven sub-aperture patches: per patch n_pulses ~ U{pulses}, n_freq ~ U{freqs}
    and an image side drawn from `sides`, Stolt coordinates and CN(0,1) samples.
    Returns a list of (M, lam_x, lam_y, values)."""
    g = np.random.default_rng(np.random.SeedSequence(seed))
    out = []
    for _ in range(n_patches):
        P = int(g.integers(pulses[0], pulses[1] + 1))
        F = int(g.integers(freqs[0], freqs[1] + 1))
        M = int(sides[int(g.integers(0, len(sides)))])
        lx, ly, _ = stolt_points(P, F, M)
        v = ((g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])) / np.sqrt(2.0)).astype(np.complex64)
        out.append((M, lx, ly, v))
    return out


def edge_rows(M: int, rows: int, per: int, seed: int):
    """Pulse rows whose samples all lie within 4 image cells of the left or right edge of an
    M-point grid (rows alternate sides; lam_x sorted along a row), with white complex64 samples:
    the truncated sum G of every sample differs from its interior form there."""
    g = np.random.default_rng(seed)
    lam_y = np.linspace(-M / 2 + 7.3, M / 2 - 8.3, rows)
    lx = np.concatenate([np.sort(g.uniform(0.0, 3.99, per)) + (-M / 2 if r % 2 == 0 else M / 2 - 4.0)
                         for r in range(rows)])
    ly = np.repeat(lam_y, per)
    v = (g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])).astype(np.complex64)
    return lx, ly, v
