"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerance: relative L2 error <= 1e-5 for the FP32 path (complex64 or complex128
sample storage), measured against the direct FP64 sum.  The spreading kernel
alone contributes ~5e-6 at width 6 on stripmap geometry (~1e-5 on uniform
random points, which the tests therefore run at width 8, ~1e-7).
Reduced-precision sample storage has its own bound from its rounding unit.
"""

import os

import numpy as np
import pytest
import torch

import oracle
from synth import edge_rows, make_workload, random_points, scene_samples, stolt_points

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def d_err(D, Dref):
    """Largest relative difference of two weight vectors (FP32 storage: a few 6e-8 ulps)."""
    return float(np.max(np.abs(D - Dref) / np.maximum(1.0, np.abs(Dref))))


def gpu_adjoint(lx, ly, vals, Mx, My=None, values="c64", layout="auto", width=6, wkw=None, order="auto"):
    from paper_1910_10908_gb300 import Plan
    My = Mx if My is None else My
    with Plan(Mx, My, values=values, layout=layout, width=width, order=order) as plan:
        plan.set_points(dev(lx), dev(ly))
        D = torch.empty(lx.shape[0], dtype=torch.float32, device="cuda")
        kept = plan.weights(D_out=D, **(wkw or {}))
        img = plan.adjoint(vals if isinstance(vals, torch.Tensor) else dev(vals))
        torch.cuda.synchronize()
        info = plan.info()
        return img.cpu().numpy().astype(np.complex128), D.cpu().numpy().astype(np.float64), kept, info


def stolt_scene(P, F, M, seed=11, noise=True):
    lx, ly, rp = stolt_points(P, F, M)
    v, _ = scene_samples(lx, ly, rp, n_targets=50, speckle_sigma=0.1, snr_db=20.0 if noise else None, seed=seed)
    return lx, ly, rp, v


def test_tiny_config_complex128_full_image():
    wl = make_workload("tiny_64")
    img, D, kept, info = gpu_adjoint(wl.lam_x, wl.lam_y, wl.values, wl.M, values="c128")
    Dref = oracle.tffr_weights(wl.lam_x, wl.M)
    assert info["layout"] == 2 and info["n_rows"] == 64
    assert d_err(D, Dref) < 3e-7
    assert kept == np.count_nonzero(Dref)
    ref = oracle.adjoint_image(wl.lam_x, wl.lam_y, wl.values, Dref, wl.M, wl.M)
    assert rel_l2(img, ref) <= TOL


@pytest.mark.parametrize("layout", ["auto", "general"])
def test_stolt_128_ragged_rows_full_image(layout):
    lx, ly, rp, v = stolt_scene(128, 256, 128)
    lens = np.diff(rp)
    assert lens.min() < lens.max()             # evanescent pairs make the outer rows shorter
    img, D, kept, info = gpu_adjoint(lx, ly, v.astype(np.complex64), 128, layout=layout)
    assert info["layout"] == (2 if layout == "auto" else 1)
    Dref = oracle.tffr_weights(lx, 128)
    ref = oracle.adjoint_image(lx, ly, v.astype(np.complex64), Dref, 128, 128)
    assert rel_l2(img, ref) <= TOL


def test_non_square_image():
    lx, ly, rp = stolt_points(64, 200, 128)
    ly = ly * (32 / 128)                       # azimuth band of a 32-row image
    g = np.random.default_rng(4)
    v = (g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])).astype(np.complex64)
    # white sample values put energy at the image edge, where width 6 sits at ~1.1e-5: use width 8
    img, _, _, info = gpu_adjoint(lx, ly, v, 128, 32, width=8)
    assert img.shape == (32, 128) and info["layout"] == 2
    ref = oracle.adjoint_image(lx, ly, v, oracle.tffr_weights(lx, 128), 128, 32)
    assert rel_l2(img, ref) <= TOL


@pytest.mark.parametrize("M,N,extent", [(64, 3000, 0.45), (128, 20000, 0.5), (16, 100, 0.5)])
def test_general_random_points_width8(M, N, extent):
    lx, ly, v = random_points(N, M, seed=M + N, extent=extent)
    img, D, _, info = gpu_adjoint(lx, ly, v, M, width=8)
    assert info["layout"] == 1
    ref = oracle.adjoint_image(lx, ly, v, oracle.tffr_weights(lx, M), M, M)
    assert rel_l2(img, ref) <= TOL


def test_points_on_cell_edges_and_grid_boundary():
    M = 32
    g = np.random.default_rng(9)
    lx = np.concatenate([np.arange(-16, 16, 0.5), [-16.0, 15.999999999, 0.0, -0.25]])
    ly = np.concatenate([np.full(64, 3.5), [-16.0, -16.0, 15.75, 0.0]])
    v = (g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])).astype(np.complex64)
    img, _, _, _ = gpu_adjoint(lx, ly, v, M, width=8, layout="general")
    ref = oracle.adjoint_image(lx, ly, v, oracle.tffr_weights(lx, M), M, M)
    assert rel_l2(img, ref) <= TOL


def test_pulse_rows_through_zero_and_at_special_magnitudes():
    """Pulse rows whose lam_x runs through zero and through magnitudes where the
    bit-pattern split changes form: exact zero, +-1e-9 and +-2^-12 (below the fast
    split's range: deferred), +-2^-11 (its edge), half-integers (cell edges),
    integers (truncation breakpoints: the FP64 decision) and powers of two (where
    the exponent steps), in both pass orders and with the separable weights."""
    M = 64
    special = np.array([0.0, 1e-9, 2.0 ** -12, 2.0 ** -11, 0.25, 0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 7.5, 8.0, 15.0,
                        16.0, 24.0, 31.5])
    base = np.unique(np.concatenate([special, -special, np.linspace(-31.9, 31.9, 97)]))
    g = np.random.default_rng(12)
    rows = 40
    lam_y = np.linspace(-31.3, 30.7, rows)
    lx = np.concatenate([base + (0.0 if r % 2 == 0 else g.uniform(-1e-3, 1e-3)) for r in range(rows)])
    ly = np.repeat(lam_y, base.shape[0])
    v = (g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])).astype(np.complex64)
    for order in ("auto", "fine_rows"):
        for sep in (False, True):
            img, D, kept, info = gpu_adjoint(lx, ly, v, M, width=8, layout="rows", order=order,
                                             wkw=dict(separable=sep, tau=1.0))
            assert info["layout"] == 2 and info["n_rows"] == rows
            Dref = oracle.tffr_weights(lx, M, lam_y=ly, My=M, separable=sep, tau=1.0)
            assert kept == np.count_nonzero(Dref)
            assert d_err(D, Dref) < 3e-7
            ref = oracle.adjoint_image(lx, ly, v, Dref, M, M)
            assert rel_l2(img, ref) <= TOL


def test_rows_whose_every_sample_takes_the_fp64_decision():
    """Every sample of every pulse row is listed for the FP64 decision, so each row's region of the
    list fills to its capacity (one slot per sample): the image and the weights against the oracle."""
    M = 256
    lx, ly, v = edge_rows(M, 40, 120, seed=31)
    img, D, kept, info = gpu_adjoint(lx, ly, v, M, width=8, layout="rows")
    assert info["layout"] == 2 and info["n_rows"] == 40
    Dref = oracle.tffr_weights(lx, M)
    assert kept == np.count_nonzero(Dref)
    assert d_err(D, Dref) < 3e-7
    ref = oracle.adjoint_image(lx, ly, v, Dref, M, M)
    assert rel_l2(img, ref) <= TOL


def test_rows_layout_forced_on_short_rows():
    lx, ly, rp = stolt_points(48, 6, 64)       # 6 samples per pulse row
    g = np.random.default_rng(1)
    v = (g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])).astype(np.complex64)
    img, _, _, info = gpu_adjoint(lx, ly, v, 64, layout="rows", width=8)
    assert info["layout"] == 2 and info["n_rows"] == 48
    ref = oracle.adjoint_image(lx, ly, v, oracle.tffr_weights(lx, 64), 64, 64)
    assert rel_l2(img, ref) <= TOL


def test_stripmap_1024_sampled_pixels():
    wl = make_workload("stripmap_1024")
    img, D, kept, info = gpu_adjoint(wl.lam_x, wl.lam_y, wl.values, wl.M)
    assert info["n_rows"] == 512 and kept == wl.N
    Dref = oracle.tffr_weights(wl.lam_x, wl.M)
    assert d_err(D, Dref) < 3e-7
    g = np.random.default_rng(21)
    jx = np.concatenate([g.integers(0, wl.M, 160), np.repeat(np.arange(504, 520), 16)])
    jy = np.concatenate([g.integers(0, wl.M, 160), np.tile(np.arange(504, 520), 16)])
    ref = oracle.adjoint_pixels(wl.lam_x, wl.lam_y, wl.values, Dref, wl.M, wl.M, jx, jy)
    assert rel_l2(img[jy, jx], ref) <= TOL


def test_stripmap_4096_sampled_pixels_bench_configuration():
    wl = make_workload("stripmap_4096")
    img, D, kept, info = gpu_adjoint(wl.lam_x, wl.lam_y, wl.values, wl.M)
    assert info["layout"] == 2 and info["n_rows"] == 4096 and kept == wl.N
    g = np.random.default_rng(22)
    n = 48
    jx, jy = g.integers(0, wl.M, n), g.integers(0, wl.M, n)
    # the targets sit at pixel-scale positions: include the brightest pixels too
    flat = np.argsort(np.abs(img).ravel())[-16:]
    jy = np.concatenate([jy, flat // wl.M])
    jx = np.concatenate([jx, flat % wl.M])
    idx = g.integers(0, wl.N, 200000)
    assert d_err(D[idx], oracle.tffr_weights(wl.lam_x[idx], wl.M)) < 3e-7
    Dref = oracle.tffr_weights(wl.lam_x, wl.M)
    ref = oracle.adjoint_pixels(wl.lam_x, wl.lam_y, wl.values, Dref, wl.M, wl.M, jx, jy)
    assert rel_l2(img[jy, jx], ref) <= TOL


def test_stripmap_4096_forward_twin_sampled_bench_configuration():
    """The forward twin at the bench size (pulse-row order), at sampled samples: the first
    and last sample of the data, and random ones.  D_n depends on lam_x_n alone (range-only
    weights), so the oracle's D is taken at those samples only."""
    from paper_1910_10908_gb300 import Plan
    wl = make_workload("stripmap_4096")
    g = np.random.default_rng(24)
    f = (g.standard_normal((wl.M, wl.M)) + 1j * g.standard_normal((wl.M, wl.M))).astype(np.complex64)
    with Plan(wl.M) as plan:
        plan.set_points(dev(wl.lam_x), dev(wl.lam_y))
        plan.weights(count=False)
        assert plan.info()["pulse_order"] == 1
        y = plan.forward(dev(f)).cpu().numpy()
    idx = np.concatenate([[0, wl.N - 1], g.integers(0, wl.N, 78)])
    Dn = oracle.tffr_weights(wl.lam_x[idx], wl.M)
    ref = Dn * oracle.forward_samples(wl.lam_x, wl.lam_y, f, None, idx=idx)
    assert rel_l2(y[idx], ref) <= TOL


@pytest.mark.parametrize("apply_weights", [True, False])
def test_forward_twin_vs_oracle(apply_weights):
    from paper_1910_10908_gb300 import Plan
    lx, ly, rp, _ = stolt_scene(128, 256, 128)
    g = np.random.default_rng(3)
    f = (g.standard_normal((128, 128)) + 1j * g.standard_normal((128, 128))).astype(np.complex64)
    with Plan(128) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(tau=1.02)
        y = plan.forward(dev(f), apply_weights=apply_weights).cpu().numpy()
    idx = g.integers(0, lx.shape[0], 400)
    Dref = oracle.tffr_weights(lx, 128, tau=1.02)
    ref = oracle.forward_samples(lx, ly, f, Dref if apply_weights else None, idx=idx)
    assert rel_l2(y[idx], ref) <= TOL


@pytest.mark.parametrize("layout", ["auto", "general"])
def test_adjointness_on_the_gpu(layout):
    from paper_1910_10908_gb300 import Plan
    lx, ly, _, _ = stolt_scene(96, 160, 64)
    g = np.random.default_rng(8)
    y = (g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])).astype(np.complex64)
    f = (g.standard_normal((64, 64)) + 1j * g.standard_normal((64, 64))).astype(np.complex64)
    with Plan(64, layout=layout) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(tau=1.02)
        Ay = plan.adjoint(dev(y)).cpu().numpy().astype(np.complex128)
        Af = plan.forward(dev(f)).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(f.astype(np.complex128), Ay)
    rhs = np.vdot(Af, y.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_empty_and_fully_thresholded():
    from paper_1910_10908_gb300 import Plan
    with Plan(32) as plan:
        e = torch.empty(0, dtype=torch.float64, device="cuda")
        plan.set_points(e, e)
        assert plan.weights() == 0
        img = plan.adjoint(torch.empty(0, dtype=torch.complex64, device="cuda"))
        assert torch.count_nonzero(img).item() == 0
    lx, ly, _, v = stolt_scene(32, 32, 32)
    with Plan(32) as plan:
        plan.set_points(dev(lx), dev(ly))
        assert plan.weights(tau=2.0) == 0
        img = plan.adjoint(dev(v.astype(np.complex64)))
        assert torch.count_nonzero(img).item() == 0


def test_errors_are_reported():
    from paper_1910_10908_gb300 import Plan, TffrError
    lx, ly, _, v = stolt_scene(32, 32, 32)
    with Plan(32) as plan:
        with pytest.raises(TffrError) as e:
            plan.adjoint(dev(v.astype(np.complex64)))
        assert e.value.status == 2
        bad = lx.copy()
        bad[7] = np.nan
        with pytest.raises(TffrError) as e:
            plan.set_points(dev(bad), dev(ly))
        assert e.value.status == 1
        bad[7] = 3e8
        with pytest.raises(TffrError) as e:
            plan.set_points(dev(bad), dev(ly))
        assert e.value.status == 1
        with pytest.raises(TffrError) as e:
            plan.weights()
        assert e.value.status == 2
        plan.set_points(dev(lx), dev(ly))        # the plan recovers
        plan.weights()
        plan.adjoint(dev(v.astype(np.complex64)))
        with pytest.raises(TffrError) as e:
            plan.weights(q=-1.0)
        assert e.value.status == 1


@pytest.mark.parametrize("kw", [dict(), dict(tau=1.02), dict(separable=True, tau=1.0), dict(mode="unit")])
def test_reconstruct_equals_the_three_calls(kw):
    """tffr_reconstruct runs the same kernels as set_points + weights + adjoint: the same image up
    to the order of the shared-memory additions (atomics: 1e-6 relative), and the oracle's; its
    errors are those of the three calls."""
    from paper_1910_10908_gb300 import Plan, TffrError
    lx, ly, _, v = stolt_scene(96, 160, 128)
    vals = dev(v.astype(np.complex64))
    with Plan(128) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(count=False, **kw)
        three = plan.adjoint(vals).clone()
        one = plan.reconstruct(dev(lx), dev(ly), vals, **kw)
        torch.cuda.synchronize()
        assert float(torch.linalg.vector_norm(one - three) / torch.linalg.vector_norm(three)) <= 1e-6
        bad = lx.copy()
        bad[3] = np.inf
        with pytest.raises(TffrError) as e:
            plan.reconstruct(dev(bad), dev(ly), vals, **kw)
        assert e.value.status == 1
        with pytest.raises(TffrError) as e:
            plan.reconstruct(dev(lx), dev(ly), vals, q=-1.0)
        assert e.value.status == 1
        with pytest.raises(TffrError) as e:                # the failed calls left no weights
            plan.adjoint(vals)
        assert e.value.status == 2
    if kw.get("mode") == "unit":
        Dref = np.ones_like(lx)
    else:
        okw = {k: kw[k] for k in ("tau", "a", "q") if k in kw}
        Dref = oracle.tffr_weights(lx, 128, lam_y=ly, My=128, separable=kw.get("separable", False), **okw)
    ref = oracle.adjoint_image(lx, ly, v.astype(np.complex64), Dref, 128, 128)
    assert rel_l2(one.cpu().numpy().astype(np.complex128), ref) <= TOL


@pytest.mark.parametrize("kw", [dict(mode="unit"), dict(tau=1.02), dict(tau=1.05), dict(separable=True, tau=1.0),
                                dict(a=0.5, q=2.5, tau=0.97)])
def test_weight_modes_vs_oracle(kw):
    lx, ly, _, v = stolt_scene(64, 96, 64)
    img, D, kept, _ = gpu_adjoint(lx, ly, v.astype(np.complex64), 64, wkw=kw)
    if kw.get("mode") == "unit":
        Dref = np.ones_like(lx)
    else:
        okw = {k: kw[k] for k in ("tau", "a", "q") if k in kw}
        Dref = oracle.tffr_weights(lx, 64, lam_y=ly, My=64, separable=kw.get("separable", False), **okw)
    assert kept == np.count_nonzero(Dref)
    assert d_err(D, Dref) < 3e-7
    if kept:
        ref = oracle.adjoint_image(lx, ly, v.astype(np.complex64), Dref, 64, 64)
        assert rel_l2(img, ref) <= TOL


def test_user_weights():
    lx, ly, _, v = stolt_scene(64, 96, 64)
    g = np.random.default_rng(5)
    Du = g.uniform(0.5, 1.5, lx.shape[0]).astype(np.float32)
    Du[::7] = 0.0
    img, D, kept, _ = gpu_adjoint(lx, ly, v.astype(np.complex64), 64,
                                  wkw=dict(mode="user", user_D=dev(Du)))
    assert np.array_equal(D.astype(np.float32), Du) and kept == np.count_nonzero(Du)
    ref = oracle.adjoint_image(lx, ly, v.astype(np.complex64), Du.astype(np.float64), 64, 64)
    assert rel_l2(img, ref) <= TOL


@pytest.mark.parametrize("values,bound", [("f16", 1e-3), ("bf16", 8e-3)])
def test_reduced_precision_sample_storage(values, bound):
    lx, ly, _, v = stolt_scene(128, 256, 128)
    if values == "f16":
        t = dev(v.astype(np.complex64)).to(torch.complex32)
        stored = t.to(torch.complex64).cpu().numpy()
    else:
        t = torch.view_as_real(dev(v.astype(np.complex64))).to(torch.bfloat16).contiguous()
        stored = torch.view_as_complex(t.float().contiguous()).cpu().numpy()
    img, _, _, _ = gpu_adjoint(lx, ly, t, 128, values=values)
    Dref = oracle.tffr_weights(lx, 128)
    ref = oracle.adjoint_image(lx, ly, v, Dref, 128, 128)
    err = rel_l2(img, ref)
    assert err <= bound
    # against the rounded samples themselves the FP32 path is as exact as ever
    ref_stored = oracle.adjoint_image(lx, ly, stored, Dref, 128, 128)
    assert rel_l2(img, ref_stored) <= TOL


@pytest.mark.parametrize("q,a", [(3.0, 0.01), (2.5, 0.5), (2.2, 0.01)])
def test_weights_dense_offsets_and_threshold_decisions(q, a):
    """Fitted-G path against the closed form on a dense sweep of offsets, with tau placed
    inside the distribution so that many samples sit next to it: the kept set must be the
    oracle's (decisions are taken in FP64) and D must agree to FP32 rounding."""
    M = 64
    lam = np.concatenate([np.linspace(-31.97, 31.97, 60001), np.arange(-32.0, 32.0, 0.5),
                          [-32.0, 31.999999999, 0.0, -0.25, 29.0 + 2 ** -30]])
    D_all = oracle.tffr_weights(lam, M, q=q, a=a, tau=-1e30)
    tau = float(np.median(D_all[D_all > 0]))
    from paper_1910_10908_gb300 import Plan
    with Plan(M) as plan:
        lx, ly = dev(lam), dev(np.zeros_like(lam))
        plan.set_points(lx, ly)
        D = torch.empty(lam.shape[0], dtype=torch.float32, device="cuda")
        kept = plan.weights(q=q, a=a, tau=tau, D_out=D)
        D = D.cpu().numpy().astype(np.float64)
    Dref = oracle.tffr_weights(lam, M, q=q, a=a, tau=tau)
    assert kept == np.count_nonzero(Dref)
    assert np.array_equal(D != 0, Dref != 0)
    assert d_err(D, Dref) < 3e-7


def test_repeated_set_points_and_weights_calls():
    """A plan reused across calls (new points, new weights, the same or other (a, q)) keeps
    the oracle's answer; the plan-time fit of the weights is cached per (a, q)."""
    from paper_1910_10908_gb300 import Plan
    lx, ly, _, v = stolt_scene(64, 96, 64)
    lx2, ly2, _, v2 = stolt_scene(48, 80, 64, seed=12)
    vals, vals2 = dev(v.astype(np.complex64)), dev(v2.astype(np.complex64))
    with Plan(64) as plan:
        for rnd in range(3):
            for (x, y, val, vv) in ((lx, ly, vals, v), (lx2, ly2, vals2, v2)):
                tx, ty = dev(x), dev(y)
                plan.set_points(tx, ty)
                for kw in (dict(), dict(a=0.5, q=2.5), dict()):
                    plan.weights(count=False, **kw)
                    img = plan.adjoint(val).cpu().numpy().astype(np.complex128)
                    Dref = oracle.tffr_weights(x, 64, **kw)
                    ref = oracle.adjoint_image(x, y, vv.astype(np.complex64), Dref, 64, 64)
                    assert rel_l2(img, ref) <= TOL, (rnd, kw)


def expected_rows(lx, ly, nx, w):
    """Runs of bit-equal lam_y and the summed / longest row-buffer lengths (fine cells floor(2 lam))."""
    bits = ly.view(np.int64)
    starts = np.flatnonzero(np.concatenate([[True], bits[1:] != bits[:-1]]))
    ends = np.append(starts[1:], lx.shape[0])
    cells = np.floor(2.0 * lx).astype(np.int64)
    lens = [min(int(cells[s:e].max() - cells[s:e].min()) + w, nx) for s, e in zip(starts, ends)]
    return len(starts), int(np.sum(lens)), int(np.max(lens))


@pytest.mark.parametrize("case", ["long_rows_across_tiles", "more_rows_than_first_capacity", "repeated_lam_y",
                                  "rows_at_the_y_edges"])
def test_pulse_row_scan(case):
    """Pulse rows found by the one-pass scan: rows longer than a scan tile (4096 samples),
    more rows than the plan's first row capacity (4096, so the scan runs twice), a lam_y
    value that comes back after another row (two separate rows), single-sample rows, and
    rows whose azimuth taps wrap around the fine grid (rows of one fine y cell, in any
    order, and the first and last cells)."""
    M, w = 64, 8
    g = np.random.default_rng({"long_rows_across_tiles": 21, "more_rows_than_first_capacity": 22,
                               "repeated_lam_y": 23, "rows_at_the_y_edges": 24}[case])
    if case == "long_rows_across_tiles":
        lens = [1, 5000, 9000, 2, 4095, 4097, 1, 300]
    elif case == "more_rows_than_first_capacity":
        lens = list(g.integers(1, 12, 5000))
    elif case == "rows_at_the_y_edges":
        lens = [300, 40, 500, 7, 1, 260, 90, 120]
    else:
        lens = [700, 1, 900, 5, 4200, 33]
    ly_rows = g.uniform(-0.45 * M, 0.45 * M, len(lens))
    if case == "repeated_lam_y":
        ly_rows[2] = ly_rows[0]
        ly_rows[4] = ly_rows[0]
    if case == "rows_at_the_y_edges":
        ly_rows = np.array([M / 2 - 1e-9, -M / 2, 0.1, M / 2 - 0.3, -M / 2 + 0.2, 0.15, -M / 2 + 0.1, 0.1 + 2 ** -40])
    ly = np.repeat(ly_rows, lens)
    lx = np.empty(ly.shape[0])
    pos = 0
    for n in lens:                              # each row covers a random stretch of x
        c = g.uniform(-0.4 * M, 0.4 * M)
        lx[pos:pos + n] = np.clip(c + g.uniform(-6.0, 6.0, n), -M / 2, M / 2 - 1e-9)
        pos += n
    v = (g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])).astype(np.complex64)
    img, D, kept, info = gpu_adjoint(lx, ly, v, M, layout="rows", width=w)
    P, cells, longest = expected_rows(lx, ly, 2 * M, w)
    assert info["layout"] == 2
    assert (info["n_rows"], info["row_cells"], info["max_row_cells"]) == (P, cells, longest)
    assert info["pulse_order"] == (P <= M)
    ref = oracle.adjoint_image(lx, ly, v, oracle.tffr_weights(lx, M), M, M)
    assert rel_l2(img, ref) <= TOL


@pytest.mark.parametrize("tau", [0.97, 1.0, 1.02])
def test_deferred_fp64_weight_decisions_pulse_rows(tau):
    """Pulse-row samples whose weight is decided in FP64 after the spread: samples within q
    of the grid edges (every tau) and samples with 1/G within the guard band of tau (tau = 1.0
    catches those near integer frequencies, where G is within 1e-5 of 1)."""
    M = 64
    g = np.random.default_rng(31)
    lens = [60] * 40
    ly = np.repeat(g.uniform(-0.45 * M, 0.45 * M, len(lens)), lens)
    lx = np.empty(ly.shape[0])
    pos = 0
    for r, n in enumerate(lens):
        if r % 4 == 0:                          # rows hugging the low and high grid edges
            base = -M / 2 if r % 8 == 0 else M / 2 - 5.0
            lx[pos:pos + n] = base + np.sort(g.uniform(0.0, 5.0 - 1e-9, n))
        elif r % 4 == 1:                        # rows on and near integer frequencies
            lx[pos:pos + n] = np.round(g.uniform(-20, 20, n)) + g.choice([0.0, 1e-7, -1e-7, 0.5], n)
        else:
            lx[pos:pos + n] = np.sort(g.uniform(-0.45 * M, 0.45 * M, n))
        pos += n
    v = (g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0])).astype(np.complex64)
    img, D, kept, info = gpu_adjoint(lx, ly, v, M, layout="rows", width=8, wkw=dict(tau=tau))
    assert info["layout"] == 2
    Dref = oracle.tffr_weights(lx, M, tau=tau)
    assert kept == np.count_nonzero(Dref)
    ref = oracle.adjoint_image(lx, ly, v, Dref, M, M)
    assert rel_l2(img, ref) <= TOL


@pytest.mark.parametrize("order", ["auto", "fine_rows"])
def test_both_orders_of_the_fft_passes(order):
    """Pulse rows first (x FFT of the P pulse rows, azimuth taps inside the column pass) and
    fine rows first (azimuth taps, then the x FFT of every fine row) give the oracle's image
    and forward samples; non-square, so the two axes' sizes are not interchangeable."""
    from paper_1910_10908_gb300 import Plan
    lx, ly, _, v = stolt_scene(100, 160, 128, seed=41)
    ly = ly * 0.5                                   # azimuth grid of 64 rows
    Mx, My = 128, 64
    v = v.astype(np.complex64)
    img, D, kept, info = gpu_adjoint(lx, ly, v, Mx, My, layout="rows", width=8, order=order)
    assert info["layout"] == 2 and info["n_rows"] == 100
    assert info["pulse_order"] == 0                 # 100 pulse rows > My = 64: fine rows either way
    Dref = oracle.tffr_weights(lx, Mx)
    ref = oracle.adjoint_image(lx, ly, v, Dref, Mx, My)
    assert rel_l2(img, ref) <= TOL
    lx2, ly2, _, v2 = stolt_scene(48, 160, 128, seed=42)
    v2 = v2.astype(np.complex64)
    img2, _, _, info2 = gpu_adjoint(lx2, ly2, v2, Mx, Mx, layout="rows", width=8, order=order)
    assert info2["pulse_order"] == (1 if order == "auto" else 0)
    Dref2 = oracle.tffr_weights(lx2, Mx)
    assert rel_l2(img2, oracle.adjoint_image(lx2, ly2, v2, Dref2, Mx, Mx)) <= TOL
    g = np.random.default_rng(43)
    f = (g.standard_normal((Mx, Mx)) + 1j * g.standard_normal((Mx, Mx))).astype(np.complex64)
    with Plan(Mx, Mx, layout="rows", width=8, order=order) as plan:
        plan.set_points(dev(lx2), dev(ly2))
        plan.weights(count=False)
        y = plan.forward(dev(f)).cpu().numpy().astype(np.complex128)
    yref = oracle.forward_samples(lx2, ly2, f, Dref2)
    assert rel_l2(y, yref) <= TOL


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_crop():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg, np.load(os.path.join(GOLDEN, mg.CROP_FILE))


def test_stripmap_4096_centre_crop_against_the_stored_fp64_crop():
    """The bench configuration (16,714,266 samples -> 4096^2, c64, FP32 path) against the
    FP64 oracle's 256 x 256 centre crop, stored by tests/golden/make_golden.py: every one of
    the 65,536 pixels, as rel-L2 over the crop and as the largest pixel error against the
    crop's largest magnitude.  The FP16 / BF16 sample-storage variants are held to the
    rounding unit of their storage on the same crop."""
    mg, ref = _golden_crop()
    wl = make_workload(mg.CROP_WORKLOAD)
    jx0, jy0, nx, ny = mg.crop_box(wl.M)
    img, _, kept, info = gpu_adjoint(wl.lam_x, wl.lam_y, wl.values, wl.M)
    assert info["pulse_order"] == 1 and kept == wl.N
    got = img[jy0:jy0 + ny, jx0:jx0 + nx]
    assert got.shape == ref.shape == (256, 256)
    assert rel_l2(got, ref) <= TOL
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))
    v = dev(wl.values)
    for values, t, bound in (("f16", v.to(torch.complex32), 1e-3),
                             ("bf16", torch.view_as_real(v).to(torch.bfloat16).contiguous(), 8e-3)):
        img_v, _, _, _ = gpu_adjoint(wl.lam_x, wl.lam_y, t, wl.M, values=values)
        assert rel_l2(img_v[jy0:jy0 + ny, jx0:jx0 + nx], ref) <= bound, values


def test_stripmap_2048_crop_and_brightest_pixels():
    """The 2048^2 configuration of the differentiable variant (1024 pulses x 2048
    frequencies, 2,089,290 samples): a 64 x 64 centre crop and the 16 brightest pixels
    against the FP64 oracle."""
    wl = make_workload("stripmap_2048")
    img, D, kept, info = gpu_adjoint(wl.lam_x, wl.lam_y, wl.values, wl.M)
    assert info["layout"] == 2 and info["n_rows"] == 1024 and kept == wl.N
    Dref = oracle.tffr_weights(wl.lam_x, wl.M)
    j0 = wl.M // 2 - 32
    crop = oracle.adjoint_image(wl.lam_x, wl.lam_y, wl.values, Dref, wl.M, wl.M, crop=(j0, j0, 64, 64))
    assert rel_l2(img[j0:j0 + 64, j0:j0 + 64], crop) <= TOL
    flat = np.argsort(np.abs(img).ravel())[-16:]
    jy, jx = flat // wl.M, flat % wl.M
    ref = oracle.adjoint_pixels(wl.lam_x, wl.lam_y, wl.values, Dref, wl.M, wl.M, jx, jy)
    assert rel_l2(img[jy, jx], ref) <= TOL


def _oracle_weights_threaded(lam, M):
    from concurrent.futures import ThreadPoolExecutor
    chunks = np.array_split(lam, 16)
    with ThreadPoolExecutor(8) as ex:
        return np.concatenate(list(ex.map(lambda c: oracle.tffr_weights(c, M), chunks)))


def test_every_patch_of_the_64_patch_batch():
    """The bench's batch of 64 uneven sub-aperture patches (43.7M samples, sides 256-1024),
    run as one batch (graph replay): every patch's image against the FP64 oracle at 12
    random pixels and its 4 brightest."""
    from paper_1910_10908_gb300.batched import PatchBatch
    from synth import patch_batch
    pb = patch_batch(64)
    with PatchBatch([(m, m, dev(lx), dev(ly)) for m, lx, ly, _ in pb]) as batch:
        for k, (_, _, _, v) in enumerate(pb):
            batch.load(k, dev(v))
        batch.capture()
        batch.replay()
        batch.stream.synchronize()
        images = [im.cpu().numpy().astype(np.complex128) for im in batch.images]
    g = np.random.default_rng(25)
    errs = []
    for (M, lx, ly, v), img in zip(pb, images):
        D = _oracle_weights_threaded(lx, M)
        bright = np.argsort(np.abs(img).ravel())[-4:]
        jx = np.concatenate([g.integers(0, M, 12), bright % M])
        jy = np.concatenate([g.integers(0, M, 12), bright // M])
        ref = oracle.adjoint_pixels(lx, ly, v, D, M, M, jx, jy)
        errs.append(rel_l2(img[jy, jx], ref))
    assert max(errs) <= TOL, max(errs)
