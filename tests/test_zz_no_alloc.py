"""The allocation-free weights entry point (tffr_weights_noalloc) against tffr_weights.

tffr_weights_noalloc serves callers that cannot allocate device memory when
they need the weights (inside a stream capture, under a fixed memory budget):
it needs no plan and keeps its scratch in a fixed device array inside the
library.  This file is collected last on purpose, so that a run stopping at
the first failure has already run every other test.  Two calls in a row check
that the shared scratch left by one call does not leak into the next.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import stolt_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def plan_weights(lx, ly, Mx, My, **kw):
    from paper_1910_10908_gb300 import Plan
    with Plan(Mx, My) as plan:
        plan.set_points(lx, ly)
        D = torch.empty(lx.shape[0], dtype=torch.float32, device="cuda")
        kept = plan.weights(D_out=D, **kw)
        torch.cuda.synchronize()
        return D.cpu().numpy().astype(np.float64), kept


def test_noalloc_weights_match_the_plan_weights_on_two_calls():
    from paper_1910_10908_gb300 import tffr_weights_noalloc
    cases = [
        (stolt_points(96, 160, 64), 64, 64, dict(tau=1.02)),
        (stolt_points(40, 300, 128), 128, 32, dict(tau=1.0, separable=True, a=0.5, q=2.5)),
    ]
    for (lx_np, ly_np, _), Mx, My, kw in cases:
        if My != Mx:
            ly_np = ly_np * (My / Mx)
        lx = torch.from_numpy(lx_np).cuda()
        ly = torch.from_numpy(ly_np).cuda()
        D_ref, kept_ref = plan_weights(lx, ly, Mx, My, **kw)
        D = torch.full((lx.shape[0],), -1.0, dtype=torch.float32, device="cuda")
        kept = tffr_weights_noalloc(lx, ly, Mx, My, D, **kw)
        torch.cuda.synchronize()
        D = D.cpu().numpy().astype(np.float64)
        assert kept == kept_ref
        assert np.array_equal(D != 0, D_ref != 0)
        assert np.max(np.abs(D - D_ref) / np.maximum(1.0, np.abs(D_ref))) < 3e-7


def test_noalloc_weights_match_the_oracle():
    """Straight against the FP64 oracle (not only against tffr_weights): range-only and
    separable weights, with tau inside the range of D so that the threshold decides."""
    from paper_1910_10908_gb300 import tffr_weights_noalloc
    lx_np, ly_np, _ = stolt_points(96, 160, 64)
    ly_np = ly_np * 0.5                                   # azimuth band of a 32-row image
    lx, ly = torch.from_numpy(lx_np).cuda(), torch.from_numpy(ly_np).cuda()
    for kw in (dict(), dict(tau=1.02), dict(tau=1.05, separable=True), dict(a=0.5, q=2.5, tau=1.0)):
        okw = {k: kw[k] for k in ("tau", "a", "q") if k in kw}
        Dref = oracle.tffr_weights(lx_np, 64, lam_y=ly_np, My=32, separable=kw.get("separable", False), **okw)
        for _ in range(2):
            D = torch.full((lx.shape[0],), -1.0, dtype=torch.float32, device="cuda")
            kept = tffr_weights_noalloc(lx, ly, 64, 32, D, **kw)
            torch.cuda.synchronize()
            D = D.cpu().numpy().astype(np.float64)
            assert kept == np.count_nonzero(Dref)
            assert np.array_equal(D != 0, Dref != 0)
            assert np.max(np.abs(D - Dref) / np.maximum(1.0, np.abs(Dref))) < 3e-7


def test_noalloc_weights_under_stream_capture():
    """Callers that cannot allocate are often inside a stream capture: after one eager call
    (which looks up the scratch array on this device), the call with count=False is
    captured into a CUDA graph and replayed twice into an output buffer holding other
    contents each time; both replays give the plan's weights."""
    from paper_1910_10908_gb300 import tffr_weights_noalloc
    lx_np, ly_np, _ = stolt_points(96, 160, 64)
    lx, ly = torch.from_numpy(lx_np).cuda(), torch.from_numpy(ly_np).cuda()
    D_ref, _ = plan_weights(lx, ly, 64, 64, tau=1.02)
    D = torch.empty(lx.shape[0], dtype=torch.float32, device="cuda")
    tffr_weights_noalloc(lx, ly, 64, 64, D, tau=1.02)              # eager: scratch looked up here
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        tffr_weights_noalloc(lx, ly, 64, 64, D, tau=1.02, count=False)
    for fill in (-1.0, 7.0):
        D.fill_(fill)
        graph.replay()
        torch.cuda.synchronize()
        got = D.cpu().numpy().astype(np.float64)
        assert np.array_equal(got != 0, D_ref != 0)
        assert np.max(np.abs(got - D_ref) / np.maximum(1.0, np.abs(D_ref))) < 3e-7


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1910_10908_gb300 import _abi
    import ctypes
    lib = _abi.load()
    o = _abi.tffr_weight_opts()
    lib.tffr_default_weight_opts(ctypes.byref(o))
    too_many = 67_108_864 + 1
    assert lib.tffr_weights_noalloc(too_many, None, None, 64, 64, ctypes.byref(o), None, None, None) \
        == _abi.TFFR_ERR_INVALID_ARG
