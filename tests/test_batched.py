"""Batches of uneven patches (GPU): the per-plan path replayed as one CUDA graph, and
the batch launches (one spread over every patch's pulse rows, then one persistent FFT
launch per image side over rows, fine rows and columns) against the per-plan images
and the FP64 oracle; the bounded wait of the persistent launch, made to run out on
purpose; the autotuner."""

import numpy as np
import pytest
import torch

import oracle
from synth import edge_rows, patch_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _load(batch, pb, dev):
    for k, (_, _, _, v) in enumerate(pb):
        batch.load(k, torch.from_numpy(v).to(dev))


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_graph_replay_matches_eager_and_oracle():
    from paper_1910_10908_gb300.batched import PatchBatch
    pb = patch_batch(6, seed=77, sides=(64, 128), pulses=(16, 96), freqs=(32, 256))
    dev = torch.device("cuda", 0)
    patches = [(M, M, torch.from_numpy(lx).to(dev), torch.from_numpy(ly).to(dev)) for M, lx, ly, _ in pb]
    # white random samples: width 8 (see the parity tests); sides below 256: per-plan path only
    with PatchBatch(patches, width=8, streams=3, persistent=False) as batch:
        assert batch.samples == sum(lx.shape[0] for _, lx, _, _ in pb)
        _load(batch, pb, dev)
        batch.adjoint_eager()
        batch.stream.synchronize()
        with torch.cuda.stream(batch.stream):
            eager = [img.clone() for img in batch.images]
            for img in batch.images:
                img.zero_()
        batch.capture()
        with torch.cuda.stream(batch.stream):
            for img in batch.images:
                img.zero_()
        batch.replay()
        batch.replay()                                  # replays are repeatable
        batch.stream.synchronize()
        for e, r in zip(eager, batch.images):
            assert torch.linalg.vector_norm(e - r) <= 1e-6 * torch.linalg.vector_norm(e)
        # new samples through the same graph
        g = np.random.default_rng(9)
        M, lx, ly, _ = pb[2]
        v2 = ((g.standard_normal(lx.shape[0]) + 1j * g.standard_normal(lx.shape[0]))).astype(np.complex64)
        batch.load(2, torch.from_numpy(v2).to(dev))
        batch.replay()
        batch.stream.synchronize()
        img = batch.images[2].cpu().numpy().astype(np.complex128)
    ref = oracle.adjoint_image(lx, ly, v2, oracle.tffr_weights(lx, M), M, M)
    assert np.linalg.norm(img - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("width", [6, 8])
def test_persistent_batch_matches_per_plan_path_and_oracle(width):
    """Two image sides (two launches), ragged pulse rows, patches in both orders of the
    passes (up to 600 pulse rows on 256 x 256 images: the fine-row order): the persistent
    images equal the per-plan images (the same arithmetic in another order) over every
    pixel and, patch by patch, the oracle's at sampled pixels and the brightest ones."""
    from paper_1910_10908_gb300.batched import PatchBatch
    pb = patch_batch(8, seed=78, sides=(256, 512), pulses=(24, 600), freqs=(48, 400))
    dev = torch.device("cuda", 0)
    patches = [(M, M, torch.from_numpy(lx).to(dev), torch.from_numpy(ly).to(dev)) for M, lx, ly, _ in pb]
    with PatchBatch(patches, width=width, streams=2) as batch:
        _load(batch, pb, dev)
        info = batch.info()
        assert info["n_patches"] == 8 and info["n_classes"] == len({M for M, _, _, _ in pb})
        orders = {p.info()["pulse_order"] for p in batch.plans}
        assert orders == {0, 1}
        batch.adjoint_eager()
        batch.stream.synchronize()
        per_plan = [img.clone() for img in batch.images]
        with torch.cuda.stream(batch.stream):
            for img in batch.images:
                img.fill_(float("nan"))
        batch.adjoint()
        batch.wait()
        persistent = [img.clone() for img in batch.images]
    for a, b in zip(persistent, per_plan):
        assert rel(a, b) <= 1e-6
    tol = 1e-5 if width == 8 else 2e-5                  # white samples: width 6 sits near 1e-5 at the edges
    g = np.random.default_rng(81)
    for (M, lx, ly, v), img in zip(pb, persistent):
        got = img.cpu().numpy().astype(np.complex128)
        bright = np.argsort(np.abs(got).ravel())[-8:]
        jx = np.concatenate([g.integers(0, M, 56), bright % M])
        jy = np.concatenate([g.integers(0, M, 56), bright // M])
        ref = oracle.adjoint_pixels(lx, ly, v, oracle.tffr_weights(lx, M), M, M, jx, jy)
        assert np.linalg.norm(got[jy, jx] - ref) / np.linalg.norm(ref) <= tol


def test_batch_spread_rows_whose_every_sample_takes_the_fp64_decision():
    """Patches whose pulse rows lie within q + 1 cells of the grid's edges: the batch spread lists
    every sample of every row for the FP64 decision in that row's region of the batch's list and
    decides them in the row's block; the images equal the per-plan images and the oracle's."""
    from paper_1910_10908_gb300.batched import PatchBatch
    M = 256
    pts = [edge_rows(M, 30 + 10 * k, 100 + 20 * k, seed=40 + k) for k in range(3)]
    dev = torch.device("cuda", 0)
    patches = [(M, M, torch.from_numpy(lx).to(dev), torch.from_numpy(ly).to(dev)) for lx, ly, _ in pts]
    with PatchBatch(patches, width=8, streams=2) as batch:
        for k, (_, _, v) in enumerate(pts):
            batch.load(k, torch.from_numpy(v).to(dev))
        batch.adjoint_eager()
        batch.stream.synchronize()
        per_plan = [img.clone() for img in batch.images]
        with torch.cuda.stream(batch.stream):
            for img in batch.images:
                img.fill_(float("nan"))
        batch.adjoint()
        batch.wait()
        persistent = [img.clone() for img in batch.images]
    for a, b in zip(persistent, per_plan):
        assert rel(a, b) <= 1e-6
    for (lx, ly, v), img in zip(pts, persistent):
        ref = oracle.adjoint_image(lx, ly, v, oracle.tffr_weights(lx, M), M, M)
        got = img.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


def test_persistent_batch_wait_runs_out_and_the_gpu_recovers():
    """Row items told not to publish their completion: every column item's wait runs out
    (after 0.05 s of device time for the first, at once for the rest), the launch ends, and
    tffr_batch_wait reports TIMEOUT.  The same batch then runs normally."""
    from paper_1910_10908_gb300 import TffrError
    from paper_1910_10908_gb300.batched import PatchBatch
    pb = patch_batch(3, seed=79, sides=(256,), pulses=(24, 64), freqs=(48, 160))
    dev = torch.device("cuda", 0)
    patches = [(M, M, torch.from_numpy(lx).to(dev), torch.from_numpy(ly).to(dev)) for M, lx, ly, _ in pb]
    with PatchBatch(patches, width=8, streams=1) as batch:
        _load(batch, pb, dev)
        batch.adjoint_eager()
        batch.stream.synchronize()
        ref = [img.clone() for img in batch.images]
        batch.set_wait(0.05, hold_rows=True)
        batch.adjoint()
        with pytest.raises(TffrError) as e:
            batch.wait()
        assert e.value.status == 5
        batch.set_wait(1.0, hold_rows=False)
        batch.adjoint()
        batch.wait()
        for a, b in zip(batch.images, ref):
            assert rel(a, b) <= 1e-6


def test_autotuner_and_graph_capture_of_the_persistent_batch():
    """The autotuner keeps one of its candidates per class and the images stay those of
    the per-plan path; the persistent launches captured once and replayed twice."""
    from paper_1910_10908_gb300.batched import PatchBatch
    pb = patch_batch(5, seed=80, sides=(256, 512, 1024), pulses=(32, 160), freqs=(64, 400))
    dev = torch.device("cuda", 0)
    patches = [(M, M, torch.from_numpy(lx).to(dev), torch.from_numpy(ly).to(dev)) for M, lx, ly, _ in pb]
    with PatchBatch(patches, width=8) as batch:
        _load(batch, pb, dev)
        batch.adjoint_eager()
        batch.stream.synchronize()
        ref = [img.clone() for img in batch.images]
        info = batch.tune(reps=2)
        assert info["tuned"]
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        for c in info["classes"]:
            assert c["blocks"] % sms == 0 and c["blocks"] >= sms and c["ms"] > 0
        batch.capture()
        for _ in range(2):
            with torch.cuda.stream(batch.stream):
                for img in batch.images:
                    img.zero_()
            batch.replay()
            batch.wait()
            for a, b in zip(batch.images, ref):
                assert rel(a, b) <= 1e-6
