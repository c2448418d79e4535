"""A batch of uneven patches replayed as one CUDA graph gives the images of the
eager calls, and each patch's image is the oracle's (GPU)."""

import numpy as np
import pytest
import torch

import oracle
from synth import patch_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def test_graph_replay_matches_eager_and_oracle():
    from paper_1910_10908_gb300.batched import PatchBatch
    pb = patch_batch(6, seed=77, sides=(64, 128), pulses=(16, 96), freqs=(32, 256))
    dev = torch.device("cuda", 0)
    patches = [(M, M, torch.from_numpy(lx).to(dev), torch.from_numpy(ly).to(dev)) for M, lx, ly, _ in pb]
    with PatchBatch(patches, width=8, streams=3) as batch:   # white random samples: width 8 (see the parity tests)
        assert batch.samples == sum(lx.shape[0] for _, lx, _, _ in pb)
        for k, (_, _, _, v) in enumerate(pb):
            batch.load(k, torch.from_numpy(v).to(dev))
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
