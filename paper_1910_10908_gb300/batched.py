"""A batch of independent tFFR reconstructions (sub-aperture patches of uneven
sizes).

Each patch has its own plan (points and weights set once, fixed value and
image buffers).  The batch's adjoint (tffr_batch_adjoint) is one spread launch
over every pulse row of every patch, then one persistent FFT launch per image
side whose blocks claim work items from a device counter (the x FFT of every
pulse row or fine row, then the column pass of every patch), so that small
patches, which cannot fill the GPU on their own, share it without launches of
their own.  The launch neither allocates nor
synchronises, so it is captured once into a CUDA graph and replayed; new
samples are copied into the fixed value buffers between replays.

For comparison the per-plan path stays: every patch's own tffr_adjoint, the
plans spread over a few streams (adjoint_eager), or one after the other on one
stream (streams=1).
"""

from __future__ import annotations

import torch

from . import (Plan, tffr_batch_adjoint, tffr_batch_create, tffr_batch_destroy, tffr_batch_get_info,
               tffr_batch_set_wait, tffr_batch_tune, tffr_batch_wait)


class PatchBatch:
    """Plans, fixed value buffers and images for a list of patches.

    patches: list of (Mx, My, lam_x, lam_y) with device float64 coordinates
    (kept by reference, like Plan.set_points).  persistent=True builds the
    batch launches (square patches of side 256, 512 or 1024 with complex64
    samples); persistent=False keeps only the per-plan path.
    """

    def __init__(self, patches, *, values: str = "c64", width: int = 6, device=None, streams: int = 8,
                 persistent: bool = True, **weight_opts):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.Stream(device=self.device)             # the batch's own (capturing) stream
        self.side = [torch.cuda.Stream(device=self.device) for _ in range(max(1, streams))]
        self.plans, self.values, self.images = [], [], []
        with torch.cuda.device(self.device):
            for k, (Mx, My, lx, ly) in enumerate(patches):
                with torch.cuda.stream(self.side[k % len(self.side)]):
                    p = Plan(Mx, My, values=values, width=width, device=self.device)
                    p.set_points(lx, ly)
                    p.weights(count=False, **weight_opts)
                    self.plans.append(p)
                    self.values.append(p.value_tensor())
                    self.images.append(torch.empty((My, Mx), dtype=torch.complex64, device=self.device))
            torch.cuda.synchronize(self.device)
            self._b = None
            if persistent:
                self._b = tffr_batch_create([p._handle() for p in self.plans], self.values, self.images,
                                            stream=self.stream)
        self.graph = None

    @property
    def samples(self) -> int:
        return sum(p.N for p in self.plans)

    def load(self, k: int, values: torch.Tensor):
        """Copy patch k's samples into its fixed buffer (ordered on the batch stream)."""
        with torch.cuda.stream(self.stream):
            self.values[k].copy_(values, non_blocking=True)

    def _persistent(self):
        if self._b is None:
            raise RuntimeError("built without the persistent batch")
        return self._b

    def adjoint(self):
        """Every patch's adjoint by the persistent launches, ordered on the batch stream."""
        tffr_batch_adjoint(self._persistent())

    def wait(self):
        """Synchronise; raises TffrError (TIMEOUT) if a launch's wait ran out."""
        tffr_batch_wait(self._persistent())

    def tune(self, reps: int = 5) -> dict:
        """Autotune the persistent FFT launches (blocks per SM); returns info()."""
        tffr_batch_tune(self._persistent(), reps)
        return self.info()

    def set_wait(self, wait_s: float = 1.0, hold_rows: bool = False):
        tffr_batch_set_wait(self._persistent(), wait_s, hold_rows)

    def info(self) -> dict:
        return tffr_batch_get_info(self._persistent())

    def _adjoints_per_plan(self):
        # fork: every side stream waits for the batch stream, runs its patches,
        # and the batch stream waits for all of them
        for st in self.side:
            st.wait_stream(self.stream)
        for p, v, img in zip(self.plans, self.values, self.images):
            p.adjoint(v, out=img)                  # on the plan's own (side) stream
        for st in self.side:
            self.stream.wait_stream(st)

    def adjoint_eager(self):
        """Every patch's own tffr_adjoint on the side streams, ordered after the batch
        stream's prior work and before its later work."""
        self._adjoints_per_plan()

    def capture(self, persistent: bool | None = None):
        """Record every patch's adjoint into one CUDA graph (once): the persistent launches,
        or (persistent=False) the per-plan calls."""
        if persistent is None:
            persistent = self._b is not None
        run = self.adjoint if persistent else self._adjoints_per_plan
        with torch.cuda.stream(self.stream):
            run()                                  # warm: every kernel has run once
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            run()
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def close(self):
        self.graph = None
        if self._b is not None:
            tffr_batch_destroy(self._b)
            self._b = None
        for p in self.plans:
            p.close()
        self.plans = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
