"""A batch of independent tFFR reconstructions (sub-aperture patches of uneven
sizes) replayed as one CUDA graph.

Each patch has its own plan; the plans are spread over a few streams so that
small patches, which cannot fill the GPU on their own, run side by side.  After
set_points and weights (which synchronise, and may allocate) the per-step work
of every patch is its adjoint alone, which neither allocates nor synchronises,
so the adjoints of all patches can be captured once into a CUDA graph on fixed
value and image buffers (the side streams fork from and join back to the
capturing stream) and replayed: one graph launch instead of a few kernel
launches per patch.  New samples are copied into the fixed value buffers
between replays.
"""

from __future__ import annotations

import torch

from . import Plan


class PatchBatch:
    """Plans, fixed value buffers and images for a list of patches.

    patches: list of (Mx, My, lam_x, lam_y) with device float64 coordinates
    (kept by reference, like Plan.set_points).
    """

    def __init__(self, patches, *, values: str = "c64", width: int = 6, device=None, streams: int = 8,
                 **weight_opts):
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
        self.graph = None

    @property
    def samples(self) -> int:
        return sum(p.N for p in self.plans)

    def load(self, k: int, values: torch.Tensor):
        """Copy patch k's samples into its fixed buffer (ordered on the batch stream)."""
        with torch.cuda.stream(self.stream):
            self.values[k].copy_(values, non_blocking=True)

    def _adjoints(self):
        # fork: every side stream waits for the batch stream, runs its patches,
        # and the batch stream waits for all of them
        for st in self.side:
            st.wait_stream(self.stream)
        for p, v, img in zip(self.plans, self.values, self.images):
            p.adjoint(v, out=img)                  # on the plan's own (side) stream
        for st in self.side:
            self.stream.wait_stream(st)

    def adjoint_eager(self):
        """Every patch's adjoint, ordered after the batch stream's prior work and
        before its later work."""
        self._adjoints()

    def capture(self):
        """Record every patch's adjoint into one CUDA graph (once)."""
        self.adjoint_eager()                       # warm: every kernel has run once
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._adjoints()
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def close(self):
        self.graph = None
        for p in self.plans:
            p.close()
        self.plans = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
