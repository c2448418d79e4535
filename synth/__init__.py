"""Seeded synthetic stripmap-SAR inputs shared by the tests, the bench and the oracle timing.

This package draws coordinates and sample values only.  It holds none of the
reconstruction arithmetic (no weights, no spreading, no transform); both the
CUDA path and the FP64 oracle consume what it produces.
"""

from .stripmap import (  # noqa: F401
    C0,
    StripmapWorkload,
    stolt_points,
    scene_samples,
    make_workload,
    random_points,
    patch_batch,
    edge_rows,
    WORKLOADS,
)
