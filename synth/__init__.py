"""Seeded synthetic inputs shaped like the paper's workloads.

Used by the tests and the benchmark on both sides (library and oracle).  It
holds no clustering arithmetic: only data generation.
"""

from .workloads import (  # noqa: F401
    SEED_BASE,
    blobs,
    mnist_like,
    md_trajectory,
    batched_problems,
    random_rigid_motion,
)
