"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds no part of the descriptor or model arithmetic: it only draws
atomic structures (positions, cells, species), sparse-set selections and model
weights from seeded NumPy generators, and names the standard workloads.
"""
from .boxes import (  # noqa: F401
    Structure,
    Batch,
    random_box,
    batched_boxes,
    concat,
    sparse_indices,
    gap_weights,
    random_rotation,
)
from .workloads import WORKLOADS, Workload, get_workload  # noqa: F401
