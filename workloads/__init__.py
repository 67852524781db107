"""Seeded synthetic plasma loads shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This package only draws particle positions and velocities (host FP64 numpy
arrays) and describes the grid they live on.  It holds none of the PIC
cycle's arithmetic: no weighting, no push, no deposit, no field solve.
"""

from .plasma import (  # noqa: F401
    Workload,
    langmuir_1d,
    two_stream_2d,
    paper_two_stream,
    cold_two_stream_1d,
    two_stream_eigenmode_1d,
    magnetized_3d,
    precision_3d,
    batch_instances,
    maxwellian_box,
    sparse_box,
    fp32_exact,
    by_name,
)
