"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package generates node sets and problem data only; it contains none of
the RBF-FD method's arithmetic (no neighbour search, no weights, no matrix,
no solver).  Both the CPU oracle and the CUDA path take its outputs as inputs.
"""

from .disk import (  # noqa: F401
    splitmix64,
    uniform01,
    disk_nodes,
    h_for_nodes,
    manufactured,
    fourier_params,
    fourier_sources,
    batched_instances,
    sample_indices,
    DiskNodes,
    CONFIGS,
)
