"""Seeded synthetic inputs for the AWG solver and for its CPU oracle.

This module is input generation only: it assembles sparse SPD matrices of the
kinds studied with the AWG preconditioners (Section 5 of the paper and the
scaled-up workloads built on it), non-overlapping partitions of their degrees
of freedom, and right-hand sides.  It holds none of the method's arithmetic:
no overlap growth, no splitting, no eigenproblem, no preconditioner.  Both the
CUDA path (through its tests and benchmark) and the oracle read their inputs
from here, so that the two sides see byte-identical problems.
"""

from .problems import (  # noqa: F401
    Problem,
    poisson2d,
    channels2d,
    grf3d,
    elasticity2d,
    paper_elasticity,
    paper_long_domain,
    random_spd,
    batch_channels,
    box_partition,
    config1,
    config2,
    config3,
    config4,
    config5,
    small_channels,
    block_rhs,
)
