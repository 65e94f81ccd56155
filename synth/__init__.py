"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds no arithmetic of the KFAC method: it draws collocation
points, Xavier-initialised weights and the closed-form problem data (right-hand
side f, boundary data g, manufactured solution u*) of the PDE problems the
paper studies (Sec. 4 and App. A).  Both sides of every parity test take their
inputs from here, so that neither needs the other.
"""
from .inputs import (  # noqa: F401
    PROBLEMS,
    Problem,
    WORKLOADS,
    Workload,
    param_count,
    layer_shapes,
    xavier_theta,
    sample_interior,
    sample_boundary,
    make_batch,
)
