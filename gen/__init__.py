"""Seeded synthetic problem generators shared by the oracle side and the CUDA side.

This package builds test inputs only: sparse matrices of the model problems the
paper benchmarks on (Sec. 4, the 3D Poisson problem) and the further model
problems of the workloads (2D Poisson with a shift, variable-coefficient
diffusion, upwind convection-diffusion), plus right-hand sides.  It holds none
of the method's arithmetic (no aggregation, no prolongation, no cycle, no
Krylov step).  Random numbers come from one counter-based generator
(``gen.rng``) so that both sides, on any machine, see identical inputs.
"""
from .rng import uniform01, splitmix64_stream
from .problems import (
    Csr,
    poisson3d,
    poisson3d_star,
    poisson2d_shift,
    varcoef3d,
    convdiff3d,
    rhs_from_solution,
    uniform_pm1,
    sample_indices,
    poisson3d_nnz,
    batched_sides,
    serving_sides,
    serving_requests,
    ServeRequest,
)

__all__ = [
    "uniform01",
    "splitmix64_stream",
    "Csr",
    "poisson3d",
    "poisson3d_star",
    "poisson2d_shift",
    "varcoef3d",
    "convdiff3d",
    "rhs_from_solution",
    "uniform_pm1",
    "sample_indices",
    "poisson3d_nnz",
    "batched_sides",
    "serving_sides",
    "serving_requests",
    "ServeRequest",
]
