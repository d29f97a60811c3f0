"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the solver: it only defines the
coefficient fields kappa(r, z), q(r, z) and the right-hand sides f_m(r, z) of
the axisymmetric problem (1/r)d_r(r kappa d_r u) + d_z(kappa d_z u) - q u = -f
as plain functions of position on [0, 1] x [0, 1] (`laguerre.py`: the
Laguerre-chain inputs on a domain in metres, and the source wavelet's
coefficients).  Each side (the CPU oracle and the CUDA path's host code)
samples them at its own grid points.
"""
from .media import (  # noqa: F401
    Medium,
    SEED_ROOT,
    bumps_medium,
    layered_inclusion_medium,
    batched_instances,
    grf_medium,
    grf_spec,
    large_medium,
    large_spec,
    manufactured_medium,
    manufactured_medium_neumann,
    WORKLOADS,
)
