"""Seeded synthetic inputs for the PMF-STGR forward model and its adjoint.

This module only draws random numbers and lays out the scanner geometry; it holds
none of the method's arithmetic (no voxelization, warp, projection or loss).  Both
the CUDA path and the FP64 oracle consume what it produces.
"""
from .workloads import (  # noqa: F401
    Grid, Detector, GaussianSet, Workload,
    circular_views, small_workload, paper_workload, paper_workload_1mm, fd_subproblem, uneven_volumes,
    gaussian_set, mbc_levels, breathing_coefficients, uniform_coefficients,
    measured_projections, select_batch, seeds_for,
)
