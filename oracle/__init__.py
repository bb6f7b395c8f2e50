"""FP64 CPU oracle for the PMF-STGR forward model and adjoint.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  It shares no code with the
CUDA path; the seeded generators in `synth` are the only thing both consume.
"""
from .oracle import (  # noqa: F401
    lib, threads, set_threads, quat_to_rot,
    voxelize, voxelize_ambiguity, voxelize_tie_band, qform_and_bound, voxelize_backward,
     combine, combine_backward, warp, warp_backward,
    project, project_backward, project_gaussians, loss, dssim, tv, mbc_normality,
    splat_params, splat, splat_backward, round_storage,
)
