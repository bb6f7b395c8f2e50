"""GB300-native (sm_103a) forward model of PMF-STGR and its adjoint.

Stages (Xie, Shao & Zhang, Sec. 2): Gaussian voxelization of the reference
volume (Eq. 4-5) and of the signed motion-basis components, the DVF combine
(Eq. 3), the pull warp (Eq. 2), and the cone-beam line integrals (Eq. 6) with
an L1/L2 projection loss -- each with a hand-written adjoint.  The compute lives
in the C-ABI library built from csrc/ (see include/pmf.h); this package is its
argument-marshalling binding.
"""
from . import ops  # noqa: F401
from ._lib import PmfError  # noqa: F401
from .ops import (  # noqa: F401
    Adam, Gaussians, Plan, adam_step, autotune, circular_views, conebeam_project, conebeam_project_backward,
    conebeam_project_backward_absmax, conebeam_project_backward_batched, conebeam_project_batched, device_counters, device_status, gs_voxelize,
    gs_voxelize_backward, gs_voxelize_count, gs_rasterize, gs_rasterize_backward, gs_rasterize_count,
    gs_density_control, gs_density_threshold, gs_grad_norm_accumulate, gs_voxelize_tiled, gs_voxelize_tiled_count,
    mbc_combine, mbc_combine_backward, mbc_normality, projection_dssim,
    projection_loss, tv_loss, views_tensor,
    warp_combine, warp_combine_backward, warp_combine_backward_bounded, warp_combine_mixed, warp_volume, warp_volume_backward, workspace_size,
)

__all__ = [
    "Adam", "Gaussians", "Plan", "PmfError", "adam_step", "autotune", "circular_views", "conebeam_project", "conebeam_project_backward",
    "conebeam_project_backward_absmax", "conebeam_project_backward_batched", "conebeam_project_batched", "device_counters", "device_status",
    "gs_voxelize", "gs_voxelize_backward", "gs_voxelize_count", "gs_rasterize", "gs_rasterize_backward",
    "gs_rasterize_count", "gs_density_control", "gs_density_threshold", "gs_grad_norm_accumulate", "gs_voxelize_tiled", "gs_voxelize_tiled_count", "mbc_combine", "mbc_combine_backward",
    "mbc_normality", "projection_dssim", "projection_loss", "tv_loss", "views_tensor", "warp_combine", "warp_combine_backward", "warp_combine_backward_bounded", "warp_combine_mixed", "warp_volume",
    "warp_volume_backward", "workspace_size",
]
