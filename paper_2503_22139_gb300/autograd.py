"""torch.autograd.Function wrappers over the C ABI: each stage's forward and its
hand-written adjoint.  PyTorch only routes gradients; every value is computed
by libpmf.so.

    V = voxelize(grid, mean, scale, quat, value, kappa)            Eq. 4-5
    W = warp_combine(grid, V, E, coeff)                            Eq. 3 + Eq. 2
    Y = conebeam_project(grid, det, views, W)                      Eq. 6
    L = projection_loss(Y, M, kind)                                Eq. 10/12, Eq. 1
    D-SSIM, TV of a crop of V, MBC normality                       Eq. 10-14

`forward_model` chains them for one batch: reference Gaussians -> V, MBC
Gaussians of each level -> E, then W, Y and the loss.  Gradients flow to every
Gaussian parameter and to the temporal coefficients; the DVF and the warped
volume's adjoint are recomputed inside the adjoint calls rather than stored.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import ops


class GaussianVoxelize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean, scale, quat, value, grid, kappa: float, dtype=torch.float32):
        gs = ops.Gaussians(mean.detach(), scale.detach(), quat.detach(), value.detach(), kappa)
        out = ops.gs_voxelize(grid, gs, dtype=dtype)
        ctx.grid, ctx.kappa, ctx.value_shape = grid, kappa, value.shape
        ctx.save_for_backward(mean, scale, quat, value)
        return out

    @staticmethod
    def backward(ctx, g):
        mean, scale, quat, value = ctx.saved_tensors
        gs = ops.Gaussians(mean.detach(), scale.detach(), quat.detach(), value.detach(), ctx.kappa)
        dm, ds, dq, dv = ops.gs_voxelize_backward(ctx.grid, gs, g.float().contiguous())
        return dm, ds, dq, dv.reshape(ctx.value_shape), None, None, None


class WarpCombine(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ref, mbc, coeff, grid):
        ctx.grid = grid
        ctx.save_for_backward(ref, mbc, coeff)
        return ops.warp_combine(grid, ref.detach(), mbc.detach(), coeff.detach())

    @staticmethod
    def backward(ctx, g):
        ref, mbc, coeff = ctx.saved_tensors
        d_ref, d_mbc, d_coeff = ops.warp_combine_backward(ctx.grid, ref.detach(), mbc.detach(), coeff.detach(),
                                                          g.float().contiguous())
        return d_ref.to(ref.dtype), d_mbc.to(mbc.dtype), d_coeff, None


class ConebeamProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol, views, grid, det, shared: bool = False):
        ctx.grid, ctx.det, ctx.shared = grid, det, shared
        ctx.vol_dtype = vol.dtype
        ctx.save_for_backward(views)
        return ops.conebeam_project(grid, det, views, vol.detach(), shared=shared)

    @staticmethod
    def backward(ctx, g):
        (views,) = ctx.saved_tensors
        d_vol = ops.conebeam_project_backward(ctx.grid, ctx.det, views, g.float().contiguous(), shared=ctx.shared)
        return d_vol.to(ctx.vol_dtype), None, None, None, None


class ProjectionLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pred, meas, kind: int = 2):
        loss, d_pred = ops.projection_loss(kind, pred.detach(), meas.detach(), with_grad=True)
        ctx.save_for_backward(d_pred)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (d_pred,) = ctx.saved_tensors
        return d_pred * g, None, None


class ProjectionDSSIM(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pred, meas, data_range: float):
        loss, d_pred = ops.projection_dssim(pred.detach(), meas.detach(), data_range, with_grad=True)
        ctx.save_for_backward(d_pred)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (d_pred,) = ctx.saved_tensors
        return d_pred * g, None, None


class TVLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol, grid, D: int, origin):
        loss, d_vol = ops.tv_loss(grid, vol.detach(), D, origin, with_grad=True)
        ctx.vol_dtype = vol.dtype
        ctx.save_for_backward(d_vol)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (d_vol,) = ctx.saved_tensors
        return (d_vol * g).to(ctx.vol_dtype), None, None, None


class MBCNormality(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mbc, grid):
        loss, d_mbc = ops.mbc_normality(grid, mbc.detach(), with_grad=True)
        ctx.mbc_dtype = mbc.dtype
        ctx.save_for_backward(d_mbc)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (d_mbc,) = ctx.saved_tensors
        return (d_mbc * g).to(ctx.mbc_dtype), None


def voxelize(grid, mean, scale, quat, value, kappa: float = 3.0, dtype=torch.float32):
    return GaussianVoxelize.apply(mean, scale, quat, value, grid, kappa, dtype)


def warp_combine(grid, ref, mbc, coeff):
    return WarpCombine.apply(ref, mbc, coeff, grid)


def conebeam_project(grid, det, views, vol, shared: bool = False):
    return ConebeamProject.apply(vol, views, grid, det, shared)


def projection_loss(pred, meas, kind: int = 2):
    return ProjectionLoss.apply(pred, meas, kind)


def projection_dssim(pred, meas, data_range: float):
    return ProjectionDSSIM.apply(pred, meas, data_range)


def tv_loss(vol, grid, D: int, origin):
    return TVLoss.apply(vol, grid, D, origin)


def mbc_normality(mbc, grid):
    return MBCNormality.apply(mbc, grid)


def forward_model(grid, det, ref: Sequence[torch.Tensor], mbc: Sequence[Sequence[torch.Tensor]],
                  coeff: torch.Tensor, views: torch.Tensor, meas: Optional[torch.Tensor] = None,
                  kappa: float = 3.0, kind=2, dtype=torch.float32, eq14: Optional[dict] = None):
    """ref = (mean, scale, quat, value); mbc = one such tuple per level.
    Returns (Y, loss) with loss None when `meas` is None.  kind "eq14": the
    objective of Eq. 14 (eq14 = dict(lambda_ssim, lambda_mbc, lambda_tv,
    data_range, tv_size, tv_origin))."""
    V = voxelize(grid, *ref, kappa=kappa, dtype=dtype)[0]
    E = torch.stack([voxelize(grid, *m, kappa=kappa, dtype=dtype) for m in mbc])
    W = warp_combine(grid, V, E, coeff)
    Y = conebeam_project(grid, det, views, W)
    if meas is None:
        return Y, None
    if kind != "eq14":
        return Y, projection_loss(Y, meas, kind)
    q = eq14
    loss = (projection_loss(Y, meas, 1) + q["lambda_ssim"] * projection_dssim(Y, meas, q["data_range"])
            + q["lambda_mbc"] * mbc_normality(E, grid) + q["lambda_tv"] * tv_loss(V, grid, q["tv_size"], q["tv_origin"]))
    return Y, loss
