"""One forward + adjoint pass of the PMF-STGR model over a batch of projections
(Sec. 2.3.2, Stages 2-3): every stage is a C-ABI call, buffers are allocated
once and reused, and nothing runs outside libpmf.so's kernels.

    V  = gs_voxelize(reference Gaussians)                  Eq. 4-5
    E_l = gs_voxelize(MBC Gaussians of level l)            Sec. 2.3.1
    W_p = warp_combine(V, E, w_p)                          Eq. 3 + Eq. 2 (DVF never stored)
    Y_p = conebeam_project(W_p)                            Eq. 6
    L, dY = projection_loss(Y, M)                          Eq. 10/12 (L1) or Eq. 1 (L2)
    dW = conebeam_project_backward(dY)
    dV, dE, dw = warp_combine_backward(dW)                 DVF recomputed
    d(ref Gaussians), d(MBC Gaussians) = gs_voxelize_backward(...)
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import torch

from . import ops
from .ops import Gaussians

# kernels each entry point launches (memsets excluded): used for the launch count
KERNELS = {
    "gs_voxelize": 4, "gs_voxelize_backward": 2, "warp_combine": 1, "conebeam_project": 1,
    # warp_combine_backward as the step calls it: bounded by the back-projector's
    # max |dW|, so without an abs-max pass of its own (4 launches unbounded)
    "projection_loss": 2, "conebeam_project_backward": 3, "warp_combine_backward": 3,
    "projection_dssim": 3, "tv_loss": 2, "mbc_normality": 3,
    # rasterizer: frames, prep, 3 scan passes, fill, render; adjoint: frames, prep, sums, chain
    "gs_rasterize": 7, "gs_rasterize_backward": 4, "pmf_shift_means": 1,
}

# The Stage 2-3 objective of Eq. 14 with the paper's weights (Sec. 2.3.2):
# L1 + 0.25 D-SSIM + 1 L_MBC + 0.05 TV on a 32^3 crop of the reference volume.
EQ14_DEFAULTS = dict(lambda_ssim=0.25, lambda_mbc=1.0, lambda_tv=0.05, tv_size=32, data_range=None)


def vox_bwd_launches(grid, gs) -> int:
    """Kernels one gs_voxelize_backward call launches: the slab pass, plus the
    final pass when the set is split into several slabs (exactly when the call
    needs a workspace)."""
    return 1 + (ops.gs_voxelize_backward_workspace(grid, gs.n, gs.channels) > 0)


class ForwardAdjoint:
    def __init__(self, grid, det, ref: Gaussians, mbc: Sequence[Gaussians], batch: int,
                 dtype: torch.dtype = torch.float32, kind=2, pair_headroom: float = 1.25,
                 eq14: Optional[dict] = None, w_dtype: torch.dtype = torch.float32, concurrent_sets: bool = True):
        """kind 1 / 2: L1 / L2 projection loss (Eq. 10/12, Eq. 1); kind "eq14":
        the full objective of Eq. 14 with `eq14` overriding EQ14_DEFAULTS
        (data_range, the D-SSIM dynamic range, is required).  V and E are
        stored in dtype; the warped volumes W in w_dtype (fp32 by default: the
        projector stages fp32 volumes with bulk tensor copies)."""
        if w_dtype not in (dtype, torch.float32):
            raise ValueError("w_dtype must be dtype or torch.float32")
        det = ops._det(det)  # (nu, nv, step) tuples or detector records
        self.concurrent_sets, self._side = bool(concurrent_sets), None
        self.grid, self.det, self.ref, self.mbc = grid, det, ref, list(mbc)
        self.B, self.dtype, self.w_dtype = int(batch), dtype, w_dtype
        self.eq14 = None
        if kind == "eq14":
            q = dict(EQ14_DEFAULTS)
            q.update(eq14 or {})
            if q["data_range"] is None:
                raise ValueError("eq14 needs data_range (the projections' dynamic range)")
            self.eq14 = q
            kind = 1
        self.kind = int(kind)
        dev = ref.mean.device
        shape, n = ops._shape(grid)
        L = len(self.mbc)
        self.L = L
        # buffers
        self.V = torch.empty((1,) + shape, dtype=dtype, device=dev)
        self.E = torch.empty((L, 3) + shape, dtype=dtype, device=dev)
        self.W = torch.empty((self.B,) + shape, dtype=w_dtype, device=dev)
        self.Y = torch.empty((self.B, det.nv, det.nu), dtype=torch.float32, device=dev)
        self.dW = torch.empty((self.B,) + shape, dtype=torch.float32, device=dev)
        self.dW_max = torch.zeros(1, dtype=torch.int32, device=dev)  # max |dW| bits, from the back-projector
        self.g_ref = (torch.empty((ref.n, 3), device=dev), torch.empty((ref.n, 3), device=dev),
                      torch.empty((ref.n, 4), device=dev), torch.empty((ref.n, ref.channels), device=dev))
        self.g_mbc = [(torch.empty((m.n, 3), device=dev), torch.empty((m.n, 3), device=dev),
                       torch.empty((m.n, 4), device=dev), torch.empty((m.n, m.channels), device=dev))
                      for m in self.mbc]
        self.g_wc = (torch.empty(shape, dtype=torch.float32, device=dev),
                     torch.empty((L, 3) + shape, dtype=torch.float32, device=dev),
                     torch.empty((self.B, L, 3), dtype=torch.float32, device=dev))
        # scratch, sized once
        self.vox_ws = []
        for gs in [ref] + self.mbc:
            cap = int(ops.gs_voxelize_count(grid, gs) * pair_headroom) + 4096
            self.vox_ws.append(ops._ws(ops.gs_voxelize_workspace(grid, gs.n, cap), dev))
        Lb = ops._lib.load()
        g = ops._grid(grid)
        self.bp_ws = ops._ws(ops._size(Lb.conebeam_project_backward_workspace, ops.ct.byref(g), self.B, n), dev)
        self.wc_ws = ops._ws(ops._size(Lb.warp_combine_backward_workspace, ops.ct.byref(g), L, self.B), dev)
        self.loss_ws = ops._ws(ops._size(Lb.projection_loss_workspace, self.B * det.nu * det.nv), dev)
        self.vb_ws = [ops._ws(ops.gs_voxelize_backward_workspace(grid, gs.n, gs.channels), dev)
                      for gs in [ref] + self.mbc]
        self._vox_bwd_launches = sum(vox_bwd_launches(grid, gs) for gs in [ref] + self.mbc)
        if self.eq14 is not None:
            q = self.eq14
            self.ssim_ws = ops._ws(ops._size(Lb.projection_dssim_workspace, self.B, det.nu, det.nv), dev)
            self.tv_ws = ops._ws(ops._size(Lb.tv_loss_workspace, int(q["tv_size"])), dev)
            self.norm_ws = ops._ws(ops._size(Lb.mbc_normality_workspace, L), dev)
            self.tv_origin = torch.zeros(3, dtype=torch.int32, device=dev)

    @property
    def launches_per_step(self) -> int:
        k = KERNELS
        n = ((1 + self.L) * k["gs_voxelize"] + self._vox_bwd_launches + k["warp_combine"]
             + k["conebeam_project"] + k["projection_loss"] + k["conebeam_project_backward"]
             + k["warp_combine_backward"])
        if self.eq14 is not None:
            n += k["projection_dssim"] + k["tv_loss"] + k["mbc_normality"]
        return n

    def run(self, views: torch.Tensor, coeff: torch.Tensor, meas: torch.Tensor,
            tv_origin: Optional[torch.Tensor] = None):
        """views [B,12] f64, coeff [B,L,3] f32, meas [B,nv,nu] f32 (device);
        tv_origin (Eq. 14 only): device int32 [3], the TV crop's corner voxel
        (x, y, z) for this step.  Returns the loss (device [1]); gradients land
        in g_ref, g_mbc, g_wc."""
        g, det = self.grid, self.det
        main = torch.cuda.current_stream()
        side = self._side_streams()
        # the Gaussian sets are independent: each MBC level voxelizes on its own
        # stream while the reference set voxelizes on the caller's (their
        # workspaces are separate), joined before the warp
        for st in side:
            st.wait_stream(main)
        for l, m in enumerate(self.mbc):
            with torch.cuda.stream(side[l] if side else main):
                ops.gs_voxelize(g, m, out=self.E[l], ws=self.vox_ws[1 + l])
        ops.gs_voxelize(g, self.ref, out=self.V, ws=self.vox_ws[0])
        for st in side:
            main.wait_stream(st)
        ops.warp_combine(g, self.V[0], self.E, coeff, out=self.W)
        ops.conebeam_project(g, det, views, self.W, shared=False, out=self.Y)
        loss, dY = ops.projection_loss(self.kind, self.Y, meas, ws=self.loss_ws)
        q = self.eq14
        if q is not None:
            ops.projection_dssim(self.Y, meas, q["data_range"], weight=q["lambda_ssim"], loss=loss, d_pred=dY,
                                 accumulate=True, ws=self.ssim_ws)
        ops.conebeam_project_backward(g, det, views, dY, shared=False, out=self.dW, ws=self.bp_ws, absmax=self.dW_max)
        ops.warp_combine_backward(g, self.V[0], self.E, coeff, self.dW, grads=self.g_wc, ws=self.wc_ws,
                                  d_out_absmax=self.dW_max)
        if q is not None:
            if tv_origin is not None and tv_origin.data_ptr() != self.tv_origin.data_ptr():
                self.tv_origin.copy_(tv_origin, non_blocking=True)
            ops.tv_loss(g, self.V[0], int(q["tv_size"]), self.tv_origin, weight=q["lambda_tv"], loss=loss,
                        d_vol=self.g_wc[0], accumulate=True, ws=self.tv_ws)
            ops.mbc_normality(g, self.E, weight=q["lambda_mbc"], loss=loss, d_mbc=self.g_wc[1], accumulate=True,
                              ws=self.norm_ws)
        # the voxelizer adjoints of the sets are latency-bound at low occupancy:
        # run them side by side, as in the forward
        for st in side:
            st.wait_stream(main)
        for l, m in enumerate(self.mbc):
            with torch.cuda.stream(side[l] if side else main):
                ops.gs_voxelize_backward(g, m, self.g_wc[1][l], grads=self.g_mbc[l], ws=self.vb_ws[1 + l])
        ops.gs_voxelize_backward(g, self.ref, self.g_wc[0].reshape((1,) + self.g_wc[0].shape), grads=self.g_ref,
                                 ws=self.vb_ws[0])
        for st in side:
            main.wait_stream(st)
        return loss

    def _side_streams(self):
        if not self.concurrent_sets:
            return []
        if self._side is None:
            self._side = [torch.cuda.Stream(device=self.ref.mean.device) for _ in self.mbc]
        return self._side


class PlainPerProjection(ForwardAdjoint):
    """The same forward + adjoint, one projection per call and unfused (the DVF
    is written and read back; the paper's projector also runs one view per
    call, Sec. 4).  Used as the per-projection baseline for the batched path."""

    def __init__(self, *args, **kwargs):
        super().__init__(*args, **kwargs)
        shape, n = ops._shape(self.grid)
        dev = self.ref.mean.device
        if self.w_dtype != self.dtype:  # warp_volume writes W in the grids' dtype
            self.w_dtype = self.dtype
            self.W = torch.empty(self.W.shape, dtype=self.dtype, device=dev)
        Lb = ops._lib.load()
        g = ops._grid(self.grid)
        self.D1 = torch.empty((1, 3) + shape, dtype=self.dtype, device=dev)
        self.dD1 = torch.empty((1, 3) + shape, dtype=torch.float32, device=dev)
        self.bp1_ws = ops._ws(ops._size(Lb.conebeam_project_backward_workspace, ops.ct.byref(g), 1, n), dev)
        self.wb1_ws = ops._ws(ops._size(Lb.warp_volume_backward_workspace, ops.ct.byref(g), 1), dev)
        self.cb1_ws = ops._ws(ops._size(Lb.mbc_combine_backward_workspace, ops.ct.byref(g), self.L, 1), dev)

    @property
    def launches_per_step(self) -> int:
        k = KERNELS
        per_view = 1 + 1 + 1 + 3 + 3 + 4  # combine, warp, project, project_bwd, warp_bwd, combine_bwd
        return (1 + self.L) * k["gs_voxelize"] + self._vox_bwd_launches + k["projection_loss"] + self.B * per_view

    def run(self, views: torch.Tensor, coeff: torch.Tensor, meas: torch.Tensor):
        g, det = self.grid, self.det
        ops.gs_voxelize(g, self.ref, out=self.V, ws=self.vox_ws[0])
        for l, m in enumerate(self.mbc):
            ops.gs_voxelize(g, m, out=self.E[l], ws=self.vox_ws[1 + l])
        for p in range(self.B):
            ops.mbc_combine(g, self.E, coeff[p:p + 1], out=self.D1)
            ops.warp_volume(g, self.V[0], self.D1, out=self.W[p:p + 1])
            ops.conebeam_project(g, det, views[p:p + 1], self.W[p:p + 1], shared=False, out=self.Y[p:p + 1])
        loss, dY = ops.projection_loss(self.kind, self.Y, meas, ws=self.loss_ws)
        gV, gE, gw = self.g_wc
        gw.zero_()  # each view's coefficient slot is written once, by accumulating into zero
        for p in range(self.B):
            ops.conebeam_project_backward(g, det, views[p:p + 1], dY[p:p + 1], shared=False,
                                          out=self.dW[p:p + 1], ws=self.bp1_ws)
            ops.mbc_combine(g, self.E, coeff[p:p + 1], out=self.D1)
            self.dD1.zero_()
            ops.warp_volume_backward(g, self.V[0], self.D1, self.dW[p:p + 1], accumulate=p > 0,
                                     grads=(gV, self.dD1), ws=self.wb1_ws)
            ops.mbc_combine_backward(g, self.E, coeff[p:p + 1], self.dD1, accumulate=p > 0,
                                     grads=(gE, gw[p:p + 1]), ws=self.cb1_ws)
        ops.gs_voxelize_backward(g, self.ref, gV.reshape((1,) + gV.shape), grads=self.g_ref, ws=self.vb_ws[0])
        for l, m in enumerate(self.mbc):
            ops.gs_voxelize_backward(g, m, gE[l], grads=self.g_mbc[l], ws=self.vb_ws[1 + l])
        return loss


class GraphedStep:
    """A ForwardAdjoint step captured once into a CUDA graph and replayed.
    Every call into the library only enqueues kernels and memsets on the
    current stream, so the whole step (all stages, both directions) is one
    graph launch; each replay reads the batch from static input buffers."""

    def __init__(self, step: ForwardAdjoint, views: torch.Tensor, coeff: torch.Tensor, meas: torch.Tensor,
                 warmup: int = 2):
        self.step = step
        self.views, self.coeff, self.meas = views.clone(), coeff.clone(), meas.clone()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                step.run(self.views, self.coeff, self.meas)
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.loss = step.run(self.views, self.coeff, self.meas)

    @property
    def launches_per_step(self) -> int:
        return self.step.launches_per_step

    def run(self, views: torch.Tensor, coeff: torch.Tensor, meas: torch.Tensor):
        if views.data_ptr() != self.views.data_ptr():
            self.views.copy_(views, non_blocking=True)
            self.coeff.copy_(coeff, non_blocking=True)
            self.meas.copy_(meas, non_blocking=True)
        self.graph.replay()
        return self.loss


class Stage1Step:
    """Stage 1 of Sec. 2.3.2 (Eq. 10-11): the reference Gaussians rasterized into
    B views by Gaussian splatting (Eq. 8-9), L1 + lambda_ssim D-SSIM against the
    measured projections, and lambda_tv TV of a D^3 sub-volume voxelized from the
    same Gaussians (the crop moves every step); gradients of both terms to every
    Gaussian parameter land in `grads` (mean, scale, quat, value).

    The sub-volume is voxelized on a D^3 grid of the volume's voxel size with the
    means shifted by the crop's centre (the grids are centred on the isocentre),
    so a crop with corner voxel o has centre (o + D/2 - n/2) v."""

    def __init__(self, grid, det, ref: Gaussians, batch: int, data_range: float, lambda_ssim: float = 0.25,
                 lambda_tv: float = 0.05, tv_size: int = 32, pair_headroom: float = 1.25):
        if ref.channels != 1:
            raise ValueError("Stage 1 renders the one-channel reference set")
        self.grid, self.det, self.ref, self.B = grid, det, ref, int(batch)
        self.data_range, self.lambda_ssim, self.lambda_tv, self.D = float(data_range), float(lambda_ssim), \
            float(lambda_tv), int(tv_size)
        self.headroom = float(pair_headroom)
        dev = ref.mean.device
        g = ops._grid(grid)
        self.crop = (self.D, self.D, self.D, float(g.vx), float(g.vy), float(g.vz))
        d = ops._det(det)
        n = ref.n
        self.Y = torch.empty((self.B, d.nv, d.nu), dtype=torch.float32, device=dev)
        self.grads = (torch.empty((n, 3), device=dev), torch.empty((n, 3), device=dev),
                      torch.empty((n, 4), device=dev), torch.empty((n, 1), device=dev))
        self.rws = None  # sized at the first step, from the first batch's pair count
        self.shifted = torch.empty_like(ref.mean)
        self.crop_gs = Gaussians(self.shifted, ref.scale, ref.quat, ref.value, ref.kappa)
        self.Vc = torch.empty((1, self.D, self.D, self.D), dtype=torch.float32, device=dev)
        self.dVc = torch.empty((1, self.D, self.D, self.D), dtype=torch.float32, device=dev)
        self.tv = torch.zeros(1, dtype=torch.float32, device=dev)
        self.origin = torch.zeros(3, dtype=torch.int32, device=dev)
        # a D^3 crop has (D/8)^3 voxelizer tiles: at most that many per Gaussian
        tiles = -(-self.D // 8) ** 3
        self.cvox_ws = ops._ws(ops.gs_voxelize_workspace(self.crop, n, n * tiles), dev)
        self.cvb_ws = ops._ws(ops.gs_voxelize_backward_workspace(self.crop, n, 1), dev)
        self._crop_vox_bwd_launches = 1 + (ops.gs_voxelize_backward_workspace(self.crop, n, 1) > 0)
        Lb = ops._lib.load()
        self.loss_ws = ops._ws(ops._size(Lb.projection_loss_workspace, self.B * d.nu * d.nv), dev)
        self.ssim_ws = ops._ws(ops._size(Lb.projection_dssim_workspace, self.B, d.nu, d.nv), dev)
        self.tv_ws = ops._ws(ops._size(Lb.tv_loss_workspace, self.D), dev)

    @staticmethod
    def crop_centre(grid, corner, D: int = 32) -> torch.Tensor:
        """Centre (mm, host float32 [3]) of the D^3 crop whose lowest voxel is corner (x, y, z)."""
        g = ops._grid(grid)
        n = (g.nx, g.ny, g.nz)
        v = (g.vx, g.vy, g.vz)
        return torch.tensor([(corner[k] + D / 2 - n[k] / 2) * v[k] for k in range(3)], dtype=torch.float32)

    @property
    def launches_per_step(self) -> int:
        k = KERNELS
        return (k["gs_rasterize"] + k["projection_loss"] + k["projection_dssim"] + k["gs_rasterize_backward"]
                + k["pmf_shift_means"] + k["gs_voxelize"] + k["tv_loss"] + self._crop_vox_bwd_launches)

    def run(self, views: torch.Tensor, meas: torch.Tensor, centre: torch.Tensor):
        """views [B,12] f64, meas [B,nv,nu] f32, centre: device f32 [3], the TV
        crop's centre (mm).  Returns (projection loss [1], TV loss [1]), device."""
        det, ref = self.det, self.ref
        if self.rws is None:
            cap = int(ops.gs_rasterize_count(det, views, ref) * self.headroom) + 4096
            self.rws = ops._ws(ops.gs_rasterize_workspace(det, self.B, ref.n, cap), ref.mean.device)
        ops.gs_rasterize(det, views, ref, out=self.Y, ws=self.rws)
        loss, dY = ops.projection_loss(1, self.Y, meas, ws=self.loss_ws)
        ops.projection_dssim(self.Y, meas, self.data_range, weight=self.lambda_ssim, loss=loss, d_pred=dY,
                             accumulate=True, ws=self.ssim_ws)
        ops.gs_rasterize_backward(det, views, ref, dY, grads=self.grads, ws=self.rws)
        ops.pmf_shift_means(ref.mean, centre, out=self.shifted)
        ops.gs_voxelize(self.crop, self.crop_gs, out=self.Vc, ws=self.cvox_ws)
        ops.tv_loss(self.crop, self.Vc[0], self.D, self.origin, weight=self.lambda_tv, loss=self.tv,
                    d_vol=self.dVc[0], accumulate=False, ws=self.tv_ws)
        ops.gs_voxelize_backward(self.crop, self.crop_gs, self.dVc, grads=self.grads, accumulate=True,
                                 ws=self.cvb_ws)
        return loss, self.tv


class GraphedStage1:
    """A Stage1Step captured once into a CUDA graph and replayed.  Stage 1 runs
    at batch 1 in the paper (5,000 iterations), where the step's two dozen
    launches are short and the host's launch rate, not the GPU, sets the pace;
    one graph launch per step removes that.  Each replay reads the views, the
    measured projections and the crop centre from static device buffers (the
    rasterizer's list capacity is fixed at the warm-up; tiles whose list would
    not fit take the rasterizer's scan-all-Gaussians path, same bits)."""

    def __init__(self, step: Stage1Step, views: torch.Tensor, meas: torch.Tensor, centre: torch.Tensor,
                 warmup: int = 2):
        self.step = step
        self.views, self.meas, self.centre = views.clone(), meas.clone(), centre.clone()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                step.run(self.views, self.meas, self.centre)
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.out = step.run(self.views, self.meas, self.centre)

    @property
    def launches_per_step(self) -> int:
        return self.step.launches_per_step

    @property
    def grads(self):
        return self.step.grads

    def run(self, views: torch.Tensor, meas: torch.Tensor, centre: torch.Tensor):
        for dst, src in ((self.views, views), (self.meas, meas), (self.centre, centre)):
            if src.data_ptr() != dst.data_ptr():
                dst.copy_(src, non_blocking=True)
        self.graph.replay()
        return self.out


# Adaptive density control defaults (Sec. 2.3.2 gives the rule, not the
# numbers): densify the Gaussians whose mean |dL/dmean| since the last control
# is in the top `densify_fraction` of their set; clone those no larger than
# `clone_scale_mm` on their largest axis, split the others (scales / 1.6); remove
# Gaussians whose every value component is below `prune_value`.
CONTROL_DEFAULTS = dict(every=50, densify_fraction=0.02, clone_scale_mm=4.0, prune_value=0.005, split_factor=1.6,
                        seed=2025)


class TwoResolutionSchedule:
    """Stages 2 and 3 of Sec. 2.3.2 as one optimisation loop over fixed
    per-projection motion coefficients: Stage 2 voxelizes on a grid of half the
    resolution (voxel size doubled, the same extent) with batches of 32
    projections, Stage 3 on the full grid with batches of 8; every step is the
    forward + adjoint of `ForwardAdjoint` followed by an Adam update of every
    Gaussian parameter (reference and MBC sets), and every `control["every"]`
    steps the sets pass through adaptive density control (their Adam moments
    restart, the statistic is the mean |dL/dmean| since the last control).
    Batches are consecutive slices of a fixed permutation of the scan."""

    def __init__(self, grid, det, ref: Gaussians, mbc: Sequence[Gaussians], views: torch.Tensor, coeff: torch.Tensor,
                 meas: torch.Tensor, steps=(1000, 1000), batches=(32, 8), kind=1, dtype=torch.bfloat16,
                 lrs=(0.02, 0.005, 0.002, 0.002, 0.01), control: Optional[dict] = None, eq14: Optional[dict] = None):
        g = ops._grid(grid)
        self.grids = ((g.nx // 2, g.ny // 2, g.nz // 2, 2 * g.vx, 2 * g.vy, 2 * g.vz),
                      (g.nx, g.ny, g.nz, g.vx, g.vy, g.vz))
        d = ops._det(det)
        # the march step follows the voxel size (0.5 voxel, Sec. 2.3.3's reading)
        self.dets = (ops.PmfDetector(d.nu, d.nv, 2.0 * d.step_mm), ops.PmfDetector(d.nu, d.nv, d.step_mm))
        self.sets = [ref] + list(mbc)
        self.views, self.coeff, self.meas = views, coeff, meas
        self.steps, self.batches = tuple(int(s) for s in steps), tuple(int(b) for b in batches)
        self.kind, self.dtype, self.lrs, self.eq14 = kind, dtype, lrs, eq14
        self.control = dict(CONTROL_DEFAULTS)
        self.control.update(control or {})
        self.gen = torch.Generator(device=ref.mean.device)
        self.gen.manual_seed(int(self.control["seed"]))
        self.history = []  # (stage, step, loss) per step, device scalars
        self.counts = []   # set sizes after every control

    def _build(self, stage):
        B = self.batches[stage]
        self.step = ForwardAdjoint(self.grids[stage], self.dets[stage], self.sets[0], self.sets[1:], batch=B,
                                   dtype=self.dtype, kind="eq14" if self.eq14 is not None else self.kind,
                                   eq14=self.eq14)
        params, lrs = [], []
        for gs in self.sets:
            params += [gs.mean, gs.scale, gs.quat, gs.value]
            lrs += list(self.lrs[:3]) + [self.lrs[3] if gs.channels == 1 else self.lrs[4]]
        self.opt = ops.Adam(params, lr=lrs)
        self.acc = [torch.zeros(gs.n, dtype=torch.float32, device=gs.mean.device) for gs in self.sets]
        self.since = 0

    def _grads(self):
        return [self.step.g_ref] + list(self.step.g_mbc)

    def _control(self, stage):
        c = self.control
        new = []
        for gs, acc in zip(self.sets, self.acc):
            # the densification threshold leaves the top densify_fraction of the set above it
            # (selected on the device; read back because the control's outputs are sized on the host)
            rank = min(int(float(c["densify_fraction"]) * gs.n), gs.n - 1)
            thr = float(ops.gs_density_threshold(acc, self.since, rank).item()) if gs.n > 0 else 0.0
            noise = torch.randn((gs.n, 2, 3), generator=self.gen, device=gs.mean.device)
            new.append(ops.gs_density_control(gs, acc, self.since, noise, thr, float(c["clone_scale_mm"]),
                                              float(c["prune_value"]), float(c["split_factor"])))
        self.sets = new
        self.counts.append(tuple(gs.n for gs in self.sets))
        self._build(stage)

    def run(self):
        """Runs both stages; returns the list of (stage, step, loss) with losses as floats."""
        P = int(self.views.shape[0])
        for stage in (0, 1):
            self._build(stage)
            B = self.batches[stage]
            nb = max(P // B, 1)
            for k in range(self.steps[stage]):
                s = (k % nb) * B
                loss = self.step.run(self.views[s:s + B], self.coeff[s:s + B], self.meas[s:s + B])
                self.history.append((stage, k, loss.clone()))
                for gl, acc in zip(self._grads(), self.acc):
                    ops.gs_grad_norm_accumulate(gl[0], acc)
                self.since += 1
                self.opt.step([g for gl in self._grads() for g in gl])
                last = k == self.steps[stage] - 1
                if int(self.control["every"]) > 0 and self.since >= int(self.control["every"]) and not last:
                    self._control(stage)
        return [(st, k, float(l.item())) for st, k, l in self.history]
