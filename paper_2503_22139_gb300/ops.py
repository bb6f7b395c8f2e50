"""Python binding of the C ABI (include/pmf.h), one function per entry point
with the same name.  Argument marshalling only: tensors are checked, outputs
and scratch are allocated with torch on the tensors' device, and the call is
enqueued on torch's current CUDA stream.  Every step of the computation runs
in libpmf.so; nothing here falls back to PyTorch math.

Grids are any object with nx, ny, nz, vx, vy, vz (or a 6-tuple); detectors any
object with nu, nv, step_mm (or a 3-tuple).  Views are float64 [P, 12] tensors
(src, detector centre, du, dv) on the device -- the pmf_view layout.
"""
from __future__ import annotations

import ctypes as ct
import math
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import PmfDetector, PmfGaussians, PmfGrid, check

_DT = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}


def _grid(g) -> PmfGrid:
    if hasattr(g, "nx"):
        return PmfGrid(int(g.nx), int(g.ny), int(g.nz), float(g.vx), float(g.vy), float(g.vz))
    nx, ny, nz, vx, vy, vz = g
    return PmfGrid(int(nx), int(ny), int(nz), float(vx), float(vy), float(vz))


def _det(d) -> PmfDetector:
    if hasattr(d, "nu"):
        return PmfDetector(int(d.nu), int(d.nv), float(d.step_mm))
    nu, nv, step = d
    return PmfDetector(int(nu), int(nv), float(step))


def _shape(g):
    gr = _grid(g)
    return (gr.nz, gr.ny, gr.nx), gr.nx * gr.ny * gr.nz


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t: Optional[torch.Tensor]):
    return ct.c_void_p(t.data_ptr()) if t is not None else ct.c_void_p(0)


def _need(t: torch.Tensor, name: str, dtype=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if dtype is None and t.dtype not in _DT:
        raise ValueError(f"{name} must be float32, bfloat16 or float16")
    return t.contiguous()


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _size(fn, *args) -> int:
    n = ct.c_size_t(0)
    check(fn(*args, ct.byref(n)), fn.__name__)
    return int(n.value)


class Gaussians:
    """Device views of a Gaussian set (Eq. 4) kept alive for a call."""

    def __init__(self, mean, scale, quat, value, kappa: float = 3.0):
        self.mean = _need(mean, "mean", torch.float32)
        self.scale = _need(scale, "scale", torch.float32)
        self.quat = _need(quat, "quat", torch.float32)
        v = _need(value, "value", torch.float32)
        self.value = v.reshape(v.shape[0], -1) if v.dim() == 1 else v
        self.n = int(self.mean.shape[0])
        self.channels = int(self.value.shape[1]) if self.value.dim() == 2 else 1
        self.kappa = float(kappa)
        if not (self.mean.shape == (self.n, 3) and self.scale.shape == (self.n, 3) and self.quat.shape == (self.n, 4)
                and self.value.shape[0] == self.n):
            raise ValueError("gaussian arrays must be mean[G,3], scale[G,3], quat[G,4], value[G,C]")

    def c_struct(self) -> PmfGaussians:
        k = self.kappa if math.isfinite(self.kappa) else float("inf")
        return PmfGaussians(self.n, self.channels, k, self.mean.data_ptr(), self.scale.data_ptr(),
                            self.quat.data_ptr(), self.value.data_ptr())


def _gs(*args) -> Gaussians:
    return args[0] if isinstance(args[0], Gaussians) else Gaussians(*args)


# ----------------------------------------------------------- voxelizer

VOXEL_TILES = ((8, 8, 8), (16, 8, 8), (8, 8, 4), (16, 8, 4))  # bin tiles of the voxelizer; the first is the default


def _tile(tile):
    t = tuple(int(x) for x in (tile or VOXEL_TILES[0]))
    return (ct.c_int32 * 3)(*t)


def gs_voxelize_workspace(grid, n: int, pair_capacity: int, tile=None) -> int:
    L = _lib.load()
    return _size(L.gs_voxelize_tiled_workspace, ct.byref(_grid(grid)), int(n), int(pair_capacity), _tile(tile))


def gs_voxelize_count(grid, gs: Gaussians, tile=None) -> int:
    """Exact number of (Gaussian, bin tile) overlaps (synchronizes)."""
    L = _lib.load()
    g = _grid(grid)
    ws = _ws(gs_voxelize_workspace(grid, gs.n, 0, tile), gs.mean.device)
    out = torch.zeros(1, dtype=torch.int64, device=gs.mean.device)
    s = gs.c_struct()
    check(L.gs_voxelize_tiled_count(ct.byref(g), ct.byref(s), _tile(tile), _p(out), _p(ws), ws.numel(), _stream()),
          "gs_voxelize_count")
    return int(out.item())


def gs_voxelize(grid, gs: Gaussians, dtype=torch.float32, pair_capacity: Optional[int] = None,
                out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None, tile=None) -> torch.Tensor:
    """Eq. 5 / signed MBC voxelization -> [C, nz, ny, nx] of `dtype`; tile: the
    bin tile (one of VOXEL_TILES; the default 8^3 calls gs_voxelize itself)."""
    L = _lib.load()
    g = _grid(grid)
    shape, n = _shape(grid)
    dev = gs.mean.device
    if out is None:
        out = torch.empty((gs.channels,) + shape, dtype=dtype, device=dev)
    if ws is None:
        cap = gs_voxelize_count(grid, gs, tile) if pair_capacity is None else int(pair_capacity)
        ws = _ws(gs_voxelize_workspace(grid, gs.n, cap, tile), dev)
    s = gs.c_struct()
    if tile is None:
        check(L.gs_voxelize(ct.byref(g), ct.byref(s), _DT[out.dtype], _p(out), _p(ws), ws.numel(), _stream()),
              "gs_voxelize")
    else:
        check(L.gs_voxelize_tiled(ct.byref(g), ct.byref(s), _DT[out.dtype], _tile(tile), _p(out), _p(ws), ws.numel(),
                                  _stream()), "gs_voxelize_tiled")
    return out


def gs_voxelize_tiled(grid, gs: Gaussians, tile, dtype=torch.float32, **kw) -> torch.Tensor:
    """gs_voxelize with the bin tile chosen (one of VOXEL_TILES)."""
    return gs_voxelize(grid, gs, dtype, tile=tuple(tile), **kw)


def gs_voxelize_tiled_count(grid, gs: Gaussians, tile) -> int:
    """gs_voxelize_count for the bin tile `tile`."""
    return gs_voxelize_count(grid, gs, tuple(tile))


def gs_voxelize_backward_workspace(grid, n: int, channels: int) -> int:
    L = _lib.load()
    return _size(L.gs_voxelize_backward_workspace, ct.byref(_grid(grid)), int(n), int(channels))


def gs_voxelize_backward(grid, gs: Gaussians, d_out: torch.Tensor, grads=None, accumulate: bool = False, ws=None):
    """Adjoint of gs_voxelize -> (d_mean, d_scale, d_quat, d_value), fp32."""
    L = _lib.load()
    g = _grid(grid)
    d_out = _need(d_out, "d_out", torch.float32)
    dev = gs.mean.device
    if grads is None:
        grads = (torch.empty((gs.n, 3), device=dev), torch.empty((gs.n, 3), device=dev),
                 torch.empty((gs.n, 4), device=dev), torch.empty((gs.n, gs.channels), device=dev))
    if ws is None:
        ws = _ws(gs_voxelize_backward_workspace(grid, gs.n, gs.channels), dev)
    s = gs.c_struct()
    check(L.gs_voxelize_backward(ct.byref(g), ct.byref(s), _p(d_out), *[_p(t) for t in grads], int(accumulate),
                                 _p(ws), ws.numel(), _stream()), "gs_voxelize_backward")
    return grads


# -------------------------------------------- adaptive density control

def gs_grad_norm_accumulate(d_mean: torch.Tensor, acc: torch.Tensor) -> torch.Tensor:
    """acc += |d_mean| per Gaussian (in place); returns acc."""
    d_mean = _need(d_mean, "d_mean", torch.float32)
    acc = _need(acc, "acc", torch.float32)
    check(_lib.load().gs_grad_norm_accumulate(int(d_mean.shape[0]), _p(d_mean), _p(acc), _stream()),
          "gs_grad_norm_accumulate")
    return acc


def gs_density_threshold(grad_acc: torch.Tensor, steps: int, rank: int) -> torch.Tensor:
    """Device fp32 scalar: the (rank + 1)-th largest of grad_acc / steps, the
    densification threshold that leaves the `rank` largest statistics above it."""
    grad_acc = _need(grad_acc, "grad_acc", torch.float32)
    out = torch.empty((), dtype=torch.float32, device=grad_acc.device)
    check(_lib.load().gs_density_threshold(int(grad_acc.numel()), _p(grad_acc), float(1.0 / max(int(steps), 1)),
                                           int(rank), _p(out), _stream()), "gs_density_threshold")
    return out


def gs_density_control(gs: Gaussians, grad_acc: torch.Tensor, steps: int, noise: torch.Tensor, grad_threshold: float,
                       scale_threshold: float, value_threshold: float, split_factor: float = 1.6) -> Gaussians:
    """Sec. 2.3.2's adaptive density control: returns the new set (synchronizes
    to read its size); noise: device float32 [n, 2, 3] standard normals."""
    L = _lib.load()
    grad_acc = _need(grad_acc, "grad_acc", torch.float32)
    noise = _need(noise, "noise", torch.float32)
    dev, n, C = gs.mean.device, gs.n, gs.channels
    cap = max(2 * n, 1)
    om, osc = torch.empty((cap, 3), device=dev), torch.empty((cap, 3), device=dev)
    oq, ov = torch.empty((cap, 4), device=dev), torch.empty((cap, C), device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = _ws(_size(L.gs_density_control_workspace, n), dev)
    s = gs.c_struct()
    check(L.gs_density_control(ct.byref(s), _p(grad_acc), float(1.0 / max(int(steps), 1)), _p(noise),
                               float(grad_threshold), float(scale_threshold), float(value_threshold),
                               float(split_factor), _p(om), _p(osc), _p(oq), _p(ov), cap, _p(cnt), _p(ws), ws.numel(),
                               _stream()), "gs_density_control")
    m = int(cnt.item())
    return Gaussians(om[:m].contiguous(), osc[:m].contiguous(), oq[:m].contiguous(), ov[:m].contiguous(), gs.kappa)


# ------------------------------------- Stage-1 X-ray rasterizer (Eq. 8-9)

def pmf_shift_means(mean: torch.Tensor, offset: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """mean [n, 3] - offset (device float32 [3]): Gaussians in the frame of a sub-volume centred at offset."""
    mean = _need(mean, "mean", torch.float32)
    offset = _need(offset, "offset", torch.float32)
    if out is None:
        out = torch.empty_like(mean)
    check(_lib.load().pmf_shift_means(int(mean.shape[0]), _p(mean), _p(offset), _p(out), _stream()),
          "pmf_shift_means")
    return out


def gs_rasterize_workspace(det, P: int, n: int, pair_capacity: int) -> int:
    L = _lib.load()
    return _size(L.gs_rasterize_workspace, ct.byref(_det(det)), int(P), int(n), int(pair_capacity))


def gs_rasterize_count(det, views: torch.Tensor, gs: Gaussians) -> int:
    """Exact number of (Gaussian, 16x16-tile) overlaps over all views (synchronizes)."""
    L = _lib.load()
    views = _need(views, "views", torch.float64)
    P = int(views.shape[0])
    ws = _ws(gs_rasterize_workspace(det, P, gs.n, 0), gs.mean.device)
    out = torch.zeros(1, dtype=torch.int64, device=gs.mean.device)
    s = gs.c_struct()
    check(L.gs_rasterize_count(ct.byref(_det(det)), P, _p(views), ct.byref(s), _p(out), _p(ws), ws.numel(),
                               _stream()), "gs_rasterize_count")
    return int(out.item())


def gs_rasterize(det, views: torch.Tensor, gs: Gaussians, pair_capacity: Optional[int] = None,
                 out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Eq. 9 Gaussian splatting of a one-channel set into P projections -> [P, nv, nu] fp32."""
    L = _lib.load()
    views = _need(views, "views", torch.float64)
    P = int(views.shape[0])
    d = _det(det)
    dev = gs.mean.device
    if out is None:
        out = torch.empty((P, d.nv, d.nu), dtype=torch.float32, device=dev)
    out = _need(out, "out", torch.float32)
    if ws is None:
        cap = gs_rasterize_count(det, views, gs) if pair_capacity is None else int(pair_capacity)
        ws = _ws(gs_rasterize_workspace(det, P, gs.n, cap), dev)
    s = gs.c_struct()
    check(L.gs_rasterize(ct.byref(d), P, _p(views), ct.byref(s), _p(out), _p(ws), ws.numel(), _stream()),
          "gs_rasterize")
    return out


def gs_rasterize_backward(det, views: torch.Tensor, gs: Gaussians, d_proj: torch.Tensor, grads=None,
                          accumulate: bool = False, ws=None):
    """Adjoint of gs_rasterize -> (d_mean, d_scale, d_quat, d_value), fp32."""
    L = _lib.load()
    views = _need(views, "views", torch.float64)
    d_proj = _need(d_proj, "d_proj", torch.float32)
    P = int(views.shape[0])
    dev = gs.mean.device
    if grads is None:
        grads = (torch.empty((gs.n, 3), device=dev), torch.empty((gs.n, 3), device=dev),
                 torch.empty((gs.n, 4), device=dev), torch.empty((gs.n, 1), device=dev))
    if ws is None:
        ws = _ws(gs_rasterize_workspace(det, P, gs.n, 0), dev)
    s = gs.c_struct()
    check(L.gs_rasterize_backward(ct.byref(_det(det)), P, _p(views), ct.byref(s), _p(d_proj),
                                  *[_p(t) for t in grads], int(accumulate), _p(ws), ws.numel(), _stream()),
          "gs_rasterize_backward")
    return grads


# ------------------------------------------------------- combine / warp

def mbc_combine(grid, mbc: torch.Tensor, coeff: torch.Tensor, out=None) -> torch.Tensor:
    L = _lib.load()
    mbc = _need(mbc, "mbc")
    coeff = _need(coeff, "coeff", torch.float32)
    P, Lv = int(coeff.shape[0]), int(coeff.shape[1])
    shape, n = _shape(grid)
    if out is None:
        out = torch.empty((P, 3) + shape, dtype=mbc.dtype, device=mbc.device)
    check(L.mbc_combine(ct.byref(_grid(grid)), Lv, P, _DT[mbc.dtype], _p(mbc), _p(coeff), _p(out), _stream()),
          "mbc_combine")
    return out


def mbc_combine_backward(grid, mbc, coeff, d_dvf, accumulate=False, grads=None, ws=None):
    L = _lib.load()
    mbc = _need(mbc, "mbc")
    coeff = _need(coeff, "coeff", torch.float32)
    d_dvf = _need(d_dvf, "d_dvf", torch.float32)
    P, Lv = int(coeff.shape[0]), int(coeff.shape[1])
    g = _grid(grid)
    if ws is None:
        ws = _ws(_size(L.mbc_combine_backward_workspace, ct.byref(g), Lv, P), mbc.device)
    if grads is None:
        grads = (torch.empty(mbc.shape, dtype=torch.float32, device=mbc.device),
                 torch.empty(coeff.shape, dtype=torch.float32, device=mbc.device))
    check(L.mbc_combine_backward(ct.byref(g), Lv, P, _DT[mbc.dtype], _p(mbc), _p(coeff), _p(d_dvf), _p(grads[0]),
                                 _p(grads[1]), int(accumulate), _p(ws), ws.numel(), _stream()), "mbc_combine_backward")
    return grads


def mbc_combine_backward_noalloc(grid, mbc, coeff, d_dvf, accumulate=False, grads=None):
    """mbc_combine_backward without a workspace: the library's fixed device
    scratch is used instead (P * L <= 128; calls must not overlap on the GPU).
    The output tensors are still allocated here unless `grads` is given."""
    L = _lib.load()
    mbc = _need(mbc, "mbc")
    coeff = _need(coeff, "coeff", torch.float32)
    d_dvf = _need(d_dvf, "d_dvf", torch.float32)
    P, Lv = int(coeff.shape[0]), int(coeff.shape[1])
    if grads is None:
        grads = (torch.empty(mbc.shape, dtype=torch.float32, device=mbc.device),
                 torch.empty(coeff.shape, dtype=torch.float32, device=mbc.device))
    check(L.mbc_combine_backward_noalloc(ct.byref(_grid(grid)), Lv, P, _DT[mbc.dtype], _p(mbc), _p(coeff), _p(d_dvf),
                                         _p(grads[0]), _p(grads[1]), int(accumulate), _stream()),
          "mbc_combine_backward_noalloc")
    return grads


def warp_volume(grid, ref, dvf, out=None) -> torch.Tensor:
    L = _lib.load()
    ref, dvf = _need(ref, "ref"), _need(dvf, "dvf")
    P = int(dvf.shape[0])
    shape, _ = _shape(grid)
    if out is None:
        out = torch.empty((P,) + shape, dtype=ref.dtype, device=ref.device)
    check(L.warp_volume(ct.byref(_grid(grid)), P, _DT[ref.dtype], _p(ref), _p(dvf), _p(out), _stream()), "warp_volume")
    return out


def warp_volume_backward(grid, ref, dvf, d_out, need_dvf=True, accumulate=False, grads=None, ws=None):
    L = _lib.load()
    ref, dvf = _need(ref, "ref"), _need(dvf, "dvf")
    d_out = _need(d_out, "d_out", torch.float32)
    P = int(dvf.shape[0])
    g = _grid(grid)
    if ws is None:
        ws = _ws(_size(L.warp_volume_backward_workspace, ct.byref(g), P), ref.device)
    if grads is None:
        grads = (torch.empty(ref.shape, dtype=torch.float32, device=ref.device),
                 torch.empty(dvf.shape, dtype=torch.float32, device=ref.device) if need_dvf else None)
    check(L.warp_volume_backward(ct.byref(g), P, _DT[ref.dtype], _p(ref), _p(dvf), _p(d_out), _p(grads[0]),
                                 _p(grads[1]), int(accumulate), _p(ws), ws.numel(), _stream()), "warp_volume_backward")
    return grads


def warp_combine(grid, ref, mbc, coeff, out=None) -> torch.Tensor:
    L = _lib.load()
    ref, mbc = _need(ref, "ref"), _need(mbc, "mbc")
    coeff = _need(coeff, "coeff", torch.float32)
    P, Lv = int(coeff.shape[0]), int(coeff.shape[1])
    shape, _ = _shape(grid)
    if out is None:
        out = torch.empty((P,) + shape, dtype=ref.dtype, device=ref.device)
    if out.dtype != ref.dtype:  # fp32 warped volumes from bf16 / fp16 grids
        return warp_combine_mixed(grid, ref, mbc, coeff, out.dtype, out)
    check(L.warp_combine(ct.byref(_grid(grid)), Lv, P, _DT[ref.dtype], _p(ref), _p(mbc), _p(coeff), _p(out),
                         _stream()), "warp_combine")
    return out


def warp_combine_mixed(grid, ref, mbc, coeff, out_dtype=torch.float32, out=None) -> torch.Tensor:
    """warp_combine writing W in out_dtype (the grids' dtype or fp32)."""
    L = _lib.load()
    ref, mbc = _need(ref, "ref"), _need(mbc, "mbc")
    coeff = _need(coeff, "coeff", torch.float32)
    P, Lv = int(coeff.shape[0]), int(coeff.shape[1])
    shape, _ = _shape(grid)
    if out is None:
        out = torch.empty((P,) + shape, dtype=out_dtype, device=ref.device)
    out = _need(out, "out", out_dtype)
    check(L.warp_combine_mixed(ct.byref(_grid(grid)), Lv, P, _DT[ref.dtype], _p(ref), _p(mbc), _p(coeff),
                               _DT[out_dtype], _p(out), _stream()), "warp_combine_mixed")
    return out


def warp_combine_backward_bounded(grid, ref, mbc, coeff, d_out, d_out_absmax, accumulate=False, grads=None, ws=None):
    """warp_combine_backward given max |d_out| (abs bits, device int32 [1])."""
    return warp_combine_backward(grid, ref, mbc, coeff, d_out, accumulate=accumulate, grads=grads, ws=ws,
                                 d_out_absmax=d_out_absmax)


def warp_combine_backward(grid, ref, mbc, coeff, d_out, accumulate=False, grads=None, ws=None, d_out_absmax=None):
    """d_out_absmax (optional, device int32 [1]): max |d_out| as written by
    conebeam_project_backward(..., absmax=...); the call then skips its own
    pass over d_out (warp_combine_backward_bounded)."""
    L = _lib.load()
    ref, mbc = _need(ref, "ref"), _need(mbc, "mbc")
    coeff = _need(coeff, "coeff", torch.float32)
    d_out = _need(d_out, "d_out", torch.float32)
    P, Lv = int(coeff.shape[0]), int(coeff.shape[1])
    g = _grid(grid)
    if ws is None:
        ws = _ws(_size(L.warp_combine_backward_workspace, ct.byref(g), Lv, P), ref.device)
    if grads is None:
        grads = (torch.empty(ref.shape, dtype=torch.float32, device=ref.device),
                 torch.empty(mbc.shape, dtype=torch.float32, device=ref.device),
                 torch.empty(coeff.shape, dtype=torch.float32, device=ref.device))
    if d_out_absmax is not None:
        d_out_absmax = _need(d_out_absmax, "d_out_absmax", torch.int32)
        check(L.warp_combine_backward_bounded(ct.byref(g), Lv, P, _DT[ref.dtype], _p(ref), _p(mbc), _p(coeff),
                                              _p(d_out), _p(d_out_absmax), _p(grads[0]), _p(grads[1]), _p(grads[2]),
                                              int(accumulate), _p(ws), ws.numel(), _stream()),
              "warp_combine_backward_bounded")
        return grads
    check(L.warp_combine_backward(ct.byref(g), Lv, P, _DT[ref.dtype], _p(ref), _p(mbc), _p(coeff), _p(d_out),
                                  _p(grads[0]), _p(grads[1]), _p(grads[2]), int(accumulate), _p(ws), ws.numel(),
                                  _stream()), "warp_combine_backward")
    return grads


# ----------------------------------------------------------- projector

def views_tensor(views, device) -> torch.Tensor:
    """float64 [P, 12] on `device` (the pmf_view layout)."""
    t = torch.as_tensor(views, dtype=torch.float64)
    return t.reshape(-1, 12).contiguous().to(device)


def conebeam_project(grid, det, views: torch.Tensor, vol: torch.Tensor, shared: Optional[bool] = None,
                     out=None) -> torch.Tensor:
    """Eq. 6 ray sums -> [P, nv, nu] fp32.  vol is [nz,ny,nx] (shared by all
    views) or [P,nz,ny,nx]."""
    L = _lib.load()
    vol = _need(vol, "vol")
    views = _need(views, "views", torch.float64)
    P = int(views.shape[0])
    d = _det(det)
    _, n = _shape(grid)
    if shared is None:
        shared = vol.numel() == n
    if out is None:
        out = torch.empty((P, d.nv, d.nu), dtype=torch.float32, device=vol.device)
    check(L.conebeam_project(ct.byref(_grid(grid)), ct.byref(d), P, _p(views), _DT[vol.dtype], _p(vol),
                             0 if shared else n, _p(out), _stream()), "conebeam_project")
    return out


def conebeam_project_backward(grid, det, views, d_proj, shared: bool = False, accumulate=False, out=None,
                              ws=None, absmax=None) -> torch.Tensor:
    """absmax (optional, device int32 [1]): receives max |out| as the bits of
    the float with the sign cleared (conebeam_project_backward_absmax), the
    bound warp_combine_backward(..., d_out_absmax=absmax) takes instead of a
    pass of its own over out."""
    L = _lib.load()
    views = _need(views, "views", torch.float64)
    d_proj = _need(d_proj, "d_proj", torch.float32)
    P = int(views.shape[0])
    d = _det(det)
    g = _grid(grid)
    shape, n = _shape(grid)
    stride = 0 if shared else n
    if ws is None:
        ws = _ws(_size(L.conebeam_project_backward_workspace, ct.byref(g), P, stride), d_proj.device)
    if out is None:
        out = torch.empty(shape if shared else (P,) + shape, dtype=torch.float32, device=d_proj.device)
    if absmax is not None:
        absmax = _need(absmax, "absmax", torch.int32)
        check(L.conebeam_project_backward_absmax(ct.byref(g), ct.byref(d), P, _p(views), _p(d_proj), _p(out), stride,
                                                 int(accumulate), _p(ws), ws.numel(), _p(absmax), _stream()),
              "conebeam_project_backward_absmax")
        return out
    check(L.conebeam_project_backward(ct.byref(g), ct.byref(d), P, _p(views), _p(d_proj), _p(out), stride,
                                      int(accumulate), _p(ws), ws.numel(), _stream()), "conebeam_project_backward")
    return out


def conebeam_project_backward_absmax(grid, det, views, d_proj, absmax, shared: bool = False, accumulate=False,
                                     out=None, ws=None) -> torch.Tensor:
    """conebeam_project_backward that also writes max |out| (abs bits) to
    absmax (device int32 [1])."""
    return conebeam_project_backward(grid, det, views, d_proj, shared=shared, accumulate=accumulate, out=out, ws=ws,
                                     absmax=absmax)


def conebeam_project_batched(items, out=None):
    """One launch over several volumes.  items: sequence of
    (grid, det, views [P,12] f64, vol, shared) tuples; returns the list of
    projections [P, nv, nu] (fp32), or fills `out` (a list of tensors)."""
    L = _lib.load()
    arr = (_lib.PmfProjectItem * max(1, len(items)))()
    outs, keep, dt = [], [], None
    for i, (grid, det, views, vol, shared) in enumerate(items):
        vol = _need(vol, "vol")
        views = _need(views, "views", torch.float64)
        dt = vol.dtype if dt is None else dt
        if vol.dtype != dt:
            raise ValueError("all volumes of a batched launch share one dtype")
        d = _det(det)
        _, n = _shape(grid)
        P = int(views.shape[0])
        o = out[i] if out is not None else torch.empty((P, d.nv, d.nu), dtype=torch.float32, device=vol.device)
        arr[i] = _lib.PmfProjectItem(_grid(grid), d, P, views.data_ptr(), vol.data_ptr(), 0 if shared else n,
                                     o.data_ptr())
        outs.append(o)
        keep += [vol, views]
    check(L.conebeam_project_batched(len(items), arr, _DT[dt or torch.float32], _stream()),
          "conebeam_project_batched")
    return outs


def conebeam_project_backward_batched(items, accumulate=False, out=None, ws=None):
    """items: sequence of (grid, det, views [P,12] f64, d_proj [P,nv,nu], shared);
    returns the list of volume gradients."""
    L = _lib.load()
    arr = (_lib.PmfBackprojectItem * max(1, len(items)))()
    outs, keep, dev = [], [], None
    for i, (grid, det, views, d_proj, shared) in enumerate(items):
        views = _need(views, "views", torch.float64)
        d_proj = _need(d_proj, "d_proj", torch.float32)
        dev = d_proj.device
        d = _det(det)
        shape, n = _shape(grid)
        P = int(views.shape[0])
        o = out[i] if out is not None else torch.empty(shape if shared else (P,) + shape, dtype=torch.float32,
                                                         device=dev)
        arr[i] = _lib.PmfBackprojectItem(_grid(grid), d, P, views.data_ptr(), d_proj.data_ptr(), o.data_ptr(),
                                         0 if shared else n)
        outs.append(o)
        keep += [views, d_proj]
    if ws is None:
        nb = ct.c_size_t(0)
        check(L.conebeam_project_backward_batched_workspace(len(items), arr, ct.byref(nb)),
              "conebeam_project_backward_batched_workspace")
        ws = _ws(nb.value, dev if dev is not None else "cuda")
    check(L.conebeam_project_backward_batched(len(items), arr, int(accumulate), _p(ws), ws.numel(), _stream()),
          "conebeam_project_backward_batched")
    return outs


def projection_loss(kind: int, pred: torch.Tensor, meas: torch.Tensor, with_grad: bool = True, ws=None):
    """kind 1 = L1 (Eq. 10/12), 2 = L2 (Eq. 1); mean over all pixels -> (loss[1], d_pred)."""
    L = _lib.load()
    pred = _need(pred, "pred", torch.float32)
    meas = _need(meas, "meas", torch.float32)
    if pred.shape != meas.shape:
        raise ValueError("pred and meas shapes differ")
    P = int(pred.shape[0])
    Q = pred.numel() // max(P, 1)
    if ws is None:
        ws = _ws(_size(L.projection_loss_workspace, P * Q), pred.device)
    loss = torch.empty(1, dtype=torch.float32, device=pred.device)
    d_pred = torch.empty_like(pred) if with_grad else None
    check(L.projection_loss(int(kind), P, Q, _p(pred), _p(meas), _p(loss), _p(d_pred), _p(ws), ws.numel(),
                            _stream()), "projection_loss")
    return loss, d_pred


# ------------------------------------------------- Eq. 14 regularisation

def projection_dssim(pred: torch.Tensor, meas: torch.Tensor, data_range: float, weight: float = 1.0,
                     with_grad: bool = True, loss: Optional[torch.Tensor] = None, d_pred: Optional[torch.Tensor] = None,
                     accumulate: bool = False, ws=None):
    """D-SSIM term of Eq. 10/12 of projections [P, nv, nu]; returns (loss [1], d_pred or None)."""
    L = _lib.load()
    pred = _need(pred, "pred", torch.float32)
    meas = _need(meas, "meas", torch.float32)
    P, nv, nu = (int(x) for x in pred.shape)
    if ws is None:
        ws = _ws(_size(L.projection_dssim_workspace, P, nu, nv), pred.device)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=pred.device)
    if with_grad and d_pred is None:
        d_pred = torch.zeros_like(pred)
    check(L.projection_dssim(P, nu, nv, _p(pred), _p(meas), float(data_range), float(weight), _p(loss),
                             _p(d_pred if with_grad else None), int(accumulate), _p(ws), ws.numel(), _stream()),
          "projection_dssim")
    return loss, (d_pred if with_grad else None)


def tv_loss(grid, vol: torch.Tensor, D: int, origin, weight: float = 1.0, with_grad: bool = True,
            loss: Optional[torch.Tensor] = None, d_vol: Optional[torch.Tensor] = None, accumulate: bool = False,
            ws=None):
    """Sub-volume TV (Eq. 11/14) of vol [nz, ny, nx] on the D^3 crop at voxel
    origin (x, y, z) (a device int32 [3] tensor or a tuple); returns (loss [1], d_vol or None)."""
    L = _lib.load()
    vol = _need(vol, "vol")
    g = _grid(grid)
    if not isinstance(origin, torch.Tensor):
        origin = torch.tensor(list(origin), dtype=torch.int32, device=vol.device)
    origin = _need(origin, "origin", torch.int32)
    if ws is None:
        ws = _ws(_size(L.tv_loss_workspace, int(D)), vol.device)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=vol.device)
    if with_grad and d_vol is None:
        d_vol = torch.zeros(vol.shape, dtype=torch.float32, device=vol.device)
    check(L.tv_loss(ct.byref(g), _DT[vol.dtype], _p(vol), int(D), _p(origin), float(weight), _p(loss),
                    _p(d_vol if with_grad else None), int(accumulate), _p(ws), ws.numel(), _stream()), "tv_loss")
    return loss, (d_vol if with_grad else None)


def mbc_normality(grid, mbc: torch.Tensor, weight: float = 1.0, with_grad: bool = True,
                  loss: Optional[torch.Tensor] = None, d_mbc: Optional[torch.Tensor] = None, accumulate: bool = False,
                  ws=None):
    """Eq. 13 normality loss of MBC grids [L, 3, nz, ny, nx]; returns (loss [1], d_mbc or None)."""
    Lb = _lib.load()
    mbc = _need(mbc, "mbc")
    g = _grid(grid)
    L = int(mbc.shape[0])
    if ws is None:
        ws = _ws(_size(Lb.mbc_normality_workspace, L), mbc.device)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=mbc.device)
    if with_grad and d_mbc is None:
        d_mbc = torch.zeros(mbc.shape, dtype=torch.float32, device=mbc.device)
    check(Lb.mbc_normality(ct.byref(g), L, _DT[mbc.dtype], _p(mbc), float(weight), _p(loss),
                           _p(d_mbc if with_grad else None), int(accumulate), _p(ws), ws.numel(), _stream()),
          "mbc_normality")
    return loss, (d_mbc if with_grad else None)


# ------------------------------------------------------------ optimiser

def pmf_adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float,
                  t: int, betas=(0.9, 0.999), eps: float = 1e-8) -> None:
    """One in-place Adam update of a contiguous fp32 device tensor (step t >= 1)."""
    for name, x in (("param", param), ("grad", grad), ("m", m), ("v", v)):
        _need(x, name, torch.float32)
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if not (param.shape == grad.shape == m.shape == v.shape):
        raise ValueError("param, grad, m and v must have one shape")
    check(_lib.load().pmf_adam_step(param.numel(), _p(param), _p(grad), _p(m), _p(v), float(lr), float(betas[0]),
                                    float(betas[1]), float(eps), int(t), _stream()), "pmf_adam_step")


adam_step = pmf_adam_step


class Adam:
    """Adam state for a list of parameter tensors (lr: one rate, or one per
    tensor); step(grads) updates them in place."""

    def __init__(self, params: Sequence[torch.Tensor], lr=1e-3, betas=(0.9, 0.999), eps: float = 1e-8):
        self.params = list(params)
        self.lrs = [float(x) for x in lr] if isinstance(lr, (list, tuple)) else [float(lr)] * len(self.params)
        if len(self.lrs) != len(self.params):
            raise ValueError("one learning rate per parameter tensor")
        self.betas, self.eps, self.t = betas, float(eps), 0
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]

    def step(self, grads: Sequence[torch.Tensor]) -> None:
        self.t += 1
        for p, g, m, v, lr in zip(self.params, grads, self.m, self.v, self.lrs):
            pmf_adam_step(p, g, m, v, lr, self.t, self.betas, self.eps)


def library_info() -> dict:
    L = _lib.load()
    return {"version": L.pmf_version().decode(), "path": _lib.library_path()}


# ---------------------------------------------------------- host helpers

def pmf_circular_views(P: int, sad_mm: float, sdd_mm: float, du_mm: float, dv_mm: float, nu: int,
                       nv: int) -> torch.Tensor:
    """The circular scan (Sec. 2.3.3) as a host float64 [P, 12] tensor of pmf_view records."""
    arr = (_lib.PmfView * max(int(P), 1))()
    check(_lib.load().pmf_circular_views(int(P), float(sad_mm), float(sdd_mm), float(du_mm), float(dv_mm), int(nu),
                                         int(nv), arr), "pmf_circular_views")
    out = torch.empty((int(P), 12), dtype=torch.float64)
    for p in range(int(P)):
        v = arr[p]
        out[p] = torch.tensor(list(v.src) + list(v.det) + list(v.du) + list(v.dv), dtype=torch.float64)
    return out


circular_views = pmf_circular_views


def pmf_workspace_size(op, grid, n: int = 0, pair_capacity: int = 0, vol_stride: int = 0, count: int = 0,
                       channels: int = 0, L: int = 0, P: int = 0) -> int:
    """Scratch bytes of one operation (op: a pmf_op code or its name, e.g. "project_backward")."""
    code = _lib.PMF_OPS[op] if isinstance(op, str) else int(op)
    a = _lib.PmfWsArgs(_grid(grid), int(n), int(pair_capacity), int(vol_stride), int(count), int(channels), int(L),
                       int(P))
    nb = ct.c_size_t(0)
    check(_lib.load().pmf_workspace_size(code, ct.byref(a), ct.byref(nb)), "pmf_workspace_size")
    return int(nb.value)


workspace_size = pmf_workspace_size


def pmf_device_counters(reset: bool = False) -> dict:
    """The current device's diagnostic counters (pmf_diag) by name; synchronizes."""
    buf = (ct.c_uint64 * _lib.PMF_DIAG_COUNT)()
    check(_lib.load().pmf_device_counters(buf, 1 if reset else 0), "pmf_device_counters")
    return {name: int(buf[i]) for i, name in enumerate(_lib.DIAG_NAMES)}


device_counters = pmf_device_counters


def pmf_device_status() -> None:
    """Synchronizes torch's current stream; raises PmfError if its work failed
    or a non-finite input reached a fixed-point scatter."""
    check(_lib.load().pmf_device_status(_stream()), "pmf_device_status")


device_status = pmf_device_status


def pmf_debug_stall_bulk_copies(on: bool) -> None:
    """Test hook: while on, the per-volume bulk-copy projector arms its
    mbarrier without issuing copies, so its bounded wait runs out (see pmf.h)."""
    check(_lib.load().pmf_debug_stall_bulk_copies(1 if on else 0), "pmf_debug_stall_bulk_copies")


# ----------------------------------------------------- training-step plan

class _DevArray:
    """__cuda_array_interface__ view of a plan-owned device buffer."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


_TYPESTR = {torch.float32: "<f4", torch.float16: "<f2"}


class _StepBuffers:
    """The caller-side buffers of a pmf_batch_desc (batch inputs, loss,
    gradients) and the descriptor that points at them."""

    def __init__(self, grid, det, ref: Gaussians, mbc: Sequence[Gaussians], batch: int,
                 dtype: torch.dtype = torch.bfloat16, kind=2, eq14: Optional[dict] = None,
                 w_dtype: torch.dtype = torch.float32):
        if len(mbc) < 1 or len(mbc) > _lib.PMF_MAX_LEVELS:
            raise ValueError(f"need 1..{_lib.PMF_MAX_LEVELS} MBC levels")
        if w_dtype not in (dtype, torch.float32):
            raise ValueError("w_dtype must be dtype or torch.float32")
        self.grid, self.det, self.ref, self.mbc = grid, det, ref, list(mbc)
        self.B, self.L, self.dtype, self.w_dtype = int(batch), len(self.mbc), dtype, w_dtype
        dev = ref.mean.device
        self.eq14 = None
        if kind in ("eq14", 3):
            from .pipeline import EQ14_DEFAULTS
            q = dict(EQ14_DEFAULTS)
            q.update(eq14 or {})
            if q["data_range"] is None:
                raise ValueError("eq14 needs data_range (the projections' dynamic range)")
            self.eq14 = q
            kind = 3
        self.kind = int(kind)
        self.tv_origin = torch.zeros(3, dtype=torch.int32, device=dev)
        gr = _det(det)
        self.views = torch.zeros((self.B, 12), dtype=torch.float64, device=dev)
        self.coeff = torch.zeros((self.B, self.L, 3), dtype=torch.float32, device=dev)
        self.meas = torch.zeros((self.B, gr.nv, gr.nu), dtype=torch.float32, device=dev)
        # the step's outputs (every set's gradients, the coefficient gradient and
        # the loss) as views of one fp32 allocation, each at a 256-byte
        # boundary: a caller moves all of them with one copy of grads_flat
        shapes = []
        for gs in [ref] + list(self.mbc):
            shapes += [(gs.n, 3), (gs.n, 3), (gs.n, 4), (gs.n, gs.channels)]
        shapes += [(self.B, self.L, 3), (1,)]
        offs, total = [], 0
        for shp in shapes:
            offs.append(total)
            total += (math.prod(shp) + 63) // 64 * 64
        self.grads_flat = torch.zeros(total, dtype=torch.float32, device=dev)
        views = [self.grads_flat[o:o + math.prod(shp)].view(shp) for o, shp in zip(offs, shapes)]
        self.g_ref = tuple(views[0:4])
        self.g_mbc = [tuple(views[4 + 4 * l:8 + 4 * l]) for l in range(len(self.mbc))]
        self.d_coeff, self.loss = views[-2], views[-1]

    def set_batch(self, views=None, coeff=None, meas=None, tv_origin=None) -> None:
        for dst, src in ((self.views, views), (self.coeff, coeff), (self.meas, meas)):
            if src is not None:
                dst.copy_(src.reshape(dst.shape), non_blocking=True)
        if tv_origin is not None:
            if not isinstance(tv_origin, torch.Tensor):
                tv_origin = torch.tensor(list(tv_origin), dtype=torch.int32)
            self.tv_origin.copy_(tv_origin.to(torch.int32), non_blocking=True)

    def desc(self, use_graph: bool = False, tune_cache: Optional[bytes] = None) -> "_lib.PmfBatchDesc":
        d = _lib.PmfBatchDesc()
        d.grid, d.det, d.dtype, d.w_dtype = _grid(self.grid), _det(self.det), _DT[self.dtype], _DT[self.w_dtype]
        d.batch, d.loss_kind, d.levels = self.B, self.kind, self.L
        d.ref = self.ref.c_struct()
        for l, m in enumerate(self.mbc):
            d.mbc[l] = m.c_struct()
            for k in range(4):
                d.d_mbc[l][k] = self.g_mbc[l][k].data_ptr()
        for k in range(4):
            d.d_ref[k] = self.g_ref[k].data_ptr()
        d.views, d.coeff, d.meas = self.views.data_ptr(), self.coeff.data_ptr(), self.meas.data_ptr()
        d.loss, d.d_coeff = self.loss.data_ptr(), self.d_coeff.data_ptr()
        d.use_graph = 1 if use_graph else 0
        d.tune_cache = tune_cache
        if self.eq14 is not None:
            q = self.eq14
            d.lambda_ssim, d.lambda_mbc, d.lambda_tv = float(q["lambda_ssim"]), float(q["lambda_mbc"]), float(q["lambda_tv"])
            d.ssim_range, d.tv_size = float(q["data_range"]), int(q["tv_size"])
        d.tv_origin = self.tv_origin.data_ptr()
        return d


class Plan(_StepBuffers):
    """pmf_plan: one native forward + adjoint step over a batch of B views.

    The caller-side buffers (batch inputs, loss, gradients) are allocated here
    and handed to the plan once; `step()` copies a new batch into them (if
    given) and enqueues the step.  With use_graph the step is captured into a
    CUDA graph on the plan's own stream the first time and replayed after."""

    def __init__(self, grid, det, ref: Gaussians, mbc: Sequence[Gaussians], batch: int,
                 dtype: torch.dtype = torch.bfloat16, kind=2, use_graph: bool = False,
                 tune_cache: Optional[str] = None, eq14: Optional[dict] = None,
                 w_dtype: torch.dtype = torch.float32):
        """kind 1 / 2: L1 / L2 loss; "eq14" (or 3): the objective of Eq. 14 with
        `eq14` overriding pipeline.EQ14_DEFAULTS (data_range required).
        w_dtype: storage of the warped volumes W (fp32, or dtype)."""
        self._h = None
        super().__init__(grid, det, ref, mbc, batch, dtype, kind, eq14, w_dtype)
        dev = ref.mean.device
        self._cache = tune_cache.encode() if tune_cache else None  # kept alive with the descriptor
        self._desc = self.desc(use_graph, self._cache)
        self._stream = torch.cuda.Stream(device=dev) if use_graph else None
        h = ct.c_void_p(0)
        with torch.cuda.device(dev):
            check(_lib.load().pmf_plan_create(ct.byref(self._desc), ct.byref(h)), "pmf_plan_create")
        self._h = h

    def step(self, views: Optional[torch.Tensor] = None, coeff: Optional[torch.Tensor] = None,
             meas: Optional[torch.Tensor] = None, tv_origin=None) -> torch.Tensor:
        """Copies the batch (when given; tv_origin: the Eq. 14 TV crop corner)
        into the plan's inputs and enqueues one step on torch's current stream;
        returns the device loss [1]."""
        self.set_batch(views, coeff, meas, tv_origin)
        L = _lib.load()
        if self._stream is None:
            check(L.pmf_plan_step(self._h, _stream()), "pmf_plan_step")
        else:
            cur = torch.cuda.current_stream()
            self._stream.wait_stream(cur)
            check(L.pmf_plan_step(self._h, ct.c_void_p(self._stream.cuda_stream)), "pmf_plan_step")
            cur.wait_stream(self._stream)
        return self.loss

    def tensors(self) -> dict:
        """Torch views of the plan's own device tensors (valid until close())."""
        t = _lib.PmfPlanTensors()
        check(_lib.load().pmf_plan_tensors_get(self._h, ct.byref(t)), "pmf_plan_tensors_get")
        shape, n = _shape(self.grid)
        gr = _det(self.det)
        dev = self.ref.mean.device

        def view(ptr, shp, dt):
            if dt == torch.bfloat16:  # no bf16 typestr: view the 16-bit payload and reinterpret
                raw = torch.as_tensor(_DevArray(ptr, shp, "<i2"), device=dev)
                return raw.view(torch.bfloat16)
            return torch.as_tensor(_DevArray(ptr, shp, _TYPESTR[dt]), device=dev)

        return {"V": view(t.V, shape, self.dtype), "E": view(t.E, (self.L, 3) + shape, self.dtype),
                "W": view(t.W, (self.B,) + shape, self.w_dtype),
                "Y": view(t.Y, (self.B, gr.nv, gr.nu), torch.float32),
                "dY": view(t.dY, (self.B, gr.nv, gr.nu), torch.float32),
                "dW": view(t.dW, (self.B,) + shape, torch.float32), "dV": view(t.dV, shape, torch.float32),
                "dE": view(t.dE, (self.L, 3) + shape, torch.float32)}

    def launch_forms(self):
        """((form, chunk, rays) of the projector, (form, chunk, rays) of its adjoint)."""
        a, b = (ct.c_int32 * 3)(), (ct.c_int32 * 3)()
        check(_lib.load().pmf_plan_launch_forms(self._h, a, b), "pmf_plan_launch_forms")
        return tuple(int(x) for x in a), tuple(int(x) for x in b)

    def voxel_tiles(self):
        """The voxelizer bin tile (x, y, z) of each Gaussian set: reference, then the MBC levels."""
        n = 1 + int(self.L)
        t = (ct.c_int32 * (3 * n))()
        check(_lib.load().pmf_plan_voxel_tiles(self._h, t), "pmf_plan_voxel_tiles")
        return [tuple(int(x) for x in t[3 * i:3 * i + 3]) for i in range(n)]

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().pmf_plan_destroy(self._h)
            self._h = ct.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pmf_autotune(grid, det, ref: Gaussians, mbc: Sequence[Gaussians], batch: int, cache_path: str,
                 dtype: torch.dtype = torch.bfloat16, kind: int = 2, views=None, coeff=None, meas=None,
                 w_dtype: torch.dtype = torch.float32) -> None:
    """Times the projector's launch forms on this configuration (and batch, if
    given) and records the fastest in cache_path, which
    Plan(..., tune_cache=cache_path) reads back."""
    buf = _StepBuffers(grid, det, ref, mbc, batch, dtype, kind, None, w_dtype)
    buf.set_batch(views, coeff, meas)
    d = buf.desc(False, None)
    with torch.cuda.device(ref.mean.device):
        check(_lib.load().pmf_autotune(ct.byref(d), str(cache_path).encode()), "pmf_autotune")


autotune = pmf_autotune
