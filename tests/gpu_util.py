"""Helpers shared by the GPU parity tests: device copies of synthetic inputs and
error metrics against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import torch

import paper_2503_22139_gb300 as pmf


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64) if t.dtype != torch.float64 else t.cpu().numpy()


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def gset(gs, kappa):
    """Device Gaussians from a synth.GaussianSet."""
    return pmf.Gaussians(dev(gs.mean), dev(gs.scale), dev(gs.quat), dev(gs.value), kappa)


def views(v):
    return pmf.views_tensor(v, "cuda")


def pixel_views(views_np, nu, nv, pixels):
    """1x1 views whose single ray is pixel (p, b, a) of the full views: the
    detector centre moves to that pixel's centre, so the oracle can evaluate
    sampled pixels one by one."""
    out = []
    for p, b, a in pixels:
        v = np.array(views_np[p], dtype=np.float64)
        ca, cb = a + 0.5 - nu / 2.0, b + 0.5 - nv / 2.0
        v = v.copy()
        v[3:6] = v[3:6] + ca * v[6:9] + cb * v[9:12]
        out.append(v)
    return np.array(out)


def tie_band(grid, gs, kappa, offset=None, mean=None):
    """The oracle's per-voxel tie mass: pairs whose q lies within the binary32
    error bound of q from kappa^2 (and the number of such pairs)."""
    import oracle
    m = gs.mean if mean is None else mean
    return oracle.voxelize_tie_band(grid, m, gs.scale, gs.quat, gs.value, kappa, 1.0, offset)


def assert_voxels_match(got, ref, amb, tol):
    """Voxelization parity that respects truncation ties: voxels with no pair
    inside the binary32 tie band of q = kappa^2 (amb == 0) must match to
    relative L2 <= tol; voxels with such pairs may differ by at most their
    tie mass (plus rounding).  Returns (fraction of voxels outside the band,
    number of voxels whose difference exceeds the rounding floor, i.e. where a
    tie was decided the other way)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    amb = np.broadcast_to(np.asarray(amb, dtype=np.float64), ref.shape)
    sure = amb == 0
    assert rel_l2(got[sure], ref[sure]) <= tol
    floor = 4 * tol * np.abs(ref).max()
    slack = amb + floor
    assert np.all(np.abs(got - ref)[~sure] <= slack[~sure])
    flipped = int(np.count_nonzero(np.abs(got - ref)[~sure] > floor))
    return float(sure.mean()), flipped
