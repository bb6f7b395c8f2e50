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
