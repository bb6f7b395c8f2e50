"""The whole forward model and its adjoint, composed from oracle stages (test
infrastructure): voxelize (Eq. 4-5) -> combine (Eq. 3) -> warp (Eq. 2) ->
project (Eq. 6) -> loss (Eq. 10/12), then the exact adjoint chain."""
from __future__ import annotations

import numpy as np

import oracle


def forward(wl, views=None, coeff=None, kappa=None, storage=None):
    """storage = (fmt, w_too[, rounder]): V and E (and W when w_too) are rounded
    to the storage format "bf16" or "f16" where the path stores them, so that
    every later stage sees the same rounded values the kernels see; rounder(x)
    replaces round-to-nearest (the tests pass one that rounds the other way
    wherever an fp32 error could)."""
    kappa = wl.kappa if kappa is None else kappa
    views = wl.views if views is None else views
    coeff = wl.coeff if coeff is None else coeff
    if storage is None:
        rnd = lambda a: a  # noqa: E731
    elif len(storage) > 2 and storage[2] is not None:
        rnd = storage[2]
    else:
        rnd = lambda a: oracle.round_storage(a, storage[0])  # noqa: E731
    g = wl.grid
    exact = {}
    exact["V"] = oracle.voxelize(g, wl.ref.mean, wl.ref.scale, wl.ref.quat, wl.ref.value, kappa)[0]
    exact["E"] = np.stack([oracle.voxelize(g, m.mean, m.scale, m.quat, m.value, kappa) for m in wl.mbc])
    V, E = rnd(exact["V"]), rnd(exact["E"])
    D = oracle.combine(E, coeff)
    W = exact["W"] = oracle.warp(g, V, D)
    if storage is not None and storage[1]:
        W = rnd(W)
    Y = oracle.project(g, wl.det.nu, wl.det.nv, wl.det.step_mm, views, W, shared=False)
    out = dict(V=V, E=E, D=D, W=W, Y=Y)
    if storage is not None:  # the values before rounding, for checks of the stored elements
        out.update({k + "_unrounded": v for k, v in exact.items()})
    return out


def step(wl, meas, kind=2, views=None, coeff=None, kappa=None, eq14=None, storage=None):
    """Loss and gradients with respect to every Gaussian parameter and the
    temporal coefficients (float64).  kind 1 / 2: L1 / L2 projection loss;
    kind "eq14": the Stage 2-3 objective of Eq. 14, L1 + lambda_ssim D-SSIM +
    lambda_mbc L_MBC + lambda_tv TV, with eq14 = dict(lambda_ssim, lambda_mbc,
    lambda_tv, data_range, tv_size, tv_origin).  storage: see `forward`."""
    kappa = wl.kappa if kappa is None else kappa
    views = wl.views if views is None else views
    coeff = wl.coeff if coeff is None else coeff
    g = wl.grid
    f = forward(wl, views, coeff, kappa, storage)
    if kind == "eq14":
        q = eq14
        loss, dY = oracle.loss(1, f["Y"], meas)
        ls, dYs = oracle.dssim(f["Y"], meas, q["data_range"])
        loss += q["lambda_ssim"] * ls
        dY = dY + q["lambda_ssim"] * dYs
    else:
        loss, dY = oracle.loss(kind, f["Y"], meas)
    dW = oracle.project_backward(g, wl.det.nu, wl.det.nv, wl.det.step_mm, views, dY, shared=False)
    dV, dD = oracle.warp_backward(g, f["V"], f["D"], dW)
    dE, dw = oracle.combine_backward(f["E"], coeff, dD)
    if kind == "eq14":
        lt, dVt = oracle.tv(f["V"], q["tv_size"], q["tv_origin"])
        ln, dEn = oracle.mbc_normality(f["E"])
        loss += q["lambda_tv"] * lt + q["lambda_mbc"] * ln
        dV = dV + q["lambda_tv"] * dVt
        dE = dE + q["lambda_mbc"] * dEn
    grads = {"coeff": dw, "dV": dV, "dE": dE, "dW": dW, "dY": dY}
    grads["ref"] = oracle.voxelize_backward(g, wl.ref.mean, wl.ref.scale, wl.ref.quat, wl.ref.value, dV, kappa)
    grads["mbc"] = [oracle.voxelize_backward(g, m.mean, m.scale, m.quat, m.value, dE[l], kappa)
                    for l, m in enumerate(wl.mbc)]
    return loss, grads, f
