"""ctypes binding of the FP64 C oracle (oracle/pmf_oracle.c).

TEST INFRASTRUCTURE ONLY.  Arrays are converted to contiguous float64 here; the
C code does all of the arithmetic.  Grids are passed as (nx, ny, nz, vx, vy, vz)
tuples or any object with those attributes.
"""
from __future__ import annotations

import ctypes as ct
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

_D = ct.POINTER(ct.c_double)
_I64 = ct.POINTER(ct.c_int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ct.CDLL(path)
            L.orc_threads.restype = ct.c_int
            L.orc_set_threads.argtypes = [ct.c_int]
            L.orc_quat_to_rot.argtypes = [_D, _D]
            L.orc_voxelize.argtypes = [_I64, _D, ct.c_int64, ct.c_int, _D, _D, _D, _D, ct.c_double, ct.c_int, _D]
            L.orc_voxelize.restype = ct.c_int
            L.orc_voxelize_ambiguity.argtypes = [_I64, _D, ct.c_int64, ct.c_int, _D, _D, _D, _D, ct.c_double,
                                                 ct.c_double, _D]
            L.orc_voxelize_ambiguity.restype = ct.c_int
            L.orc_voxelize_tie_band.argtypes = [_I64, _D, ct.c_int64, ct.c_int, _D, _D, _D, _D, ct.c_double,
                                                ct.c_double, _D, _D, _I64]
            L.orc_voxelize_tie_band.restype = ct.c_int
            L.orc_qform_and_bound.argtypes = [_D, _D, _D, _D, ct.c_double, _D]
            L.orc_voxelize_backward.argtypes = [_I64, _D, ct.c_int64, ct.c_int, _D, _D, _D, _D, ct.c_double,
                                                _D, _D, _D, _D, _D]
            L.orc_voxelize_backward.restype = ct.c_int
            L.orc_combine.argtypes = [ct.c_int64, ct.c_int, ct.c_int, _D, _D, _D]
            L.orc_combine_backward.argtypes = [ct.c_int64, ct.c_int, ct.c_int, _D, _D, _D, _D, _D]
            L.orc_warp.argtypes = [_I64, _D, ct.c_int, _D, _D, _D]
            L.orc_warp_backward.argtypes = [_I64, _D, ct.c_int, _D, _D, _D, _D, _D]
            L.orc_project.argtypes = [_I64, _D, ct.c_int, ct.c_int, ct.c_double, ct.c_int, _D, _D, ct.c_int64, _D]
            L.orc_project_backward.argtypes = [_I64, _D, ct.c_int, ct.c_int, ct.c_double, ct.c_int, _D, _D, _D,
                                               ct.c_int64]
            L.orc_project_gaussians.argtypes = [ct.c_int, ct.c_int, ct.c_double, ct.c_int, _D, ct.c_int64,
                                                _D, _D, _D, _D, ct.c_int64, ct.c_int64, _D]
            L.orc_loss.argtypes = [ct.c_int, ct.c_int64, _D, _D, _D]
            L.orc_loss.restype = ct.c_double
            L.orc_dssim.argtypes = [ct.c_int, ct.c_int, ct.c_int, _D, _D, ct.c_double, _D]
            L.orc_dssim.restype = ct.c_double
            L.orc_tv.argtypes = [_I64, _D, ct.c_int, _I64, _D]
            L.orc_tv.restype = ct.c_double
            L.orc_mbc_normality.argtypes = [ct.c_int, ct.c_int64, _D, _D]
            L.orc_mbc_normality.restype = ct.c_double
            L.orc_splat_params.argtypes = [_D, _D, _D, _D, ct.c_double, _D]
            L.orc_splat_params.restype = ct.c_int
            L.orc_splat.argtypes = [ct.c_int, ct.c_int, ct.c_int, _D, ct.c_int64, _D, _D, _D, _D, ct.c_double, _D]
            L.orc_splat_backward.argtypes = [ct.c_int, ct.c_int, ct.c_int, _D, ct.c_int64, _D, _D, _D, _D,
                                             ct.c_double, _D, _D, _D, _D, _D]
            _lib = L
    return _lib


def threads() -> int:
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return a.ctypes.data_as(_D)


def _grid(grid):
    if hasattr(grid, "nx"):
        dims = (grid.nx, grid.ny, grid.nz)
        vox = (grid.vx, grid.vy, grid.vz)
    else:
        dims, vox = tuple(grid[:3]), tuple(grid[3:6])
    d = np.array(dims, dtype=np.int64)
    v = np.array(vox, dtype=np.float64)
    return d, v, int(d[0] * d[1] * d[2])


def quat_to_rot(q) -> np.ndarray:
    q = _f64(q)
    R = np.zeros(9)
    lib().orc_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def voxelize(grid, mean, scale, quat, value, kappa=3.0, cull=True) -> np.ndarray:
    """Eq. 4-5 voxelization; returns out[C][nz][ny][nx] (float64)."""
    d, v, n = _grid(grid)
    mean, scale, quat = _f64(mean).reshape(-1, 3), _f64(scale).reshape(-1, 3), _f64(quat).reshape(-1, 4)
    value = _f64(value)
    if value.ndim == 1:
        value = value[:, None]
    g, c = value.shape
    out = np.zeros(n * c)
    rc = lib().orc_voxelize(d.ctypes.data_as(_I64), _p(v), g, c, _p(mean), _p(scale), _p(quat), _p(value),
                            float(kappa), int(bool(cull)), _p(out))
    if rc != 0:
        raise ValueError("oracle voxelize rejected its arguments")
    return out.reshape(c, d[2], d[1], d[0])


def voxelize_ambiguity(grid, mean, scale, quat, value, kappa=3.0, eps=1e-4) -> np.ndarray:
    """Per-voxel mass of truncation decisions within eps*kappa^2 of the cutoff
    ([nz][ny][nx]); voxel values are unique only up to this mass."""
    d, v, n = _grid(grid)
    mean, scale, quat = _f64(mean).reshape(-1, 3), _f64(scale).reshape(-1, 3), _f64(quat).reshape(-1, 4)
    value = _f64(value)
    if value.ndim == 1:
        value = value[:, None]
    g, c = value.shape
    out = np.zeros(n)
    rc = lib().orc_voxelize_ambiguity(d.ctypes.data_as(_I64), _p(v), g, c, _p(mean), _p(scale), _p(quat),
                                      _p(value), float(kappa), float(eps), _p(out))
    if rc != 0:
        raise ValueError("oracle voxelize_ambiguity rejected its arguments")
    return out.reshape(d[2], d[1], d[0])


def voxelize_tie_band(grid, mean, scale, quat, value, kappa=3.0, units=2.0, offset=None):
    """Per-voxel mass of the truncation decisions that binary32 evaluation of q
    can flip ([nz][ny][nx]), from the first-order error bound of q per pair
    (band |q - kappa^2| <= units * bound), and the number of pairs in the band.
    offset (mm) shifts the voxel coordinates the bound sees (crops evaluated with
    shifted means)."""
    d, v, n = _grid(grid)
    mean, scale, quat = _f64(mean).reshape(-1, 3), _f64(scale).reshape(-1, 3), _f64(quat).reshape(-1, 4)
    value = _f64(value)
    if value.ndim == 1:
        value = value[:, None]
    g, c = value.shape
    out = np.zeros(n)
    cnt = np.zeros(1, dtype=np.int64)
    off = _f64(offset if offset is not None else (0.0, 0.0, 0.0))
    rc = lib().orc_voxelize_tie_band(d.ctypes.data_as(_I64), _p(v), g, c, _p(mean), _p(scale), _p(quat),
                                     _p(value), float(kappa), float(units), _p(off), _p(out),
                                     cnt.ctypes.data_as(_I64))
    if rc != 0:
        raise ValueError(f"oracle voxelize_tie_band failed ({rc})")
    return out.reshape(d[2], d[1], d[0]), int(cnt[0])


def qform_and_bound(mean, scale, quat, x, kappa=3.0):
    """(q, bound): the quadratic form of one Gaussian at x (mm) and the
    first-order bound on its binary32 evaluation error."""
    out = np.zeros(2)
    lib().orc_qform_and_bound(_p(_f64(mean)), _p(_f64(scale)), _p(_f64(quat)), _p(_f64(x)), float(kappa), _p(out))
    return float(out[0]), float(out[1])


def round_storage(x, fmt) -> np.ndarray:
    """Round to the nearest value of a storage format, ties to even, returned
    in float64: fmt "bf16" (8 significant bits, the float32 exponent range) or
    "f16" (11 significant bits, subnormals below 2^-14, largest finite 65504;
    larger magnitudes become infinite).  Written from the formats' definitions:
    the significand is scaled to an integer and rounded half to even."""
    x = np.asarray(x, dtype=np.float64)
    bits = {"bf16": 8, "f16": 11}[fmt]
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    if fmt == "f16":
        e = np.maximum(e, -13)  # below 2^-14 the quantum stays 2^-24
        m = np.ldexp(x, -e)
    out = np.ldexp(np.round(np.ldexp(m, bits)), e - bits)
    if fmt == "f16":
        out = np.where(np.abs(out) > 65504.0, np.copysign(np.inf, x), out)
    return out


def voxelize_backward(grid, mean, scale, quat, value, d_out, kappa=3.0):
    """Adjoint of `voxelize`; returns (d_mean, d_scale, d_quat, d_value)."""
    d, v, n = _grid(grid)
    mean, scale, quat = _f64(mean).reshape(-1, 3), _f64(scale).reshape(-1, 3), _f64(quat).reshape(-1, 4)
    value = _f64(value)
    if value.ndim == 1:
        value = value[:, None]
    g, c = value.shape
    dout = _f64(d_out).reshape(-1)
    assert dout.size == n * c
    dm, ds, dq, dv = np.zeros((g, 3)), np.zeros((g, 3)), np.zeros((g, 4)), np.zeros((g, c))
    rc = lib().orc_voxelize_backward(d.ctypes.data_as(_I64), _p(v), g, c, _p(mean), _p(scale), _p(quat), _p(value),
                                     float(kappa), _p(dout), _p(dm), _p(ds), _p(dq), _p(dv))
    if rc != 0:
        raise ValueError("oracle voxelize_backward rejected its arguments")
    return dm, ds, dq, dv


def combine(E, w) -> np.ndarray:
    """Eq. 3: E[L][3][N...], w[P][L][3] -> D[P][3][N...]."""
    E = _f64(E)
    w = _f64(w)
    L = E.shape[0]
    n = E[0, 0].size
    P = w.shape[0]
    D = np.zeros((P, 3) + E.shape[2:])
    lib().orc_combine(n, L, P, _p(E), _p(w), _p(D))
    return D


def combine_backward(E, w, dD):
    E, w, dD = _f64(E), _f64(w), _f64(dD)
    L, P, n = E.shape[0], w.shape[0], E[0, 0].size
    dE = np.zeros_like(E)
    dw = np.zeros_like(w)
    lib().orc_combine_backward(n, L, P, _p(E), _p(w), _p(dD), _p(dE), _p(dw))
    return dE, dw


def warp(grid, V, D) -> np.ndarray:
    """Eq. 2: V[N...], D[P][3][N...] (mm) -> W[P][N...]."""
    d, v, n = _grid(grid)
    V, D = _f64(V), _f64(D)
    P = D.shape[0]
    W = np.zeros((P,) + tuple(d[::-1]))
    lib().orc_warp(d.ctypes.data_as(_I64), _p(v), P, _p(V), _p(D), _p(W))
    return W


def warp_backward(grid, V, D, dW):
    d, v, n = _grid(grid)
    V, D, dW = _f64(V), _f64(D), _f64(dW)
    P = D.shape[0]
    dV = np.zeros(n)
    dD = np.zeros(D.shape)
    lib().orc_warp_backward(d.ctypes.data_as(_I64), _p(v), P, _p(V), _p(D), _p(dW), _p(dV), _p(dD))
    return dV.reshape(tuple(d[::-1])), dD


def project(grid, nu, nv, step, views, vol, shared=None) -> np.ndarray:
    """Eq. 6 ray sum; vol is [N...] (shared by every view) or [P][N...]."""
    d, v, n = _grid(grid)
    views = _f64(views).reshape(-1, 12)
    P = views.shape[0]
    vol = _f64(vol)
    if shared is None:
        shared = vol.size == n
    Y = np.zeros((P, nv, nu))
    lib().orc_project(d.ctypes.data_as(_I64), _p(v), int(nu), int(nv), float(step), P, _p(views), _p(vol),
                      0 if shared else n, _p(Y))
    return Y


def project_backward(grid, nu, nv, step, views, dY, shared=False) -> np.ndarray:
    d, v, n = _grid(grid)
    views = _f64(views).reshape(-1, 12)
    P = views.shape[0]
    dY = _f64(dY)
    out = np.zeros(n if shared else P * n)
    lib().orc_project_backward(d.ctypes.data_as(_I64), _p(v), int(nu), int(nv), float(step), P, _p(views),
                               _p(dY), _p(out), 0 if shared else n)
    return out.reshape(tuple(d[::-1]) if shared else (P,) + tuple(d[::-1]))


def project_gaussians(nu, nv, step, views, mean, scale, quat, value, m_lo, m_hi) -> np.ndarray:
    views = _f64(views).reshape(-1, 12)
    P = views.shape[0]
    mean, scale, quat = _f64(mean).reshape(-1, 3), _f64(scale).reshape(-1, 3), _f64(quat).reshape(-1, 4)
    value = _f64(value).reshape(-1)
    Y = np.zeros((P, nv, nu))
    lib().orc_project_gaussians(int(nu), int(nv), float(step), P, _p(views), mean.shape[0], _p(mean), _p(scale),
                                _p(quat), _p(value), int(m_lo), int(m_hi), _p(Y))
    return Y


def loss(kind, pred, meas, with_grad=True):
    """kind 1 = L1, 2 = L2, both averaged over all pixels; returns (loss, d_pred)."""
    pred, meas = _f64(pred), _f64(meas)
    g = np.zeros_like(pred) if with_grad else None
    val = lib().orc_loss(int(kind), pred.size, _p(pred), _p(meas), _p(g) if with_grad else None)
    return float(val), g


def dssim(pred, meas, data_range, with_grad=True):
    """D-SSIM term of Eq. 10/12 over projections [P, nv, nu]: mean over
    projections of 1 - mean SSIM (11x11 Gaussian window, sigma 1.5, zero
    padding, C1 = (0.01 range)^2, C2 = (0.03 range)^2); returns (loss, d_pred)."""
    pred, meas = _f64(pred), _f64(meas)
    P, nv, nu = pred.shape
    g = np.zeros_like(pred) if with_grad else None
    val = lib().orc_dssim(P, nu, nv, _p(pred), _p(meas), float(data_range), _p(g) if with_grad else None)
    return float(val), g


def tv(vol, D, origin, with_grad=True):
    """Sub-volume TV (Eq. 11/14) of vol [nz, ny, nx] on the D^3 crop at voxel
    origin (x, y, z); returns (loss, d_vol)."""
    vol = _f64(vol)
    nz, ny, nx = vol.shape
    dims = np.array([nx, ny, nz], dtype=np.int64)
    o = np.array(origin, dtype=np.int64)
    if not (np.all(o >= 0) and np.all(o + D <= dims) and D >= 2):
        raise ValueError("crop outside the volume")
    g = np.zeros_like(vol) if with_grad else None
    val = lib().orc_tv(dims.ctypes.data_as(_I64), _p(vol), int(D), o.ctypes.data_as(_I64),
                       _p(g) if with_grad else None)
    return float(val), g


def mbc_normality(E, with_grad=True):
    """Eq. 13 normality loss of MBC grids E [L, 3, ...]; returns (loss, dE)."""
    E = _f64(E)
    L = E.shape[0]
    N = int(np.prod(E.shape[2:]))
    g = np.zeros_like(E) if with_grad else None
    val = lib().orc_mbc_normality(L, N, _p(E), _p(g) if with_grad else None)
    return float(val), g



def splat_params(view, mean, scale, quat, value):
    """Eq. 8-9 for one Gaussian in one view: (p^_a, p^_b, Sigma^_00, Sigma^_01,
    Sigma^_11, rho^, |Sigma~|, |Sigma^|), or None behind the source."""
    out = np.zeros(8)
    ok = lib().orc_splat_params(_p(_f64(view)), _p(_f64(mean)), _p(_f64(scale)), _p(_f64(quat)), float(value),
                                _p(out))
    return out if ok else None


def splat(nu, nv, views, mean, scale, quat, value, kappa=3.0) -> np.ndarray:
    """Eq. 9 X-ray rasterization of the Gaussians into P projections [P][nv][nu]."""
    views = _f64(views).reshape(-1, 12)
    P, G = views.shape[0], int(np.asarray(mean).reshape(-1, 3).shape[0])
    Y = np.zeros((P, nv, nu))
    lib().orc_splat(int(nu), int(nv), int(P), _p(views), G, _p(_f64(mean)), _p(_f64(scale)), _p(_f64(quat)),
                    _p(_f64(value).reshape(-1)), float(kappa), _p(Y))
    return Y


def splat_backward(nu, nv, views, mean, scale, quat, value, dY, kappa=3.0):
    """Adjoint of splat: (d_mean, d_scale, d_quat, d_value)."""
    views = _f64(views).reshape(-1, 12)
    P, G = views.shape[0], int(np.asarray(mean).reshape(-1, 3).shape[0])
    dm, ds, dq, dv = np.zeros((G, 3)), np.zeros((G, 3)), np.zeros((G, 4)), np.zeros(G)
    lib().orc_splat_backward(int(nu), int(nv), int(P), _p(views), G, _p(_f64(mean)), _p(_f64(scale)),
                             _p(_f64(quat)), _p(_f64(value).reshape(-1)), float(kappa),
                             _p(_f64(dY).reshape(P, nv, nu)), _p(dm), _p(ds), _p(dq), _p(dv))
    return dm, ds, dq, dv
