"""Independent NumPy brute force for tiny inputs (TEST INFRASTRUCTURE ONLY).

A second, differently written statement of the same definitions as the C
oracle, used to cross-check it: the rotation comes from SciPy, the inverse
covariance from a matrix inverse, trilinear interpolation from a zero-padded
array, and every ray sums every sample index from 0 past the far side of the
volume with no clipping.  Only for volumes of a few thousand voxels.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation


def _grid(grid):
    if hasattr(grid, "nx"):
        return (grid.nx, grid.ny, grid.nz), (grid.vx, grid.vy, grid.vz)
    return tuple(int(x) for x in grid[:3]), tuple(float(x) for x in grid[3:6])


def rotation(q) -> np.ndarray:
    """Rotation matrix of quaternion (w, x, y, z) via SciPy (scalar-last input)."""
    q = np.asarray(q, dtype=np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def centres(grid) -> np.ndarray:
    """Voxel-centre coordinates, shape [nz, ny, nx, 3] (x, y, z in mm)."""
    (nx, ny, nz), (vx, vy, vz) = _grid(grid)
    x = (np.arange(nx) + 0.5 - nx / 2) * vx
    y = (np.arange(ny) + 0.5 - ny / 2) * vy
    z = (np.arange(nz) + 0.5 - nz / 2) * vz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def voxelize(grid, mean, scale, quat, value, kappa=np.inf) -> np.ndarray:
    xs = centres(grid)
    value = np.asarray(value, dtype=np.float64)
    if value.ndim == 1:
        value = value[:, None]
    out = np.zeros((value.shape[1],) + xs.shape[:3])
    for g in range(len(mean)):
        R = rotation(quat[g])
        sig = R @ np.diag(np.asarray(scale[g], dtype=np.float64) ** 2) @ R.T
        A = np.linalg.inv(sig)
        d = xs - np.asarray(mean[g], dtype=np.float64)
        q = np.einsum("...i,ij,...j->...", d, A, d)
        e = np.where(q <= kappa * kappa, np.exp(-0.5 * q), 0.0)
        out += value[g][:, None, None, None] * e[None]
    return out


def trilinear(V, u) -> np.ndarray:
    """Zero-padded trilinear interpolation of V[nz,ny,nx] at continuous indices
    u[..., 3] = (x, y, z)."""
    V = np.asarray(V, dtype=np.float64)
    nz, ny, nx = V.shape
    Vp = np.pad(V, 1)
    u = np.asarray(u, dtype=np.float64)
    fl = np.floor(u)
    f = u - fl
    i0 = fl.astype(np.int64) + 1  # padded index of the floor corner
    out = np.zeros(u.shape[:-1])
    lim = np.array([nx + 1, ny + 1, nz + 1])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                idx = i0 + np.array([dx, dy, dz])
                ok = np.all((idx >= 0) & (idx <= lim), axis=-1)
                idc = np.clip(idx, 0, lim)
                val = np.where(ok, Vp[idc[..., 2], idc[..., 1], idc[..., 0]], 0.0)
                wgt = ((f[..., 0] if dx else 1 - f[..., 0]) * (f[..., 1] if dy else 1 - f[..., 1])
                       * (f[..., 2] if dz else 1 - f[..., 2]))
                out += wgt * val
    return out


def combine(E, w) -> np.ndarray:
    return np.einsum("plk,lk...->pk...", np.asarray(w, np.float64), np.asarray(E, np.float64))


def warp(grid, V, D) -> np.ndarray:
    (nx, ny, nz), (vx, vy, vz) = _grid(grid)
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for Dp in np.asarray(D, np.float64):
        u = np.stack([X + Dp[0] / vx, Y + Dp[1] / vy, Z + Dp[2] / vz], axis=-1)
        out.append(trilinear(V, u))
    return np.stack(out)


def pixel_rays(view, nu, nv):
    view = np.asarray(view, dtype=np.float64)
    src, det, du, dv = view[0:3], view[3:6], view[6:9], view[9:12]
    a = np.arange(nu) + 0.5 - nu / 2
    b = np.arange(nv) + 0.5 - nv / 2
    pix = det[None, None] + b[:, None, None] * dv[None, None] + a[None, :, None] * du[None, None]
    d = pix - src
    return src, d / np.linalg.norm(d, axis=-1, keepdims=True)


def project(grid, nu, nv, step, views, vol) -> np.ndarray:
    """step * sum_{m=0..M} Trilin(vol_p, idx(src + m step r)), M past the far
    side of the volume's bounding sphere."""
    (nx, ny, nz), (vx, vy, vz) = _grid(grid)
    views = np.asarray(views, np.float64).reshape(-1, 12)
    vol = np.asarray(vol, np.float64)
    shared = vol.ndim == 3
    n = np.array([nx, ny, nz], dtype=np.float64)
    v = np.array([vx, vy, vz])
    out = np.zeros((len(views), nv, nu))
    for p, view in enumerate(views):
        src, r = pixel_rays(view, nu, nv)
        far = np.linalg.norm(src) + np.linalg.norm((n + 2) * v)
        m = np.arange(int(np.ceil(far / step)) + 2, dtype=np.float64)
        x = src + (m[:, None, None, None] * step) * r[None]
        u = x / v + n / 2 - 0.5
        W = vol if shared else vol[p]
        out[p] = step * trilinear(W, u).sum(axis=0)
    return out


def line_integral(src, r, mean, scale, quat, rho) -> float:
    """Closed-form integral over t in (-inf, inf) of rho exp(-q(src + t r)/2)
    for a unit direction r: with A = Sigma^-1 and m = src - mean,
    rho sqrt(2 pi / r^T A r) exp(-(m^T A m - (r^T A m)^2 / r^T A r) / 2)."""
    R = rotation(quat)
    A = np.linalg.inv(R @ np.diag(np.asarray(scale, np.float64) ** 2) @ R.T)
    m = np.asarray(src, np.float64) - np.asarray(mean, np.float64)
    r = np.asarray(r, np.float64)
    a = r @ A @ r
    b = r @ A @ m
    c = m @ A @ m
    return float(rho * np.sqrt(2 * np.pi / a) * np.exp(-0.5 * (c - b * b / a)))


def ray_space(view, x) -> np.ndarray:
    """phi(x) of the X-ray rasterizer: (a, b) where the ray from the source
    through x meets the detector plane (pixels, from the detector centre), and
    the distance |x - src|.  Found by solving det + a du + b dv = src + s (x - src)."""
    view = np.asarray(view, dtype=np.float64)
    src, det, du, dv = view[0:3], view[3:6], view[6:9], view[9:12]
    A = np.stack([du, dv, -(x - src)], axis=1)
    a, b, _ = np.linalg.solve(A, src - det)
    return np.array([a, b, np.linalg.norm(x - src)])


def splat(nu, nv, views, mean, scale, quat, value, kappa=np.inf, h=1e-4) -> np.ndarray:
    """Eq. 8-9 with the Jacobian of phi taken by central differences (step h mm)
    and every matrix operation done by NumPy."""
    views = np.asarray(views, dtype=np.float64).reshape(-1, 12)
    mean = np.asarray(mean, dtype=np.float64).reshape(-1, 3)
    scale = np.asarray(scale, dtype=np.float64).reshape(-1, 3)
    quat = np.asarray(quat, dtype=np.float64).reshape(-1, 4)
    value = np.asarray(value, dtype=np.float64).reshape(-1)
    ia, ib = np.meshgrid(np.arange(nu) + 0.5 - nu / 2, np.arange(nv) + 0.5 - nv / 2)
    xh = np.stack([ia, ib], axis=-1)  # [nv, nu, 2]
    Y = np.zeros((len(views), nv, nu))
    for p, view in enumerate(views):
        src, det, du, dv = view[0:3], view[3:6], view[6:9], view[9:12]
        normal = np.cross(du, dv)
        for g in range(len(mean)):
            if np.dot(normal, mean[g] - src) * np.dot(normal, det - src) <= 0:
                continue
            J = np.zeros((3, 3))
            for t in range(3):
                e = np.zeros(3)
                e[t] = h
                J[:, t] = (ray_space(view, mean[g] + e) - ray_space(view, mean[g] - e)) / (2 * h)
            R = rotation(quat[g])
            Sig = R @ np.diag(scale[g] ** 2) @ R.T
            St = J @ Sig @ J.T
            Sh = St[:2, :2]
            rho_hat = np.sqrt(2 * np.pi * np.linalg.det(St) / np.linalg.det(Sh)) * value[g]
            d = xh - ray_space(view, mean[g])[:2]
            q = np.einsum("...i,ij,...j->...", d, np.linalg.inv(Sh), d)
            Y[p] += np.where(q <= kappa ** 2, rho_hat * np.exp(-0.5 * q), 0.0)
    return Y
