"""Pins for the oracle's cone-beam projector (Eq. 6-7 discretised), warp (Eq. 2)
and combine (Eq. 3): exact sums, closed-form line integrals, symmetries and a
NumPy brute force."""
import numpy as np
import pytest

import oracle
from oracle import brute
from synth import Grid, circular_views


def _axis_view(axis, y0, z0, sad=1000.0):
    """A single-pixel view whose one ray runs along +axis through the point whose
    other two coordinates are (y0, z0) (in cyclic order after `axis`)."""
    src = np.zeros(3)
    det = np.zeros(3)
    o1, o2 = (axis + 1) % 3, (axis + 2) % 3
    src[axis], det[axis] = -sad, 500.0
    src[o1] = det[o1] = y0
    src[o2] = det[o2] = z0
    du = np.zeros(3)
    dv = np.zeros(3)
    du[o1] = 1.0
    dv[o2] = 1.0
    return np.concatenate([src, det, du, dv])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_axis_aligned_ray_is_exact_voxel_row_sum(axis):
    """A ray along a grid axis through voxel centres, with step v/2 and the source
    on the half-voxel lattice, samples every voxel centre and every midpoint, so
    the trilinear sum is exactly 2 sum_i V_i and the line integral v sum_i V_i."""
    grid = Grid(7, 6, 5, 1.0, 1.0, 1.0)
    rng = np.random.default_rng(axis)
    V = rng.random(grid.shape)
    n = (grid.nx, grid.ny, grid.nz)
    o1, o2 = (axis + 1) % 3, (axis + 2) % 3
    i1, i2 = 2, 3
    c1 = i1 + 0.5 - n[o1] / 2
    c2 = i2 + 0.5 - n[o2] / 2
    view = _axis_view(axis, c1, c2)
    Y = oracle.project(grid, 1, 1, 0.5, view[None], V)
    idx = [slice(None)] * 3
    idx[2 - o1], idx[2 - o2] = i1, i2
    expect = 1.0 * V[tuple(idx)].sum()
    assert Y[0, 0, 0] == pytest.approx(expect, rel=1e-12)


def test_continuous_ray_sum_matches_closed_form_line_integral():
    """Eq. 7 for one anisotropic Gaussian: the source-anchored sample sum with a
    step well below the Gaussian's width equals the closed-form integral
    rho sqrt(2 pi / r^T A r) exp(-(m^T A m - (r^T A m)^2 / r^T A r)/2)."""
    nu, nv = 5, 4
    views = circular_views(3, 1000.0, 1500.0, nu, nv, 3.0, 2.5, start=0.4)
    mean, scale, quat, rho = np.array([2.0, -1.5, 1.0]), np.array([3.0, 4.0, 5.0]), np.array([0.7, -0.2, 0.5, 0.3]), 0.9
    Y = oracle.project_gaussians(nu, nv, 0.5, views, mean[None], scale[None], quat[None], np.array([rho]), 1800, 2200)
    for p in range(3):
        src, r = brute.pixel_rays(views[p], nu, nv)
        for b in range(nv):
            for a in range(nu):
                expect = brute.line_integral(src, r[b, a], mean, scale, quat, rho)
                assert Y[p, b, a] == pytest.approx(expect, rel=1e-10)


def test_voxelized_projection_converges_at_second_order():
    """Voxelize -> trilinear ray march approaches the analytic line integral at
    O(h^2) as the voxel shrinks (same physical Gaussian and step = h/2)."""
    mean, scale, quat, rho = np.array([1.3, -0.7, 0.9]), np.array([6.0, 7.0, 8.0]), np.array([0.9, 0.2, -0.3, 0.1]), 1.0
    views = circular_views(2, 1000.0, 1500.0, 6, 6, 4.0, 4.0, start=0.2)
    exact = np.empty((2, 6, 6))
    for p in range(2):
        src, r = brute.pixel_rays(views[p], 6, 6)
        for b in range(6):
            for a in range(6):
                exact[p, b, a] = brute.line_integral(src, r[b, a], mean, scale, quat, rho)
    errs = []
    for h in (4.0, 2.0, 1.0):
        n = int(round(96 / h))
        grid = Grid(n, n, n, h, h, h)
        V = oracle.voxelize(grid, mean[None], scale[None], quat[None], np.array([[rho]]), kappa=np.inf)[0]
        Y = oracle.project(grid, 6, 6, h / 2, views, V)
        errs.append(np.linalg.norm(Y - exact) / np.linalg.norm(exact))
    order1 = np.log2(errs[0] / errs[1])
    order2 = np.log2(errs[1] / errs[2])
    assert 1.6 < order1 < 2.6 and 1.6 < order2 < 2.6, errs
    # trilinear interpolation biases each transverse axis by about (h^2/12) f'',
    # i.e. a relative error of order (h / sigma)^2 / 6 at the finest grid
    assert errs[2] < (1.0 / 6.0) ** 2 / 6.0


def test_rotation_by_90_degrees_permutes_views():
    """Rotating the volume by +90 degrees about z and advancing the gantry by 90
    degrees leaves every projection unchanged (nx = ny, centred grid)."""
    grid = Grid(10, 10, 6, 2.0, 2.0, 3.0)
    rng = np.random.default_rng(9)
    V = rng.random(grid.shape)
    # V'(x, y) = V(y, -x)  <=>  V'[k][j'][i'] = V[k][n-1-i'][j']
    V2 = V[:, ::-1, :].transpose(0, 2, 1)
    a = oracle.project(grid, 12, 8, 1.0, circular_views(4, 300.0, 450.0, 12, 8, 2.0, 2.0, start=0.3), V)
    b = oracle.project(grid, 12, 8, 1.0, circular_views(4, 300.0, 450.0, 12, 8, 2.0, 2.0, start=0.3 + np.pi / 2), V2)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_integer_translation_moves_with_the_geometry():
    """Samples are anchored at the source, so translating the object by t voxels
    and the whole scanner by t*v mm gives the same projections."""
    grid = Grid(12, 12, 10, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(4)
    V = np.zeros(grid.shape)
    V[3:7, 3:8, 2:6] = rng.random((4, 5, 4))
    t = np.array([2, -1, 1])  # voxels (x, y, z)
    Vt = np.roll(V, shift=(t[2], t[1], t[0]), axis=(0, 1, 2))
    views = circular_views(3, 400.0, 600.0, 10, 9, 2.5, 2.5, start=0.1)
    vt = views.copy()
    shift = t * 2.0
    vt[:, 0:3] += shift
    vt[:, 3:6] += shift
    a = oracle.project(grid, 10, 9, 1.0, views, V)
    b = oracle.project(grid, 10, 9, 1.0, vt, Vt)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_project_matches_numpy_brute_force():
    grid = Grid(8, 7, 6, 2.0, 2.5, 3.0)
    rng = np.random.default_rng(8)
    V = rng.random((2,) + grid.shape)
    views = circular_views(2, 100.0, 160.0, 4, 3, 4.0, 5.0, start=0.7)
    views[1, 2] += 3.0  # an off-plane source
    a = oracle.project(grid, 4, 3, 1.1, views, V)
    b = brute.project(grid, 4, 3, 1.1, views, V)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_projector_adjoint_dot_product():
    grid = Grid(9, 8, 7, 2.0, 2.0, 2.5)
    rng = np.random.default_rng(10)
    views = circular_views(3, 120.0, 200.0, 7, 5, 3.0, 3.0, start=0.2)
    x = rng.normal(size=(3,) + grid.shape)
    y = rng.normal(size=(3, 5, 7))
    Ax = oracle.project(grid, 7, 5, 1.3, views, x)
    Aty = oracle.project_backward(grid, 7, 5, 1.3, views, y)
    lhs, rhs = (Ax * y).sum(), (x * Aty).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # shared-volume adjoint: one dvol accumulates every view
    xs = rng.normal(size=grid.shape)
    Axs = oracle.project(grid, 7, 5, 1.3, views, xs)
    Atys = oracle.project_backward(grid, 7, 5, 1.3, views, y, shared=True)
    assert (Axs * y).sum() == pytest.approx((xs * Atys).sum(), rel=1e-12)


# ------------------------------------------------------------------- warp


def test_zero_dvf_is_identity():
    grid = Grid(9, 8, 7, 2.0, 2.5, 1.5)
    V = np.random.default_rng(1).random(grid.shape)
    W = oracle.warp(grid, V, np.zeros((2, 3) + grid.shape))
    np.testing.assert_array_equal(W[0], V)
    np.testing.assert_array_equal(W[1], V)


def test_integer_translation_dvf_shifts_exactly():
    """Eq. 2 pulls: d = t v gives W[i] = V[i + t], zero beyond the border."""
    grid = Grid(9, 8, 7, 2.0, 2.5, 1.5)
    V = np.random.default_rng(2).random(grid.shape)
    t = (2, -1, 3)
    D = np.zeros((1, 3) + grid.shape)
    for a, (ta, va) in enumerate(zip(t, (grid.vx, grid.vy, grid.vz))):
        D[0, a] = ta * va
    W = oracle.warp(grid, V, D)[0]
    expect = np.zeros_like(V)
    nz, ny, nx = grid.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                ii, jj, kk = i + t[0], j + t[1], k + t[2]
                if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                    expect[k, j, i] = V[kk, jj, ii]
    np.testing.assert_array_equal(W, expect)


def test_trilinear_reproduces_linear_fields():
    """Trilinear interpolation is exact for a linear field sampled inside the grid."""
    grid = Grid(10, 9, 8, 2.0, 1.0, 4.0)
    nz, ny, nx = grid.shape
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    V = 0.3 * I - 1.1 * J + 0.7 * K + 2.0
    rng = np.random.default_rng(6)
    u = np.stack([rng.uniform(0, nx - 1, I.shape), rng.uniform(0, ny - 1, I.shape),
                  rng.uniform(0, nz - 1, I.shape)])
    D = np.stack([(u[0] - I) * grid.vx, (u[1] - J) * grid.vy, (u[2] - K) * grid.vz])[None]
    W = oracle.warp(grid, V, D)[0]
    np.testing.assert_allclose(W, 0.3 * u[0] - 1.1 * u[1] + 0.7 * u[2] + 2.0, rtol=1e-12, atol=1e-12)


def test_warp_matches_numpy_brute_force():
    grid = Grid(9, 8, 7, 2.0, 2.5, 1.5)
    rng = np.random.default_rng(12)
    V = rng.random(grid.shape)
    D = rng.normal(0, 3.0, (2, 3) + grid.shape)
    np.testing.assert_allclose(oracle.warp(grid, V, D), brute.warp(grid, V, D), rtol=1e-12, atol=1e-13)


def test_warp_adjoint_dot_product_in_volume():
    grid = Grid(9, 8, 7, 2.0, 2.5, 1.5)
    rng = np.random.default_rng(13)
    D = rng.normal(0, 3.0, (3, 3) + grid.shape)
    x = rng.normal(size=grid.shape)
    y = rng.normal(size=(3,) + grid.shape)
    Ax = oracle.warp(grid, x, D)
    Aty, _ = oracle.warp_backward(grid, x, D, y)
    assert (Ax * y).sum() == pytest.approx((x * Aty).sum(), rel=1e-12)


def test_warp_dvf_gradient_matches_central_differences():
    grid = Grid(7, 6, 5, 2.0, 2.5, 1.5)
    rng = np.random.default_rng(14)
    V = rng.random(grid.shape)
    D = rng.normal(0, 2.0, (2, 3) + grid.shape)
    G = rng.normal(size=(2,) + grid.shape)
    _, dD = oracle.warp_backward(grid, V, D, G)
    h = 1e-6
    for idx in [(0, 0, 2, 3, 4), (1, 1, 1, 2, 3), (0, 2, 3, 4, 5), (1, 0, 4, 1, 1)]:
        Dp, Dm = D.copy(), D.copy()
        Dp[idx] += h
        Dm[idx] -= h
        fd = ((oracle.warp(grid, V, Dp) * G).sum() - (oracle.warp(grid, V, Dm) * G).sum()) / (2 * h)
        assert dD[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- combine


def test_combine_matches_einsum_and_special_cases():
    rng = np.random.default_rng(15)
    E = rng.normal(size=(3, 3, 4, 5, 6))
    w = rng.normal(size=(5, 3, 3))
    np.testing.assert_allclose(oracle.combine(E, w), brute.combine(E, w), rtol=1e-13, atol=1e-13)
    unit = np.zeros((1, 3, 3))
    unit[0, 1, :] = 1.0
    np.testing.assert_array_equal(oracle.combine(E, unit)[0], E[1])
    np.testing.assert_array_equal(oracle.combine(E, np.zeros((2, 3, 3))), np.zeros((2, 3, 4, 5, 6)))


def test_combine_adjoint_dot_product():
    rng = np.random.default_rng(16)
    E = rng.normal(size=(3, 3, 20))
    w = rng.normal(size=(4, 3, 3))
    dD = rng.normal(size=(4, 3, 20))
    dE, dw = oracle.combine_backward(E, w, dD)
    D = oracle.combine(E, w)
    # linear in E for fixed w and linear in w for fixed E
    assert (D * dD).sum() == pytest.approx((E * dE).sum(), rel=1e-12)
    assert (D * dD).sum() == pytest.approx((w * dw).sum(), rel=1e-12)


# -------------------------------------------------------------------- loss


def test_loss_values_and_gradients():
    rng = np.random.default_rng(17)
    a, b = rng.normal(size=(3, 4, 5)), rng.normal(size=(3, 4, 5))
    b.flat[7] = a.flat[7]
    l2, g2 = oracle.loss(2, a, b)
    l1, g1 = oracle.loss(1, a, b)
    assert l2 == pytest.approx(np.mean((a - b) ** 2), rel=1e-14)
    assert l1 == pytest.approx(np.mean(np.abs(a - b)), rel=1e-14)
    np.testing.assert_allclose(g2, 2 * (a - b) / a.size, rtol=1e-14)
    np.testing.assert_allclose(g1, np.sign(a - b) / a.size, rtol=1e-14)
    assert g1.flat[7] == 0.0
