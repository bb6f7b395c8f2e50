"""Pins for the oracle's Gaussian voxelizer (Eq. 4-5) against closed forms,
library routines and invariants -- nothing here re-types the oracle's loop."""
import math

import numpy as np
import pytest
from scipy.stats import multivariate_normal

import oracle
from oracle import brute
from synth import Grid


def _one(mean, scale, quat, rho):
    return (np.array([mean], float), np.array([scale], float), np.array([quat], float),
            np.array([[rho]], float))


def test_isotropic_voxel_sum_is_product_of_1d_sums():
    """An isotropic Gaussian factorises, so its voxel sum is the product of three
    1-D sums over the voxel-centre coordinates (exact, kappa = inf)."""
    grid = Grid(20, 18, 16, 1.5, 2.0, 2.5)
    mu, sig, rho = (0.7, -1.3, 2.1), 3.1, 0.8
    out = oracle.voxelize(grid, *_one(mu, (sig,) * 3, (0.3, -0.5, 0.2, 0.9), rho), kappa=np.inf)
    sums = []
    for n, v, m in zip((grid.nx, grid.ny, grid.nz), (grid.vx, grid.vy, grid.vz), mu):
        c = (np.arange(n) + 0.5 - n / 2) * v
        sums.append(np.exp(-0.5 * ((c - m) / sig) ** 2).sum())
    expect = rho * sums[0] * sums[1] * sums[2]
    assert out.sum() == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("scale", [(3.0, 3.0, 3.0), (2.4, 3.5, 5.0)])
def test_voxel_sum_matches_continuous_mass(scale):
    """Poisson summation: for scales >= 1.5 voxels and a grid holding the whole
    Gaussian, sum_v G(x_v) = rho (2 pi)^{3/2} s1 s2 s3 / (vx vy vz) up to
    ~exp(-2 pi^2 (s/v)^2), for any rotation."""
    grid = Grid(72, 72, 72, 1.0, 1.0, 1.0)  # +-36 mm: > 7 sigma, so the box cuts off < 1e-11
    rho = 1.7
    out = oracle.voxelize(grid, *_one((0.31, -0.47, 0.23), scale, (0.6, 0.2, -0.7, 0.33), rho), kappa=np.inf)
    expect = rho * (2 * np.pi) ** 1.5 * np.prod(scale)
    assert out.sum() == pytest.approx(expect, rel=1e-9)


def test_truncated_mass_matches_chi_square_tail():
    """With the hard cutoff q <= kappa^2 the retained mass is 1 - P(chi^2_3 > kappa^2),
    P = erfc(kappa/sqrt 2) + sqrt(2/pi) kappa exp(-kappa^2/2) (0.0293 at kappa = 3),
    up to the lattice error of the cut surface (well below 2e-3 at 5-voxel scales)."""
    grid = Grid(64, 64, 64, 1.0, 1.0, 1.0)
    kappa, s = 3.0, (5.0, 4.5, 5.5)
    full = (2 * np.pi) ** 1.5 * np.prod(s)
    out = oracle.voxelize(grid, *_one((0.2, 0.1, -0.3), s, (0.9, 0.1, 0.3, -0.2), 1.0), kappa=kappa)
    tail = math.erfc(kappa / math.sqrt(2)) + math.sqrt(2 / math.pi) * kappa * math.exp(-kappa ** 2 / 2)
    assert tail == pytest.approx(0.0293, abs=1e-4)
    assert out.sum() / full == pytest.approx(1.0 - tail, rel=2e-3)


def test_single_anisotropic_gaussian_matches_scipy_pdf():
    """Every voxel of one rotated anisotropic Gaussian equals
    rho (2 pi)^{3/2} |Sigma|^{1/2} N(x; mu, Sigma), with Sigma = R S^2 R^T built
    from SciPy's quaternion rotation: pins the quaternion order (w,x,y,z), the
    rotation's orientation and the quadratic form."""
    grid = Grid(12, 10, 9, 2.0, 1.5, 2.5)
    mu, s, q, rho = np.array([1.1, -0.9, 0.4]), np.array([2.0, 4.5, 3.0]), np.array([0.8, 0.3, -0.4, 0.25]), 0.6
    out = oracle.voxelize(grid, *_one(mu, s, q, rho), kappa=np.inf)[0]
    R = brute.rotation(q)
    sig = R @ np.diag(s ** 2) @ R.T
    xs = brute.centres(grid).reshape(-1, 3)
    expect = rho * (2 * np.pi) ** 1.5 * np.sqrt(np.linalg.det(sig)) * multivariate_normal(mu, sig).pdf(xs)
    np.testing.assert_allclose(out.reshape(-1), expect, rtol=1e-11, atol=1e-14)


def test_quaternion_sign_and_norm_invariance():
    grid = Grid(10, 10, 10, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(5)
    m, s = rng.normal(0, 3, (6, 3)), rng.uniform(1.5, 4, (6, 3))
    q, val = rng.normal(size=(6, 4)), rng.random((6, 1))
    a = oracle.voxelize(grid, m, s, q, val, kappa=3.0)
    b = oracle.voxelize(grid, m, s, -q, val, kappa=3.0)
    c = oracle.voxelize(grid, m, s, 3.7 * q, val, kappa=3.0)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_allclose(a, c, rtol=1e-12, atol=1e-14)


def test_culled_loop_equals_full_loop():
    """Skipping voxels outside the kappa-ellipsoid's bounding box changes nothing."""
    grid = Grid(14, 12, 10, 2.0, 2.0, 3.0)
    rng = np.random.default_rng(11)
    G = 40
    m = (rng.random((G, 3)) - 0.5) * np.array([32, 28, 34])
    s = rng.uniform(1.0, 6.0, (G, 3))
    q, val = rng.normal(size=(G, 4)), rng.normal(size=(G, 3))
    a = oracle.voxelize(grid, m, s, q, val, kappa=2.5, cull=True)
    b = oracle.voxelize(grid, m, s, q, val, kappa=2.5, cull=False)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("kappa", [np.inf, 2.0])
def test_voxelize_matches_numpy_brute_force(kappa):
    grid = Grid(9, 8, 7, 2.0, 2.5, 1.5)
    rng = np.random.default_rng(21)
    G = 5
    m = (rng.random((G, 3)) - 0.5) * np.array([18, 20, 10])
    s = rng.uniform(1.0, 5.0, (G, 3))
    q, val = rng.normal(size=(G, 4)), rng.normal(size=(G, 3))
    a = oracle.voxelize(grid, m, s, q, val, kappa=kappa)
    b = brute.voxelize(grid, m, s, q, val, kappa=kappa)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-13)


def test_negative_values_are_permitted():
    """Sec. 2.3.1: the MBC voxelizer carries signed values; negating the values
    negates the volume."""
    grid = Grid(8, 8, 8, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(3)
    m, s, q, val = rng.normal(0, 3, (4, 3)), rng.uniform(2, 4, (4, 3)), rng.normal(size=(4, 4)), rng.normal(size=(4, 3))
    a = oracle.voxelize(grid, m, s, q, val)
    b = oracle.voxelize(grid, m, s, q, -val)
    np.testing.assert_array_equal(a, -b)
    assert a.min() < 0 < a.max()


def test_ambiguity_mass_is_the_band_between_two_cutoffs():
    """For positive values, voxelize(kappa sqrt(1+eps)) - voxelize(kappa sqrt(1-eps))
    keeps exactly the pairs in the band |q - kappa^2| <= eps kappa^2, which is
    what the ambiguity mass sums; with kappa = inf there is no band."""
    grid = Grid(16, 14, 12, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(41)
    G = 30
    m = (rng.random((G, 3)) - 0.5) * np.array([32, 28, 24])
    s = rng.uniform(1.0, 5.0, (G, 3))
    q, val = rng.normal(size=(G, 4)), rng.random((G, 1))
    eps = 0.05
    amb = oracle.voxelize_ambiguity(grid, m, s, q, val, 3.0, eps)
    hi = oracle.voxelize(grid, m, s, q, val, kappa=3.0 * np.sqrt(1 + eps))[0]
    lo = oracle.voxelize(grid, m, s, q, val, kappa=3.0 * np.sqrt(1 - eps))[0]
    # the band's upper edge is inclusive on both sides; the lower cutoff keeps q <= lo2
    # exactly, so the difference is the band minus pairs sitting exactly on lo2 (none here)
    np.testing.assert_allclose(hi - lo, amb, rtol=1e-12, atol=1e-15)
    assert amb.max() > 0
    assert oracle.voxelize_ambiguity(grid, m, s, q, val, np.inf, eps).max() == 0.0


def _q_binary32(mu, s, quat, x):
    """q evaluated entirely in binary32 (NumPy float32, no fused operations) in
    three different orders: the symmetric inverse-covariance form, the sum of
    squares of R^T d / s, and A d dotted with d."""
    f = np.float32
    mu, s, quat, x = (np.asarray(a, f) for a in (mu, s, quat, x))
    n = np.sqrt(f(quat @ quat))
    w, a, b, c = quat * (f(1) / n)
    R = np.array([[1 - 2 * (b * b + c * c), 2 * (a * b - w * c), 2 * (a * c + w * b)],
                  [2 * (a * b + w * c), 1 - 2 * (a * a + c * c), 2 * (b * c - w * a)],
                  [2 * (a * c - w * b), 2 * (b * c + w * a), 1 - 2 * (a * a + b * b)]], dtype=f)
    d = (x - mu).astype(f)
    is2 = (f(1) / (s * s)).astype(f)
    A = np.array([[R[i, 0] * R[j, 0] * is2[0] + R[i, 1] * R[j, 1] * is2[1] + R[i, 2] * R[j, 2] * is2[2]
                   for j in range(3)] for i in range(3)], dtype=f)
    tx = A[0, 0] * d[0] + (A[0, 1] + A[1, 0]) * d[1] + (A[0, 2] + A[2, 0]) * d[2]
    ty = A[1, 1] * d[1] + (A[1, 2] + A[2, 1]) * d[2]
    q1 = d[0] * tx + d[1] * ty + A[2, 2] * d[2] * d[2]
    r = (R.T @ d).astype(f) / s
    q2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2]
    q3 = (A @ d).astype(f) @ d
    return [float(q1), float(q2), float(q3)]


def test_binary32_error_of_q_stays_inside_the_tie_bound():
    """The tie band rests on a first-order bound of the error of q evaluated in
    binary32.  Evaluating q in binary32 in three orders for points near the
    kappa = 3 surface of Gaussians with paper-scale coordinates (+-200 mm) and
    anisotropic scales (1-6 mm), every error stays inside the bound -- with
    room to spare, so the bound is valid -- and the bound is a small fraction
    of kappa^2 (the band holds few pairs)."""
    rng = np.random.default_rng(17)
    worst, widths = 0.0, []
    for _ in range(3000):
        mu = rng.uniform(-200, 200, 3) * np.array([1.0, 1.0, 0.5])
        s = np.exp(rng.uniform(np.log(1.0), np.log(6.0), 3))
        quat = rng.normal(size=4)
        u = rng.normal(size=3)
        x = mu + brute.rotation(quat) @ (s * u / np.linalg.norm(u) * 3.0 * rng.uniform(0.98, 1.02))
        mu, s, quat, x = (np.asarray(a, np.float32).astype(np.float64) for a in (mu, s, quat, x))
        q64, bound = oracle.qform_and_bound(mu, s, quat, x, 3.0)
        for q32 in _q_binary32(mu, s, quat, x):
            worst = max(worst, abs(q32 - q64) / bound)
        widths.append(bound / 9.0)
    assert 0.0 < worst <= 0.5
    assert np.median(widths) <= 1e-4 and np.max(widths) <= 1e-3


def test_tie_band_lies_between_two_fixed_bands():
    """The per-pair band sits between the fixed relative bands eps kappa^2 with
    eps the smallest and the largest per-pair width, so its mass is sandwiched
    between the two ambiguity masses; with kappa = inf it is empty."""
    grid = Grid(16, 14, 12, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(41)
    G = 30
    m = (rng.random((G, 3)) - 0.5) * np.array([32, 28, 24])
    s = rng.uniform(1.0, 5.0, (G, 3))
    q, val = rng.normal(size=(G, 4)), rng.random((G, 1))
    units = 100.0  # wide enough that the band holds pairs on this small grid
    amb, npairs = oracle.voxelize_tie_band(grid, m, s, q, val, 3.0, units)
    widths = []
    for g in range(G):
        for x in brute.centres(grid).reshape(-1, 3)[::7]:
            widths.append(units * oracle.qform_and_bound(m[g], s[g], q[g], x, 3.0)[1] / 9.0)
    lo = oracle.voxelize_ambiguity(grid, m, s, q, val, 3.0, 0.5 * min(widths))
    hi = oracle.voxelize_ambiguity(grid, m, s, q, val, 3.0, 2.0 * max(widths))
    assert npairs > 0 and amb.sum() > 0
    assert np.all(lo <= amb + 1e-15) and np.all(amb <= hi + 1e-15)
    assert oracle.voxelize_tie_band(grid, m, s, q, val, np.inf)[0].max() == 0.0
