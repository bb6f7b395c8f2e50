"""Pins of the oracle's Stage-1 X-ray rasterizer (Eq. 8-9) against things other
than itself: the closed-form line integral of a 3-D Gaussian (exact through the
mean, and in the parallel-beam limit), the convergence order of the local
affine approximation, the projected mass, symmetries, a NumPy brute force with
a numerically differentiated ray-space map, and central finite differences of
every parameter gradient."""
import numpy as np
import pytest

import oracle
from oracle import brute
from synth import circular_views


def _gaussians(seed, G, lo=-20.0, hi=20.0, s_lo=2.0, s_hi=5.0):
    rng = np.random.default_rng(seed)
    mean = rng.uniform(lo, hi, (G, 3))
    scale = rng.uniform(s_lo, s_hi, (G, 3))
    quat = rng.normal(size=(G, 4))
    value = rng.uniform(0.5, 1.5, G)
    return mean, scale, quat, value


def _inv_cov(scale, quat):
    R = brute.rotation(quat)
    return R @ np.diag(1.0 / np.asarray(scale) ** 2) @ R.T


def _pixel_ray(view, nu, nv, i, j):
    view = np.asarray(view, dtype=np.float64)
    src, det, du, dv = view[0:3], view[3:6], view[6:9], view[9:12]
    d = det + (i + 0.5 - nu / 2) * du + (j + 0.5 - nv / 2) * dv - src
    return src, d / np.linalg.norm(d)


def _line_integral(src, r, mean, scale, quat, value):
    """Closed form of the integral of rho exp(-1/2 (x-mu)^T A (x-mu)) along the
    whole line src + t r (the source is far outside the Gaussian's support)."""
    A = _inv_cov(scale, quat)
    m = src - mean
    m = m - (r @ m) * r  # the line's point nearest the mean: no cancellation in the exponent
    rAr, rAm, mAm = r @ A @ r, r @ A @ m, m @ A @ m
    return value * np.sqrt(2 * np.pi / rAr) * np.exp(-0.5 * (mAm - rAm * rAm / rAr))


def _exact_image(nu, nv, view, mean, scale, quat, value):
    Y = np.zeros((nv, nu))
    for j in range(nv):
        for i in range(nu):
            src, r = _pixel_ray(view, nu, nv, i, j)
            for g in range(len(mean)):
                Y[j, i] += _line_integral(src, r, mean[g], scale[g], quat[g], value[g])
    return Y


def test_matches_the_numpy_brute_force():
    vw = circular_views(3, 300.0, 450.0, 24, 20, 1.5, 1.5, start=0.3)
    mean, scale, quat, value = _gaussians(1, 6, -10, 10)
    for kappa in (np.inf, 3.0):
        a = oracle.splat(24, 20, vw, mean, scale, quat, value, kappa=kappa)
        b = brute.splat(24, 20, vw, mean, scale, quat, value, kappa=kappa)
        # the brute force differentiates phi numerically (step 1e-4 mm)
        assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()


def test_pixel_through_the_mean_equals_the_exact_line_integral():
    """Eq. 9 at p^ is rho sqrt(2 pi |Sigma~| / |Sigma^|) = rho sqrt(2 pi / (r^T Sigma^-1 r)),
    the exact integral along the ray through the mean, at any distance."""
    nu, nv = 16, 12
    vw = circular_views(4, 500.0, 800.0, nu, nv, 2.0, 2.0, start=0.7)
    rng = np.random.default_rng(2)
    for p in range(4):
        i, j = int(rng.integers(0, nu)), int(rng.integers(0, nv))
        src, r = _pixel_ray(vw[p], nu, nv, i, j)
        mean = src + rng.uniform(400.0, 600.0) * r
        scale, quat = rng.uniform(1.0, 6.0, 3), rng.normal(size=4)
        Y = oracle.splat(nu, nv, vw[p:p + 1], mean[None], scale[None], quat[None], np.array([1.3]), kappa=np.inf)
        exact = _line_integral(src, r, mean, scale, quat, 1.3)
        # |Sigma~| / |Sigma^| mixes pixel^2 and mm^2 entries: a few digits of fp64
        assert Y[0, j, i] == pytest.approx(exact, rel=1e-10)
        prm = oracle.splat_params(vw[p], mean, scale, quat, 1.3)
        assert prm[0] == pytest.approx(i + 0.5 - nu / 2, abs=1e-9)
        assert prm[1] == pytest.approx(j + 0.5 - nv / 2, abs=1e-9)


def test_parallel_beam_limit_matches_the_exact_line_integrals():
    """With the source 10^6 mm away the perspective map is affine across each
    Gaussian to sigma/z ~ 5e-6, so every pixel equals the exact line integral to
    that order (the error is first order in sigma/z: see the next test)."""
    nu, nv = 20, 18
    sad, sdd = 1.0e6, 1.5e6
    vw = circular_views(2, sad, sdd, nu, nv, 3.0, 3.0, start=0.4)  # 2 mm pixels at the isocentre
    mean, scale, quat, value = _gaussians(3, 4, -8, 8)
    Y = oracle.splat(nu, nv, vw, mean, scale, quat, value, kappa=np.inf)
    for p in range(2):
        E = _exact_image(nu, nv, vw[p], mean, scale, quat, value)
        assert np.abs(Y[p] - E).max() <= 2e-6 * np.abs(E).max()


def test_cone_beam_error_of_the_affine_approximation_is_first_order():
    """At a finite source distance z the local affine map errs by O(sigma/z)
    relative to the exact line integrals (the magnification varies across a
    Gaussian's depth, which skews its true footprint; the 2-D Gaussian of Eq. 9
    has no skew): doubling the source and detector distances halves the error."""
    nu, nv = 24, 20
    mean, scale, quat, value = _gaussians(4, 5, -15, 15, 3.0, 6.0)
    errs = []
    for k in (1.0, 2.0, 4.0):
        sad, sdd = 250.0 * k, 375.0 * k
        vw = circular_views(1, sad, sdd, nu, nv, 2.4, 2.4, start=0.2)
        Y = oracle.splat(nu, nv, vw, mean, scale, quat, value, kappa=np.inf)[0]
        E = _exact_image(nu, nv, vw[0], mean, scale, quat, value)
        errs.append(np.linalg.norm(Y - E) / np.linalg.norm(E))
    assert errs[0] < 5e-3
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2, errs


def test_projected_mass_in_the_parallel_limit():
    """Summing the projection over the detector, each pixel weighted by its area
    at the Gaussian's depth z (|du||dv| (z/h)^2, h the source-detector distance),
    gives the Gaussian's mass rho (2 pi)^(3/2) s1 s2 s3."""
    nu, nv = 64, 64
    sad, sdd = 1.0e6, 1.5e6
    vw = circular_views(1, sad, sdd, nu, nv, 1.5, 1.5, start=1.1)  # 1 mm pixels at the isocentre
    mean = np.array([[1.5, -2.0, 0.7]])
    scale = np.array([[3.0, 4.0, 2.5]])
    quat = np.array([[0.3, -0.2, 0.9, 0.1]])
    value = np.array([0.8])
    Y = oracle.splat(nu, nv, vw, mean, scale, quat, value, kappa=np.inf)
    src, det = vw[0, 0:3], vw[0, 3:6]
    n = (det - src) / np.linalg.norm(det - src)
    z = n @ (mean[0] - src)
    area = 1.5 * 1.5 * (z / sdd) ** 2
    mass = 0.8 * (2 * np.pi) ** 1.5 * 3.0 * 4.0 * 2.5
    assert Y.sum() * area == pytest.approx(mass, rel=1e-9)


def test_quaternion_sign_and_behind_the_source():
    nu, nv = 16, 16
    vw = circular_views(2, 300.0, 450.0, nu, nv, 1.5, 1.5)
    mean, scale, quat, value = _gaussians(5, 3, -10, 10)
    a = oracle.splat(nu, nv, vw, mean, scale, quat, value)
    b = oracle.splat(nu, nv, vw, mean, scale, -quat, value)
    assert np.array_equal(a, b)
    # a Gaussian behind the source of view 0 contributes nothing there
    src = vw[0, 0:3]
    behind = (src * 1.5)[None]
    Y = oracle.splat(nu, nv, vw[:1], behind, scale[:1], quat[:1], value[:1], kappa=np.inf)
    assert not Y.any()
    assert oracle.splat_params(vw[0], behind[0], scale[0], quat[0], 1.0) is None


def test_truncation_removes_only_pixels_outside_the_ellipse():
    nu, nv = 30, 26
    vw = circular_views(1, 300.0, 450.0, nu, nv, 1.0, 1.0)
    mean, scale, quat, value = _gaussians(6, 1, -3, 3, 1.5, 2.5)
    full = oracle.splat(nu, nv, vw, mean, scale, quat, value, kappa=np.inf)[0]
    cut = oracle.splat(nu, nv, vw, mean, scale, quat, value, kappa=2.0)[0]
    prm = oracle.splat_params(vw[0], mean[0], scale[0], quat[0], value[0])
    S = np.array([[prm[2], prm[3]], [prm[3], prm[4]]])
    ia, ib = np.meshgrid(np.arange(nu) + 0.5 - nu / 2, np.arange(nv) + 0.5 - nv / 2)
    d = np.stack([ia - prm[0], ib - prm[1]], -1)
    q = np.einsum("...i,ij,...j->...", d, np.linalg.inv(S), d)
    assert np.array_equal(cut[q <= 4.0], full[q <= 4.0])
    assert not cut[q > 4.0].any() and full[q > 4.0].any()


def _ellipse_mask(nu, nv, views, mean, scale, quat, kappa, h=1e-4):
    """Which (view, Gaussian, pixel) triples lie inside the truncation ellipse of
    Eq. 9, with the ray-space map solved by NumPy, its Jacobian by central
    differences and the 2-D covariance inverted by NumPy (as in the brute force)."""
    ia, ib = np.meshgrid(np.arange(nu) + 0.5 - nu / 2, np.arange(nv) + 0.5 - nv / 2)
    xh = np.stack([ia, ib], axis=-1)
    out = np.zeros((len(views), len(mean), nv, nu), dtype=bool)
    for p, view in enumerate(views):
        for g in range(len(mean)):
            J = np.stack([(brute.ray_space(view, mean[g] + e) - brute.ray_space(view, mean[g] - e)) / (2 * h)
                          for e in np.eye(3) * h], axis=1)
            R = brute.rotation(quat[g])
            Sh = (J @ R @ np.diag(np.asarray(scale[g]) ** 2) @ R.T @ J.T)[:2, :2]
            d = xh - brute.ray_space(view, mean[g])[:2]
            out[p, g] = np.einsum("...i,ij,...j->...", d, np.linalg.inv(Sh), d) <= kappa * kappa
    return out


@pytest.mark.parametrize("kappa", [np.inf, 3.0])
@pytest.mark.parametrize("param", ["mean", "scale", "quat", "value"])
def test_gradients_match_central_differences(param, kappa):
    """At kappa = 3 the image is only piecewise smooth in the parameters: a pixel
    that crosses a Gaussian's kappa-ellipse adds or drops a term.  No central
    difference of these seeds moves any pixel across an ellipse (checked with the
    NumPy ray-space map), so the differences see exactly the pixels inside, and
    the adjoint must skip the rest."""
    nu, nv = 18, 14
    vw = circular_views(2, 300.0, 450.0, nu, nv, 1.6, 1.6, start=0.5)
    mean, scale, quat, value = _gaussians(7, 3, -8, 8, 2.0, 4.0)
    dY = np.random.default_rng(8).normal(size=(2, nv, nu))
    grads = dict(zip(("mean", "scale", "quat", "value"),
                     oracle.splat_backward(nu, nv, vw, mean, scale, quat, value, dY, kappa=kappa)))
    args = dict(mean=mean, scale=scale, quat=quat, value=value)
    if np.isfinite(kappa):
        inside = _ellipse_mask(nu, nv, vw, mean, scale, quat, kappa)
        assert inside.any() and not inside.all()
    x = args[param]
    fd = np.zeros_like(x)
    h = 1e-5
    for idx in np.ndindex(x.shape):
        for sgn in (1, -1):
            xp = x.copy()
            xp[idx] += sgn * h
            a = dict(args, **{param: xp})
            if np.isfinite(kappa) and param != "value":
                assert np.array_equal(_ellipse_mask(nu, nv, vw, a["mean"], a["scale"], a["quat"], kappa), inside)
            fd[idx] += sgn * np.sum(dY * oracle.splat(nu, nv, vw, a["mean"], a["scale"], a["quat"], a["value"],
                                                      kappa=kappa)) / (2 * h)
    g = grads[param]
    assert np.abs(g - fd).max() <= 1e-6 * max(np.abs(fd).max(), 1e-12)
