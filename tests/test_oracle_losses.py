"""Pins of the oracle's Eq. 13-14 loss terms against things other than itself:
closed forms, invariants, library routines (SciPy correlation for the SSIM
window sums, NumPy differences for TV) and central finite differences."""
import numpy as np
import pytest
from scipy import ndimage

import oracle


def _window():
    t = np.arange(11) - 5.0
    w = np.exp(-t * t / (2 * 1.5 ** 2))
    return np.outer(w, w) / w.sum() ** 2


def _corr(img):
    return ndimage.correlate(img, _window(), mode="constant", cval=0.0)


# ---------------------------------------------------------------- D-SSIM

def test_dssim_of_identical_images_is_zero_with_zero_gradient():
    Y = np.random.default_rng(1).random((3, 17, 23)) * 5
    val, g = oracle.dssim(Y, Y, 5.0)
    assert abs(val) < 1e-14
    assert np.abs(g).max() < 1e-14


def test_dssim_constant_images_match_the_closed_form():
    """For constant images a and b the windowed moments are a s, b s, a^2 s,
    b^2 s, a b s with s(q) the window mass inside the image (a SciPy
    correlation of ones), which fixes every term of the SSIM formula."""
    a, b, rng_ = 2.0, 3.5, 4.0
    nv, nu = 19, 26
    Y, M = np.full((1, nv, nu), a), np.full((1, nv, nu), b)
    s = _corr(np.ones((nv, nu)))
    C1, C2 = (0.01 * rng_) ** 2, (0.03 * rng_) ** 2
    var = s * (1 - s)
    S = ((2 * a * b * s * s + C1) * (2 * a * b * var + C2)) / (((a * a + b * b) * s * s + C1) *
                                                              ((a * a + b * b) * var + C2))
    # the oracle forms s_x^2 = E[x^2] - mu_x^2 by difference, which cancels to
    # ~1e-16 a^2 where s = 1: a few ulps of a^2 against C2, hence 1e-10
    assert oracle.dssim(Y, M, rng_, with_grad=False)[0] == pytest.approx(1 - S.mean(), rel=1e-10)


def test_dssim_matches_window_sums_from_scipy():
    rng = np.random.default_rng(2)
    Y, M = rng.random((2, 14, 21)), rng.random((2, 14, 21))
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ref = 0.0
    for p in range(2):
        mx, my = _corr(Y[p]), _corr(M[p])
        sxx, syy, sxy = _corr(Y[p] ** 2) - mx * mx, _corr(M[p] ** 2) - my * my, _corr(Y[p] * M[p]) - mx * my
        S = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
        ref += 1 - S.mean()
    assert oracle.dssim(Y, M, 1.0, with_grad=False)[0] == pytest.approx(ref / 2, rel=1e-12)


def test_dssim_is_symmetric_and_bounded():
    rng = np.random.default_rng(3)
    Y, M = rng.random((2, 12, 15)), rng.random((2, 12, 15))
    a, b = oracle.dssim(Y, M, 1.0, with_grad=False)[0], oracle.dssim(M, Y, 1.0, with_grad=False)[0]
    assert a == pytest.approx(b, rel=1e-13)
    assert 0 < a < 2


def test_dssim_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    Y, M = rng.random((2, 9, 13)), rng.random((2, 9, 13))
    _, g = oracle.dssim(Y, M, 1.0)
    h = 1e-6
    for idx in [(0, 0, 0), (0, 4, 6), (1, 8, 12), (1, 2, 11), (0, 7, 1)]:
        Yp, Ym = Y.copy(), Y.copy()
        Yp[idx] += h
        Ym[idx] -= h
        fd = (oracle.dssim(Yp, M, 1.0, False)[0] - oracle.dssim(Ym, M, 1.0, False)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-10)


# ------------------------------------------------------------------- TV

def test_tv_of_constant_is_zero():
    V = np.full((10, 9, 8), 3.25)
    val, g = oracle.tv(V, 5, (1, 2, 3))
    assert val == 0.0 and not g.any()


def test_tv_of_a_linear_field_is_the_mean_slope():
    z, y, x = np.meshgrid(np.arange(12), np.arange(11), np.arange(10), indexing="ij")
    V = 0.5 * x - 2.0 * y + 0.25 * z
    assert oracle.tv(V, 6, (2, 1, 4), with_grad=False)[0] == pytest.approx((0.5 + 2.0 + 0.25) / 3, rel=1e-14)


def test_tv_matches_numpy_differences_and_ignores_voxels_outside_the_crop():
    rng = np.random.default_rng(5)
    V = rng.random((11, 12, 13))
    o, D = (3, 2, 4), 6
    c = V[o[2]:o[2] + D, o[1]:o[1] + D, o[0]:o[0] + D]
    ref = np.mean([np.abs(np.diff(c, axis=a)).mean() for a in (2, 1, 0)])
    val, g = oracle.tv(V, D, o)
    assert val == pytest.approx(ref, rel=1e-13)
    W = V.copy()
    W[0, 0, 0] += 7.0  # outside the crop
    assert oracle.tv(W, D, o, with_grad=False)[0] == val
    mask = np.zeros_like(V, dtype=bool)
    mask[o[2]:o[2] + D, o[1]:o[1] + D, o[0]:o[0] + D] = True
    assert not g[~mask].any()


def test_tv_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    V = rng.random((7, 8, 9))
    o, D = (1, 2, 1), 5
    _, g = oracle.tv(V, D, o)
    h = 1e-7  # random values: no difference is within h of zero
    for idx in [(1, 2, 1), (3, 4, 3), (5, 6, 5), (2, 5, 4)]:
        Vp, Vm = V.copy(), V.copy()
        Vp[idx] += h
        Vm[idx] -= h
        fd = (oracle.tv(Vp, D, o, False)[0] - oracle.tv(Vm, D, o, False)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6)


# ------------------------------------------------------- MBC normality

def test_normality_of_unit_components_is_zero():
    rng = np.random.default_rng(7)
    E = rng.normal(size=(3, 3, 4, 5, 6))
    E /= np.sqrt((E ** 2).sum(axis=(2, 3, 4), keepdims=True))
    val, g = oracle.mbc_normality(E)
    assert abs(val) < 1e-24 and np.abs(g).max() < 1e-12


def test_normality_of_scaled_unit_components():
    """E = c U with unit components: loss (c^2 - 1)^2 and gradient 4 (c^2 - 1) E / (3L)."""
    rng = np.random.default_rng(8)
    L, c = 2, 1.7
    U = rng.normal(size=(L, 3, 3, 4, 5))
    U /= np.sqrt((U ** 2).sum(axis=(2, 3, 4), keepdims=True))
    val, g = oracle.mbc_normality(c * U)
    assert val == pytest.approx((c * c - 1) ** 2, rel=1e-13)
    np.testing.assert_allclose(g, 4 * (c * c - 1) * c * U / (3 * L), rtol=1e-12)


def test_normality_gradient_matches_central_differences():
    rng = np.random.default_rng(9)
    E = rng.normal(size=(3, 3, 2, 3, 2)) * 0.3
    _, g = oracle.mbc_normality(E)
    h = 1e-6
    for idx in [(0, 0, 0, 0, 0), (1, 2, 1, 2, 1), (2, 1, 0, 1, 1)]:
        Ep, Em = E.copy(), E.copy()
        Ep[idx] += h
        Em[idx] -= h
        fd = (oracle.mbc_normality(Ep, False)[0] - oracle.mbc_normality(Em, False)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-7)
