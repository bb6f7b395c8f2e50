"""Central finite differences pin the oracle's adjoint: each Gaussian-parameter
gradient of the voxelizer (without truncation and at kappa = 3), and every
gradient of the whole forward model on the 16^3 / 200-Gaussian / 4-view
sub-problem (kappa = inf)."""
import copy

import numpy as np
import pytest

import oracle
from oracle import brute
from synth import Grid, fd_subproblem
from tests import oracle_chain


def _vox_loss(grid, m, s, q, v, G, kappa):
    return float((oracle.voxelize(grid, m, s, q, v, kappa) * G).sum())


def _inside_mask(grid, m, s, q, kappa):
    """Which (Gaussian, voxel) pairs lie inside the truncation ellipsoid
    q <= kappa^2, with q from a SciPy rotation and a NumPy matrix inverse."""
    xs = brute.centres(grid)
    out = []
    for g in range(len(m)):
        R = brute.rotation(q[g])
        A = np.linalg.inv(R @ np.diag(np.asarray(s[g], float) ** 2) @ R.T)
        d = xs - m[g]
        out.append(np.einsum("...i,ij,...j->...", d, A, d) <= kappa * kappa)
    return np.stack(out)


@pytest.mark.parametrize("kappa", [np.inf, 3.0])
def test_voxelize_backward_matches_central_differences(kappa):
    """At kappa = 3 the loss is only piecewise smooth: a pair whose q crosses
    kappa^2 adds or drops a term.  The seed is chosen so that no central
    difference moves any pair across the cutoff (checked below, independently of
    the oracle), so the differences see exactly the terms inside the ellipsoids,
    and the adjoint must drop the same ones -- the pairs outside the ellipsoid
    but inside its bounding box would otherwise add about 1% to the gradients."""
    grid = Grid(10, 9, 8, 2.0, 2.0, 2.5)
    rng = np.random.default_rng(31)
    Gn = 4
    m = (rng.random((Gn, 3)) - 0.5) * np.array([16, 14, 16])
    s = rng.uniform(2.0, 5.0, (Gn, 3))
    q = rng.normal(size=(Gn, 4)) * 1.3
    v = rng.normal(size=(Gn, 3))
    G = rng.normal(size=(3,) + grid.shape)
    dm, ds, dq, dv = oracle.voxelize_backward(grid, m, s, q, v, G, kappa)
    h = 1e-5
    if np.isfinite(kappa):
        inside = _inside_mask(grid, m, s, q, kappa)
        assert inside.any() and not inside.all()  # the cutoff removes pairs of the oracle's bounding boxes
    for name, arr, grad in (("mean", m, dm), ("scale", s, ds), ("quat", q, dq), ("value", v, dv)):
        for idx in np.ndindex(arr.shape):
            ap, am = arr.copy(), arr.copy()
            ap[idx] += h
            am[idx] -= h
            args_p = dict(m=m, s=s, q=q, v=v)
            args_m = dict(m=m, s=s, q=q, v=v)
            key = {"mean": "m", "scale": "s", "quat": "q", "value": "v"}[name]
            args_p[key], args_m[key] = ap, am
            if np.isfinite(kappa):
                assert np.array_equal(_inside_mask(grid, args_p["m"], args_p["s"], args_p["q"], kappa), inside)
                assert np.array_equal(_inside_mask(grid, args_m["m"], args_m["s"], args_m["q"], kappa), inside)
            fd = (_vox_loss(grid, **args_p, G=G, kappa=kappa) - _vox_loss(grid, **args_m, G=G, kappa=kappa)) / (2 * h)
            assert grad[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8), (name, idx)


def _perturbed(wl, which, level, idx, delta):
    w2 = copy.deepcopy(wl)
    if which == "coeff":
        c = w2.coeff.astype(np.float64)
        c[idx] += delta
        return w2, c
    gs = w2.ref if level is None else w2.mbc[level]
    arr = getattr(gs, which).astype(np.float64)
    arr[idx] += delta
    setattr(gs, which, arr)
    return w2, w2.coeff.astype(np.float64)


def test_full_chain_gradients_match_central_differences():
    """Loss = mean (Y - M)^2 of project(warp(V, combine(E, w))) with V, E
    voxelized from Gaussians; relative agreement <= 1e-3.  The loss is smooth
    in the reference Gaussians (warp and projector are linear in V), so those
    take h = 1e-3; it is only piecewise smooth in anything that moves the DVF
    (trilinear weights kink at voxel faces), so the coefficients and MBC
    Gaussians take h = 1e-5 in FP64 to keep the kink error out."""
    wl = fd_subproblem()
    meas = wl.measured
    loss, grads, _ = oracle_chain.step(wl, meas, kind=2, coeff=wl.coeff.astype(np.float64))
    rng = np.random.default_rng(5)
    checks = [("coeff", None, tuple(rng.integers(0, [4, 3, 3])), grads["coeff"])]
    for which, gi in (("mean", 0), ("scale", 1), ("quat", 2), ("value", 3)):
        checks.append((which, None, (int(rng.integers(0, 200)), int(rng.integers(0, 3 if which != "quat" else 4)) if which != "value" else 0), grads["ref"][gi]))
        lvl = int(rng.integers(0, 3))
        nlev = wl.mbc[lvl].g
        checks.append((which, lvl, (int(rng.integers(0, nlev)), int(rng.integers(0, 4 if which == "quat" else 3))), grads["mbc"][lvl][gi]))
    for which, lvl, idx, garr in checks:
        h = 1e-3 if (which != "coeff" and lvl is None) else 1e-5
        wp, cp = _perturbed(wl, which, lvl, idx, h)
        wm, cm = _perturbed(wl, which, lvl, idx, -h)
        lp, _, _ = oracle_chain.step(wp, meas, kind=2, coeff=cp)
        lm, _, _ = oracle_chain.step(wm, meas, kind=2, coeff=cm)
        fd = (lp - lm) / (2 * h)
        scale = max(abs(fd), 1e-3 * np.abs(garr).max())
        assert abs(garr[idx] - fd) <= 1e-3 * scale, (which, lvl, idx, garr[idx], fd)


def test_eq14_objective_gradients_match_central_differences():
    """The Stage 2-3 objective (Eq. 14): L1 + 0.25 D-SSIM + 1 L_MBC + 0.05 TV
    on an 8^3 crop.  L1, TV and the DVF are piecewise smooth, so every
    parameter takes h = 1e-5 in FP64 (no residual, voxel difference or sample
    position sits within that of a kink for these seeds)."""
    wl = fd_subproblem()
    # scale the MBC vectors so that ||e_{l,k}||^2 ~ 1.5: every term of the
    # objective is then O(1), and central differences resolve all of them
    E = oracle_chain.forward(wl)["E"]
    s = np.sqrt(1.5 / np.mean(np.sum(E.reshape(E.shape[0], 3, -1) ** 2, axis=2)))
    for m in wl.mbc:
        m.value = (m.value * s).astype(np.float32)
    meas = wl.measured
    q = dict(lambda_ssim=0.25, lambda_mbc=1.0, lambda_tv=0.05, data_range=float(meas.max() - meas.min()),
             tv_size=8, tv_origin=(3, 4, 5))
    coeff = wl.coeff.astype(np.float64)
    loss, grads, _ = oracle_chain.step(wl, meas, kind="eq14", coeff=coeff, eq14=q)
    rng = np.random.default_rng(6)
    checks = [("coeff", None, tuple(rng.integers(0, [4, 3, 3])), grads["coeff"])]
    for which, gi in (("mean", 0), ("scale", 1), ("value", 3)):
        checks.append((which, None, (int(rng.integers(0, 200)), int(rng.integers(0, 3)) if which != "value" else 0),
                       grads["ref"][gi]))
        lvl = int(rng.integers(0, 3))
        checks.append((which, lvl, (int(rng.integers(0, wl.mbc[lvl].g)), int(rng.integers(0, 3))), grads["mbc"][lvl][gi]))
    for which, lvl, idx, garr in checks:
        h = 1e-5
        wp, cp = _perturbed(wl, which, lvl, idx, h)
        wm, cm = _perturbed(wl, which, lvl, idx, -h)
        lp, _, _ = oracle_chain.step(wp, meas, kind="eq14", coeff=cp, eq14=q)
        lm, _, _ = oracle_chain.step(wm, meas, kind="eq14", coeff=cm, eq14=q)
        fd = (lp - lm) / (2 * h)
        scale = max(abs(fd), 1e-3 * np.abs(garr).max())
        assert abs(garr[idx] - fd) <= 1e-3 * scale, (which, lvl, idx, garr[idx], fd)
