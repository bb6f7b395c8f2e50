"""Pins of the oracle's adaptive density control (Sec. 2.3.2) against things
other than itself: a clone leaves the voxelized volume unchanged (the C
oracle's voxelizer), pruning removes exactly the pruned Gaussians' share of the
volume (linearity), split children lie at Mahalanobis distance |z| from the
parent (a NumPy matrix inverse), and the counts and order of the output."""
import numpy as np
import pytest

import oracle
from oracle import density
from synth import Grid, gaussian_set

GRID = Grid(20, 18, 16, 2.0, 2.0, 2.0)


def _set(seed, G=40, C=1):
    gs = gaussian_set(np.random.default_rng(seed), GRID, G, 0.8, 2.5, channels=C, value_std=None if C == 1 else 1.0)
    return gs.mean.astype(np.float64), gs.scale.astype(np.float64), gs.quat.astype(np.float64), \
        gs.value.astype(np.float64)


def _vox(m, s, q, v, C=1):
    return oracle.voxelize(GRID, m, s, q, v.reshape(-1, C), kappa=np.inf)


def test_grad_norm_accumulation():
    d = np.random.default_rng(1).normal(size=(7, 3))
    acc = density.accumulate_grad_norm(np.full(7, 0.25), d)
    assert np.allclose(acc, 0.25 + np.sqrt((d ** 2).sum(1)), rtol=0, atol=1e-15)


def test_clones_leave_the_volume_unchanged():
    m, s, q, v = _set(2)
    stat = np.full(len(m), 1.0)
    out = density.density_control(m, s, q, v, stat, 1.0, np.zeros((len(m), 2, 3)), grad_threshold=0.5,
                                  scale_threshold=100.0, value_threshold=0.0)
    assert len(out[0]) == 2 * len(m)
    np.testing.assert_allclose(_vox(*out), _vox(m, s, q, v), rtol=1e-12, atol=1e-14)


def test_pruning_removes_exactly_the_empty_gaussians():
    m, s, q, v = _set(3)
    v[::3] *= 1e-4  # every third Gaussian is nearly empty
    tau = 1e-3
    out = density.density_control(m, s, q, v, np.zeros(len(m)), 1.0, np.zeros((len(m), 2, 3)), grad_threshold=1.0,
                                  scale_threshold=0.0, value_threshold=tau)
    empty = np.abs(v[:, 0]) < tau
    assert len(out[0]) == len(m) - empty.sum()
    np.testing.assert_allclose(_vox(m, s, q, v) - _vox(*out), _vox(m[empty], s[empty], q[empty], v[empty]),
                               rtol=0, atol=1e-13)


def test_multichannel_values_are_empty_only_when_every_channel_is():
    m, s, q, v = _set(4, G=6, C=3)
    v[:] = 1e-6
    v[2, 1] = 0.5  # one large component keeps Gaussian 2
    act = density.actions(s, v, np.zeros(6), 1.0, 0.0, 1e-3)
    assert list(act) == [0, 0, 1, 0, 0, 0]


def test_split_children_sit_at_mahalanobis_distance_z():
    m, s, q, v = _set(5, G=12)
    z = np.random.default_rng(6).normal(size=(12, 2, 3))
    out = density.density_control(m, s, q, v, np.full(12, 3.0), 1.0, z, grad_threshold=1.0, scale_threshold=0.0,
                                  value_threshold=0.0, split_factor=1.6)
    om, osc, oq, ov = out
    assert len(om) == 24
    for i in range(12):
        R = oracle.quat_to_rot(q[i])
        Sinv = np.linalg.inv(R @ np.diag(s[i] ** 2) @ R.T)
        for k in range(2):
            d = om[2 * i + k] - m[i]
            assert d @ Sinv @ d == pytest.approx(z[i, k] @ z[i, k], rel=1e-10)
            np.testing.assert_allclose(osc[2 * i + k], s[i] / 1.6, rtol=1e-15)
            np.testing.assert_array_equal(oq[2 * i + k], q[i])
            assert ov[2 * i + k, 0] == 0.5 * v[i, 0]
        # the children are antipodal when z_1 = -z_0: their mean is the parent's
    zz = np.concatenate([z[:, :1], -z[:, :1]], axis=1)
    om2 = density.density_control(m, s, q, v, np.full(12, 3.0), 1.0, zz, 1.0, 0.0, 0.0)[0]
    np.testing.assert_allclose(0.5 * (om2[0::2] + om2[1::2]), m, rtol=0, atol=1e-12)


def test_mixed_actions_keep_input_order():
    m, s, q, v = _set(7, G=10)
    s[:5] *= 0.1  # small: cloned when densified
    stat = np.array([0, 2, 0, 2, 0, 2, 0, 2, 0, 2], dtype=np.float64)
    v[0] = 0.0  # empty: removed
    act = density.actions(s, v, stat, 1.0, float(s[:5].max()), 1e-6)
    assert list(act) == [0, 2, 1, 2, 1, 3, 1, 3, 1, 3]
    out = density.density_control(m, s, q, v, stat, 1.0, np.zeros((10, 2, 3)), 1.0, float(s[:5].max()), 1e-6)
    expect = [1, 1, 2, 3, 3, 4, 5, 5, 6, 7, 7, 8, 9, 9]  # source Gaussian of every output, in order
    np.testing.assert_array_equal(out[2], q[expect])


def test_densify_threshold_is_the_order_statistic():
    """The threshold leaves exactly `rank` statistics above it when they are
    distinct, is itself one of the statistics, and at ties leaves fewer; the
    statistics are binary32 products (the precision of the control's test)."""
    rng = np.random.default_rng(3)
    acc = rng.exponential(1.0, 5000).astype(np.float32)
    scale = 1.0 / 7.0
    stat = acc * np.float32(scale)
    for rank in (0, 1, 99, 2500, 4999):
        t = density.densify_threshold(acc, scale, rank)
        assert np.float32(t) in stat
        assert int(np.sum(stat > np.float32(t))) == rank
        assert int(np.sum(stat >= np.float32(t))) >= rank + 1
    tied = np.repeat(np.float32([3.0, 2.0, 1.0]), [5, 5, 5])
    assert density.densify_threshold(tied, 1.0, 7) == 2.0      # ranks 5-9 share 2.0
    assert int(np.sum(tied > 2.0)) == 5                        # fewer than 7 lie above it
    assert density.densify_threshold(tied, 1.0, 0) == 3.0
    with pytest.raises(ValueError):
        density.densify_threshold(tied, 1.0, 15)
