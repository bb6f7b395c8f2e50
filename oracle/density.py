"""Adaptive density control of a Gaussian set (Sec. 2.3.2), plain NumPy.

TEST INFRASTRUCTURE ONLY: used by tests/, never by the library.  One Gaussian
at a time, in input order, following the rule of Sec. 2.3.2; where the paper
gives no statistic, threshold or split geometry, these readings fill them:

  * the densification statistic of a Gaussian is the mean, over the steps since
    the last control, of the Euclidean norm of dL/d(mean);
  * a Gaussian is empty, and removed, when every channel of its value has
    magnitude below value_threshold;
  * a Gaussian whose statistic exceeds grad_threshold is densified: cloned (two
    copies at the same place) when its largest scale is at most
    scale_threshold, otherwise split into two Gaussians whose means are drawn
    from the parent, mean + R diag(s) z_k with z_k the caller's standard-normal
    samples, and whose scales are s / split_factor;
  * the density of both Gaussians a densification leaves is half the parent's;
  * the output keeps the input order, a densified Gaussian's two results in
    place of it.
"""
from __future__ import annotations

import numpy as np

from .brute import rotation


def accumulate_grad_norm(acc, d_mean):
    """acc + |dL/dmean| per Gaussian."""
    return np.asarray(acc, np.float64) + np.linalg.norm(np.asarray(d_mean, np.float64).reshape(-1, 3), axis=1)


def densify_threshold(grad_acc, grad_scale, rank):
    """The densification threshold that leaves the `rank` largest statistics
    above it: the (rank + 1)-th largest of stat_i = grad_acc_i * grad_scale
    (0 <= rank < n).  The product and the order are taken in binary32, the
    precision in which the control compares stat_i with the threshold, so that
    both sides pick the same element."""
    stat = np.asarray(grad_acc, np.float32).reshape(-1) * np.float32(grad_scale)
    if not 0 <= rank < stat.size:
        raise ValueError("rank must be in [0, n)")
    return float(np.sort(stat)[::-1][rank])


def actions(scale, value, stat, grad_threshold, scale_threshold, value_threshold):
    """Per Gaussian: 0 remove, 1 keep, 2 clone, 3 split."""
    scale = np.asarray(scale, np.float64).reshape(-1, 3)
    value = np.asarray(value, np.float64).reshape(scale.shape[0], -1)
    out = np.ones(scale.shape[0], dtype=np.int64)
    for i in range(scale.shape[0]):
        if np.all(np.abs(value[i]) < value_threshold):
            out[i] = 0
        elif stat[i] > grad_threshold:
            out[i] = 2 if scale[i].max() <= scale_threshold else 3
    return out


def density_control(mean, scale, quat, value, grad_acc, grad_scale, noise, grad_threshold, scale_threshold,
                    value_threshold, split_factor=1.6):
    """Returns (mean, scale, quat, value) of the controlled set; grad_acc *
    grad_scale is the statistic (grad_scale = 1 / steps), noise [n][2][3]."""
    mean = np.asarray(mean, np.float64).reshape(-1, 3)
    n = mean.shape[0]
    scale = np.asarray(scale, np.float64).reshape(n, 3)
    quat = np.asarray(quat, np.float64).reshape(n, 4)
    value = np.asarray(value, np.float64).reshape(n, -1)
    noise = np.asarray(noise, np.float64).reshape(n, 2, 3)
    stat = np.asarray(grad_acc, np.float64).reshape(n) * grad_scale
    act = actions(scale, value, stat, grad_threshold, scale_threshold, value_threshold)
    om, osc, oq, ov = [], [], [], []
    for i in range(n):
        if act[i] == 0:
            continue
        if act[i] == 1:
            om.append(mean[i]); osc.append(scale[i]); oq.append(quat[i]); ov.append(value[i])
        elif act[i] == 2:
            for _ in range(2):
                om.append(mean[i]); osc.append(scale[i]); oq.append(quat[i]); ov.append(0.5 * value[i])
        else:
            R = rotation(quat[i])
            for k in range(2):
                om.append(mean[i] + R @ (scale[i] * noise[i, k]))
                osc.append(scale[i] / split_factor); oq.append(quat[i]); ov.append(0.5 * value[i])
    C = value.shape[1]
    as_arr = lambda xs, w: np.array(xs, dtype=np.float64).reshape(-1, w)
    return as_arr(om, 3), as_arr(osc, 3), as_arr(oq, 4), as_arr(ov, C)
