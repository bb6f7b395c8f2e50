"""Adaptive density control (Sec. 2.3.2) on the GPU against the oracle's rule
(removal, clones, splits, half densities, input order), the gradient-norm
accumulator, and the two-resolution Stage 2-3 schedule that drives them."""
import numpy as np
import pytest
import torch

import paper_2503_22139_gb300 as pmf
from oracle import density
from paper_2503_22139_gb300.pipeline import TwoResolutionSchedule
from synth import Grid, gaussian_set, small_workload
from tests.gpu_util import dev, gset, host, rel_l2, views

pytestmark = pytest.mark.gpu


def _mixed(seed, G, C):
    grid = Grid(40, 36, 30, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(seed)
    gs = gaussian_set(rng, grid, G, 0.5, 3.0, channels=C, value_std=None if C == 1 else 1.0)
    gs.value[rng.random(G) < 0.15] *= 1e-4           # some nearly empty
    acc = rng.uniform(0.0, 2.0, G).astype(np.float32)   # statistic acc / steps with steps = 4
    acc[np.abs(acc / 4 - 0.3) < 1e-3] += 0.01          # no statistic within rounding of the threshold
    noise = rng.normal(size=(G, 2, 3)).astype(np.float32)
    return gs, acc, noise


@pytest.mark.parametrize("C", [1, 3])
def test_density_control_matches_the_oracle(C):
    gs, acc, noise = _mixed(31 + C, 3000, C)
    thr, clone_s, prune = 0.3, 2.5, 1e-3
    got = pmf.gs_density_control(gset(gs, 3.0), dev(acc), 4, dev(noise), thr, clone_s, prune, 1.6)
    ref = density.density_control(gs.mean, gs.scale, gs.quat, gs.value, acc, 0.25, noise, thr, clone_s, prune, 1.6)
    act = density.actions(gs.scale, gs.value, acc.astype(np.float64) * 0.25, thr, clone_s, prune)
    assert set(act) == {0, 1, 2, 3}
    assert got.n == len(ref[0])
    # quaternions and values are copied or halved exactly; split scales are one
    # fp32 division and split means fp32 sums
    np.testing.assert_allclose(host(got.scale), ref[1], rtol=1e-6, atol=0)
    np.testing.assert_array_equal(host(got.quat), ref[2].astype(np.float32))
    np.testing.assert_array_equal(host(got.value), ref[3].astype(np.float32))
    assert rel_l2(host(got.mean), ref[0]) <= 1e-6


def test_density_control_is_deterministic_and_accumulates_gradient_norms():
    gs, acc, noise = _mixed(35, 2000, 1)
    g = gset(gs, 3.0)
    a = pmf.gs_density_control(g, dev(acc), 4, dev(noise), 0.3, 2.5, 1e-3)
    b = pmf.gs_density_control(g, dev(acc), 4, dev(noise), 0.3, 2.5, 1e-3)
    for x, y in zip((a.mean, a.scale, a.quat, a.value), (b.mean, b.scale, b.quat, b.value)):
        assert torch.equal(x, y)
    d = np.random.default_rng(36).normal(size=(2000, 3)).astype(np.float32)
    t = dev(np.full(2000, 0.5, np.float32))
    pmf.gs_grad_norm_accumulate(dev(d), t)
    np.testing.assert_allclose(host(t), density.accumulate_grad_norm(np.full(2000, 0.5), d), rtol=1e-6)


@pytest.mark.parametrize("n", [1, 7, 3000, 150_000])
def test_densify_threshold_matches_the_oracle_bit_for_bit(n):
    """The device radix select against the oracle's binary32 sort, over ranks
    from the top to the bottom, with exponential statistics, repeated values,
    zeros and one huge value."""
    rng = np.random.default_rng(40 + n)
    acc = rng.exponential(1.0, n).astype(np.float32)
    if n > 10:
        acc[rng.integers(0, n, n // 10)] = acc[0]   # ties
        acc[rng.integers(0, n, n // 20)] = 0.0
        acc[n // 2] = 3.0e38
    d = dev(acc)
    for rank in sorted({0, 1, n // 50, n // 2, n - 1} & set(range(n))):
        got = float(pmf.gs_density_threshold(d, 9, rank).item())
        assert got == density.densify_threshold(acc, np.float32(1.0 / 9), rank), rank


def test_two_resolution_schedule_runs_both_stages_with_control():
    """Stage 2 on 32^3 at 8 mm (batches of 8), Stage 3 on 64^3 at 4 mm (batches
    of 4), density control every 3 steps: every loss finite, the sets change
    size at each control, the loss falls within each stage."""
    wl = small_workload(with_measured=True)
    ref, mbc = gset(wl.ref, wl.kappa), [gset(m, wl.kappa) for m in wl.mbc]
    sched = TwoResolutionSchedule(wl.grid, wl.det, ref, mbc, views(wl.views), dev(wl.coeff), dev(wl.measured),
                                  steps=(7, 7), batches=(8, 4), kind=2,
                                  control=dict(every=3, densify_fraction=0.05, clone_scale_mm=6.0, prune_value=0.02))
    hist = sched.run()
    assert len(hist) == 14 and all(np.isfinite(l) for _, _, l in hist)
    assert len(sched.counts) == 4  # after steps 3 and 6 of each stage
    n0 = wl.ref.mean.shape[0]
    assert sched.counts[0][0] != n0
    for st in (0, 1):
        ls = [l for s, _, l in hist if s == st]
        assert min(ls[1:]) < ls[0]
    assert sched.step.V.shape[-3:] == (64, 64, 64)
