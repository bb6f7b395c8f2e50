"""GPU parity of the Eq. 13-14 terms (D-SSIM, sub-volume TV, MBC normality)
against the FP64 oracle on seeded inputs, several tiles with ragged edges,
through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from synth import Grid, measured_projections
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _projection_pair(P, nv, nu, seed):
    """Projection-like images: smooth positive fields around 200 plus noise."""
    rng = np.random.default_rng(seed)
    Y = measured_projections(rng, P, nu, nv, 300.0)
    M = Y + rng.normal(0.0, 5.0, Y.shape) + measured_projections(rng, P, nu, nv, 30.0)
    return Y.astype(np.float32), M.astype(np.float32)


@pytest.mark.parametrize("shape", [(3, 45, 70), (2, 384, 512)])
def test_dssim_matches_oracle(shape):
    P, nv, nu = shape
    Y, M = _projection_pair(P, nv, nu, 11)
    rng_ = float(M.max() - M.min())
    loss, g = pmf.projection_dssim(dev(Y), dev(M), rng_, weight=1.0)
    ref, gref = oracle.dssim(Y, M, rng_)
    # SSIM is formed per pixel in fp32 from moments about the tile mean: a few
    # ulps of S (~1e-7 each), averaged; the gradient meets the gradient bar
    assert abs(float(loss.item()) - ref) <= 2e-6
    assert rel_l2(host(g), gref) <= 1e-4


def test_dssim_identical_inputs_and_accumulate():
    Y, _ = _projection_pair(2, 40, 50, 12)
    loss, g = pmf.projection_dssim(dev(Y), dev(Y), 300.0)
    assert abs(float(loss.item())) <= 1e-6
    assert float(g.abs().max()) <= 1e-9
    # accumulate: loss += w * term and d_pred += w * d term
    _, M = _projection_pair(2, 40, 50, 13)
    base = torch.full((1,), 2.5, device="cuda")
    # a starting gradient of the term's own magnitude, so that fp32 addition
    # does not swamp the comparison
    g0 = np.random.default_rng(14).normal(0.0, 1e-6, (2, 40, 50)).astype(np.float32)
    gbase = dev(g0)
    pmf.projection_dssim(dev(Y), dev(M), 300.0, weight=0.25, loss=base, d_pred=gbase, accumulate=True)
    ref, gref = oracle.dssim(Y, M, 300.0)
    assert float(base.item()) == pytest.approx(2.5 + 0.25 * ref, abs=1e-6)
    assert rel_l2(host(gbase), g0 + 0.25 * gref) <= 1e-4


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_tv_matches_oracle_including_a_clamped_origin(dt):
    g = Grid(40, 36, 30, 2.0, 2.0, 2.0)
    V = np.random.default_rng(14).random(g.shape).astype(np.float32)
    Vd = dev(V).to(dt)
    Vq = host(Vd)  # the values the kernel reads
    for origin, clamped, D in [((5, 7, 9), (5, 7, 9), 16), ((-3, 100, 2), (0, 36 - 20, 2), 20)]:
        loss, gv = pmf.tv_loss(g, Vd, D, origin, weight=0.05)
        ref, gref = oracle.tv(Vq, D, clamped)
        assert float(loss.item()) == pytest.approx(0.05 * ref, rel=1e-5)
        # the subgradient is a signed count times a constant: exact up to its rounding
        assert rel_l2(host(gv), 0.05 * gref) <= 1e-6


def test_tv_accumulate_leaves_voxels_outside_the_crop():
    g = Grid(24, 24, 24, 2.0, 2.0, 2.0)
    V = dev(np.random.default_rng(15).random(g.shape))
    d = torch.full(g.shape, 3.0, device="cuda")
    pmf.tv_loss(g, V, 8, (2, 3, 4), weight=1.0, d_vol=d, accumulate=True)
    mask = torch.zeros(g.shape, dtype=torch.bool, device="cuda")
    mask[4:12, 3:11, 2:10] = True
    assert torch.all(d[~mask] == 3.0)
    assert not torch.all(d[mask] == 3.0)


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_mbc_normality_matches_oracle(dt):
    g = Grid(30, 28, 20, 2.0, 2.0, 2.0)
    L = 3
    E = (np.random.default_rng(16).normal(size=(L, 3) + g.shape) / np.sqrt(g.n)).astype(np.float32)
    E *= np.array([0.8, 1.0, 1.3])[None, :, None, None, None]
    Ed = dev(E).to(dt)
    Eq = host(Ed)
    loss, gE = pmf.mbc_normality(g, Ed, weight=1.0)
    ref, gref = oracle.mbc_normality(Eq)
    assert float(loss.item()) == pytest.approx(ref, rel=1e-5)
    assert rel_l2(host(gE), gref) <= 1e-5
