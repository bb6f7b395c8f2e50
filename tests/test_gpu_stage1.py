"""The Stage-1 training step of Sec. 2.3.2 (Eq. 10-11: Gaussian-splatting
rasterizer, L1 + 0.25 D-SSIM, 0.05 TV of a voxelized 32^3 crop) against the FP64
oracle chain, and the shifted-mean crop voxelization against a crop of the
whole-grid voxelization."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300.pipeline import GraphedStage1, Stage1Step
from synth import Grid, small_workload
from tests.gpu_util import dev, gset, host, rel_l2, views

pytestmark = pytest.mark.gpu


def test_crop_voxelization_equals_a_crop_of_the_whole_grid():
    wl = small_workload(with_measured=False)  # 64^3 @ 4 mm
    g = gset(wl.ref, wl.kappa)
    full = pmf.gs_voxelize(wl.grid, g)[0]
    D, corner = 16, (5, 30, 41)
    centre = Stage1Step.crop_centre(wl.grid, corner, D).cuda()
    shifted = pmf.ops.pmf_shift_means(g.mean, centre)
    crop = pmf.gs_voxelize((D, D, D, 4.0, 4.0, 4.0), pmf.Gaussians(shifted, g.scale, g.quat, g.value, g.kappa))[0]
    ref = full[corner[2]:corner[2] + D, corner[1]:corner[1] + D, corner[0]:corner[0] + D]
    assert rel_l2(host(crop), host(ref)) <= 1e-5
    assert torch.equal(shifted, g.mean - centre)


def test_stage1_step_matches_the_oracle_chain():
    wl = small_workload(with_measured=True)  # 2,000 Gaussians, 8 views of 128^2, 64^3 @ 4 mm
    g = gset(wl.ref, wl.kappa)
    meas = wl.measured.astype(np.float32)
    drange = float(meas.max() - meas.min())
    D, corner = 32, (7, 19, 3)
    step = Stage1Step(wl.grid, wl.det, g, batch=wl.p, data_range=drange)
    centre = Stage1Step.crop_centre(wl.grid, corner, D)
    lp, ltv = step.run(views(wl.views), dev(meas), centre.cuda())
    torch.cuda.synchronize()
    # oracle: L1 + 0.25 D-SSIM of the rasterized projections, 0.05 TV of the crop
    m = wl.ref
    Y = oracle.splat(wl.det.nu, wl.det.nv, wl.views, m.mean, m.scale, m.quat, m.value, wl.kappa)
    l1, dY = oracle.loss(1, Y, meas)
    ds, dds = oracle.dssim(Y, meas, drange)
    sh = m.mean.astype(np.float64) - centre.numpy().astype(np.float64)
    crop = Grid(D, D, D, 4.0, 4.0, 4.0)
    Vc = oracle.voxelize(crop, sh, m.scale, m.quat, m.value, wl.kappa)[0]
    tv, dtv = oracle.tv(Vc, D, (0, 0, 0))
    assert float(lp.item()) == pytest.approx(l1 + 0.25 * ds, rel=1e-5)
    assert float(ltv.item()) == pytest.approx(0.05 * tv, rel=1e-5)
    assert rel_l2(host(step.Y), Y) <= 1e-5
    gr = oracle.splat_backward(wl.det.nu, wl.det.nv, wl.views, m.mean, m.scale, m.quat, m.value, dY + 0.25 * dds,
                               wl.kappa)
    gv = oracle.voxelize_backward(crop, sh, m.scale, m.quat, m.value, 0.05 * dtv[None], wl.kappa)
    for k, name in enumerate(("mean", "scale", "quat", "value")):
        ref = gr[k].reshape(-1) + gv[k].reshape(-1)
        assert rel_l2(host(step.grads[k]).reshape(-1), ref) <= 1e-3, name


def test_graphed_stage1_replays_equal_the_eager_steps():
    """The CUDA-graph replay of the Stage-1 step gives the eager step's losses
    and gradients bit for bit, with the views, measured projections and crop
    changing between replays (batch 1, as Stage 1 runs in the paper)."""
    wl = small_workload(with_measured=True)
    g = gset(wl.ref, wl.kappa)
    meas = dev(wl.measured.astype(np.float32))
    drange = float(wl.measured.max() - wl.measured.min())
    vw = views(wl.views)
    corners = [(7, 19, 3), (30, 2, 11), (0, 31, 25)]
    centres = [Stage1Step.crop_centre(wl.grid, c, 32).cuda() for c in corners]
    eager = Stage1Step(wl.grid, wl.det, g, batch=1, data_range=drange)
    graphed = GraphedStage1(Stage1Step(wl.grid, wl.det, g, batch=1, data_range=drange), vw[:1], meas[:1], centres[0])
    for k in range(len(corners)):
        p = 3 * k + 1
        le, te = [t.clone() for t in eager.run(vw[p:p + 1], meas[p:p + 1], centres[k])]
        ge = [t.clone() for t in eager.grads]
        lg, tg = graphed.run(vw[p:p + 1], meas[p:p + 1], centres[k])
        torch.cuda.synchronize()
        assert torch.equal(le, lg) and torch.equal(te, tg) and torch.isfinite(le).all()
        for a, b in zip(ge, graphed.grads):
            assert torch.equal(a, b)
