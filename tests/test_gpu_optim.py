"""The Adam update kernel against torch.optim.Adam (a library reference of the
same rule), and a short optimisation on the small workload: fitting Gaussian
parameters to the projections of a ground-truth set through the whole
forward + adjoint step lowers the loss."""
import numpy as np
import pytest
import torch

import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300.pipeline import ForwardAdjoint
from synth import small_workload
from tests.gpu_util import dev, gset, views

pytestmark = pytest.mark.gpu


def test_adam_matches_torch_optim_adam():
    gen = torch.Generator("cuda").manual_seed(3)
    p0 = torch.randn(10007, device="cuda", generator=gen)
    grads = [torch.randn(10007, device="cuda", generator=gen) * (k + 1) for k in range(6)]
    ours, ref = p0.clone(), p0.clone().requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    st = pmf.Adam([ours], lr=0.01)
    for g in grads:
        st.step([g])
        ref.grad = g.clone()
        opt.step()
    torch.testing.assert_close(ours, ref.detach(), rtol=1e-5, atol=1e-6)


def test_adam_fit_to_ground_truth_projections_lowers_the_loss():
    wl = small_workload()
    gt = gset(wl.ref, wl.kappa)
    mbc = [gset(m, wl.kappa) for m in wl.mbc]
    vt, coeff = views(wl.views), dev(wl.coeff)
    E = torch.stack([pmf.gs_voxelize(wl.grid, m) for m in mbc])
    meas = pmf.conebeam_project(wl.grid, wl.det, vt, pmf.warp_combine(wl.grid, pmf.gs_voxelize(wl.grid, gt)[0], E,
                                                                       coeff), shared=False)
    # start from the ground truth with densities scaled by 0.7 and shifted centres
    rng = np.random.default_rng(9)
    start = pmf.Gaussians(dev(wl.ref.mean + rng.normal(0, 0.5, wl.ref.mean.shape)), dev(wl.ref.scale),
                          dev(wl.ref.quat), dev(wl.ref.value * 0.7), wl.kappa)
    step = ForwardAdjoint(wl.grid, wl.det, start, mbc, batch=wl.p, dtype=torch.bfloat16)
    opt = pmf.Adam([start.value, start.mean], lr=[0.01, 0.05])
    losses = []
    for _ in range(30):
        loss = step.run(vt, coeff, meas)
        losses.append(float(loss.item()))
        opt.step([step.g_ref[3], step.g_ref[0]])
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], losses
