"""The torch.autograd.Function wrappers route the hand-written adjoints:
loss.backward() through the whole forward model must reproduce the FP64
oracle's gradients (<= 1e-3 relative) for every Gaussian parameter and the
temporal coefficients."""
import numpy as np
import pytest
import torch

import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300 import autograd as pag
from synth import fd_subproblem
from tests import oracle_chain
from tests.gpu_util import dev, host, rel_l2, views

pytestmark = pytest.mark.gpu


def _leaf(a):
    return dev(a).requires_grad_(True)


@pytest.mark.parametrize("kind", [2, 1])
def test_autograd_chain_matches_oracle_gradients(kind):
    wl = fd_subproblem()
    ref = [_leaf(x) for x in (wl.ref.mean, wl.ref.scale, wl.ref.quat, wl.ref.value)]
    mbc = [[_leaf(x) for x in (m.mean, m.scale, m.quat, m.value)] for m in wl.mbc]
    coeff = _leaf(wl.coeff)
    Y, loss = pag.forward_model(wl.grid, wl.det, ref, mbc, coeff, views(wl.views), dev(wl.measured),
                                kappa=wl.kappa, kind=kind)
    loss.backward()
    lref, gref, fref = oracle_chain.step(wl, wl.measured, kind=kind)
    assert rel_l2(host(Y), fref["Y"]) <= 1e-5
    assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
    assert rel_l2(host(coeff.grad), gref["coeff"]) <= 1e-3
    for i in range(4):
        assert rel_l2(host(ref[i].grad), gref["ref"][i]) <= 1e-3, i
        for l in range(3):
            assert rel_l2(host(mbc[l][i].grad), gref["mbc"][l][i]) <= 1e-3, (l, i)


def test_autograd_shared_volume_projection_gradient():
    """d/dV of sum(w * project(V)) with one volume shared by all views equals
    the shared-volume adjoint."""
    wl = fd_subproblem()
    V = torch.rand(wl.grid.shape, device="cuda", requires_grad=True)
    vt = views(wl.views)
    Y = pag.conebeam_project(wl.grid, wl.det, vt, V, shared=True)
    wgt = torch.randn_like(Y)
    (Y * wgt).sum().backward()
    expect = pmf.conebeam_project_backward(wl.grid, wl.det, vt, wgt, shared=True)
    torch.testing.assert_close(V.grad, expect, rtol=0, atol=0)


def test_autograd_eq14_objective_matches_oracle_gradients():
    """loss.backward() of the Eq. 14 objective routes every term's adjoint."""
    wl = fd_subproblem()
    E = oracle_chain.forward(wl)["E"]
    s = np.sqrt(1.5 / np.mean(np.sum(E.reshape(E.shape[0], 3, -1) ** 2, axis=2)))
    for m in wl.mbc:
        m.value = (m.value * s).astype(np.float32)
    q = dict(lambda_ssim=0.25, lambda_mbc=1.0, lambda_tv=0.05,
             data_range=float(wl.measured.max() - wl.measured.min()), tv_size=8, tv_origin=(3, 4, 5))
    ref = [_leaf(x) for x in (wl.ref.mean, wl.ref.scale, wl.ref.quat, wl.ref.value)]
    mbc = [[_leaf(x) for x in (m.mean, m.scale, m.quat, m.value)] for m in wl.mbc]
    coeff = _leaf(wl.coeff)
    Y, loss = pag.forward_model(wl.grid, wl.det, ref, mbc, coeff, views(wl.views), dev(wl.measured),
                                kappa=wl.kappa, kind="eq14", eq14=q)
    loss.backward()
    lref, gref, _ = oracle_chain.step(wl, wl.measured, kind="eq14", eq14=q)
    assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
    assert rel_l2(host(coeff.grad), gref["coeff"]) <= 1e-3
    for i in range(4):
        assert rel_l2(host(ref[i].grad), gref["ref"][i]) <= 1e-3, i
        for l in range(3):
            assert rel_l2(host(mbc[l][i].grad), gref["mbc"][l][i]) <= 1e-3, (l, i)
