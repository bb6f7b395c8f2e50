"""The Stage 2-3 objective of Eq. 14 (L1 + 0.25 D-SSIM + 1 L_MBC + 0.05 TV) as
the GPU step computes it, against the oracle chain: loss and every gradient,
on the gradient-check sub-problem and on the small workload."""
import numpy as np
import pytest
import torch

import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300.pipeline import ForwardAdjoint
from synth import small_workload, fd_subproblem
from tests import oracle_chain
from tests.gpu_util import dev, gset, host, rel_l2, views

pytestmark = pytest.mark.gpu


def _normalise_mbc(wl):
    """Scale the MBC vectors so that ||e_{l,k}||^2 ~ 1.5 and every term of the
    objective is O(1)."""
    E = oracle_chain.forward(wl)["E"]
    s = np.sqrt(1.5 / np.mean(np.sum(E.reshape(E.shape[0], 3, -1) ** 2, axis=2)))
    for m in wl.mbc:
        m.value = (m.value * s).astype(np.float32)
    return wl


@pytest.mark.parametrize("make,tv", [(fd_subproblem, (8, (3, 4, 5))), (small_workload, (32, (10, 20, 5)))])
def test_eq14_step_matches_oracle(make, tv):
    wl = _normalise_mbc(make())
    meas = wl.measured
    q = dict(lambda_ssim=0.25, lambda_mbc=1.0, lambda_tv=0.05, data_range=float(meas.max() - meas.min()),
             tv_size=tv[0], tv_origin=tv[1])
    lref, gref, fref = oracle_chain.step(wl, meas, kind="eq14", eq14=q)
    step = ForwardAdjoint(wl.grid, wl.det, gset(wl.ref, wl.kappa), [gset(m, wl.kappa) for m in wl.mbc],
                          batch=wl.p, dtype=torch.float32, kind="eq14",
                          eq14=dict(data_range=q["data_range"], tv_size=tv[0]))
    origin = torch.tensor(tv[1], dtype=torch.int32, device="cuda")
    loss = step.run(views(wl.views), dev(wl.coeff), dev(meas), tv_origin=origin)
    torch.cuda.synchronize()
    assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
    assert rel_l2(host(step.Y), fref["Y"]) <= 1e-5
    assert rel_l2(host(step.g_wc[2]), gref["coeff"]) <= 1e-3
    assert rel_l2(host(step.g_wc[0]), gref["dV"]) <= 1e-3
    assert rel_l2(host(step.g_wc[1]), gref["dE"]) <= 1e-3
    for i in range(4):
        assert rel_l2(host(step.g_ref[i]), gref["ref"][i]) <= 1e-3
        for l in range(len(wl.mbc)):
            assert rel_l2(host(step.g_mbc[l][i]), gref["mbc"][l][i]) <= 1e-3
