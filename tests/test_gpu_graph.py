"""The whole forward + adjoint step captured in a CUDA graph replays to the
same bits as eager execution, batch after batch."""
import numpy as np
import pytest
import torch

from paper_2503_22139_gb300.pipeline import ForwardAdjoint, GraphedStep
from synth import small_workload
from tests.gpu_util import dev, gset, views

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager():
    wl = small_workload()
    mk = lambda: ForwardAdjoint(wl.grid, wl.det, gset(wl.ref, wl.kappa), [gset(m, wl.kappa) for m in wl.mbc],
                                batch=4)
    eager, cap = mk(), mk()
    batches = [(views(wl.views[i:i + 4]), dev(wl.coeff[i:i + 4]), dev(wl.measured[i:i + 4])) for i in (0, 4)]
    g = GraphedStep(cap, *batches[0])
    for b in batches + batches[::-1]:
        le = eager.run(*b).clone()
        lg = g.run(*b).clone()
        torch.cuda.synchronize()
        assert torch.equal(le, lg)
        for x, y in zip(eager.g_ref + eager.g_wc + tuple(t for m in eager.g_mbc for t in m),
                        cap.g_ref + cap.g_wc + tuple(t for m in cap.g_mbc for t in m)):
            assert torch.equal(x, y)
