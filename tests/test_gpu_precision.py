"""Reduced-precision storage (bf16 / fp16 for V, E, W; fp32 accumulation
everywhere): per-stage error of the whole forward + adjoint against the FP64
oracle on the small workload.  The bar on projections is relative L2 <= 2e-3;
the stage errors are bounded by the storage format's rounding."""
import numpy as np
import pytest
import torch

import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300.pipeline import ForwardAdjoint, PlainPerProjection
from synth import small_workload
from tests import oracle_chain
from tests.gpu_util import dev, gset, host, rel_l2, views

pytestmark = pytest.mark.gpu

# unit roundoff of the storage format (round to nearest even)
UNIT = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -11, torch.float32: 2.0 ** -24}


@pytest.fixture(scope="module")
def ref_step():
    wl = small_workload()
    loss, grads, f = oracle_chain.step(wl, wl.measured, kind=2)
    return wl, loss, grads, f


def stage_errors(wl, step, grads, f):
    return {
        "V": rel_l2(host(step.V[0]), f["V"]),
        "E": rel_l2(host(step.E), f["E"]),
        "W": rel_l2(host(step.W), f["W"]),
        "Y": rel_l2(host(step.Y), f["Y"]),
        "dW": rel_l2(host(step.dW), grads["dW"]),
        "dV": rel_l2(host(step.g_wc[0]), grads["dV"]),
        "dE": rel_l2(host(step.g_wc[1]), grads["dE"]),
        "d_coeff": rel_l2(host(step.g_wc[2]), grads["coeff"]),
        "d_ref_mean": rel_l2(host(step.g_ref[0]), grads["ref"][0]),
        "d_mbc_value": rel_l2(host(step.g_mbc[0][3]), grads["mbc"][0][3]),
    }


def _run(wl, dt, cls=ForwardAdjoint, w_dtype=torch.float32):
    step = cls(wl.grid, wl.det, gset(wl.ref, wl.kappa), [gset(m, wl.kappa) for m in wl.mbc], batch=wl.p, dtype=dt,
               w_dtype=w_dtype)
    step.run(views(wl.views), dev(wl.coeff), dev(wl.measured))
    torch.cuda.synchronize()
    return step


@pytest.mark.parametrize("w_same", [False, True], ids=["W-fp32", "W-reduced"])
@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_reduced_storage_per_stage_error(ref_step, dt, w_same):
    """V and E in bf16 / fp16; W in fp32 (the default) or in the same format."""
    wl, loss, grads, f = ref_step
    step = _run(wl, dt, w_dtype=dt if w_same else torch.float32)
    assert step.W.dtype == (dt if w_same else torch.float32)
    e = stage_errors(wl, step, grads, f)
    print(dt, step.W.dtype, {k: f"{v:.2e}" for k, v in e.items()})
    u = UNIT[dt]
    assert e["Y"] <= 2e-3
    # storing a value rounds it by at most u relative, so rel-L2 <= u (truncation ties aside)
    assert e["V"] <= u and e["E"] <= u
    assert e["W"] <= 2 * u
    for k in ("dW", "dV", "dE", "d_coeff", "d_ref_mean", "d_mbc_value"):
        assert e[k] <= max(10 * u, 1e-3), k


def test_plain_per_projection_path_matches_oracle(ref_step):
    wl, loss, grads, f = ref_step
    e = stage_errors(wl, _run(wl, torch.float32, PlainPerProjection), grads, f)
    print("plain f32", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["Y"] <= 1e-5 and e["W"] <= 1e-4
    for k in ("dW", "dV", "dE", "d_coeff", "d_ref_mean", "d_mbc_value"):
        assert e[k] <= 1e-3, k
