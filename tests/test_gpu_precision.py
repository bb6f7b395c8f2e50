"""Reduced-precision storage (bf16 / fp16 for V, E, W; fp32 accumulation
everywhere): per-stage error of the whole forward + adjoint against the FP64
oracle on the small workload, twice.  (1) End to end: the oracle keeps every
tensor in FP64, so the error is the cost of storage; the bar on projections is
relative L2 <= 2e-3 and the stage errors are bounded by the storage format's
rounding.  (2) Storage only: the oracle rounds V, E (and W) to the same format
where the path stores them, so what remains is the kernels' own arithmetic,
held to the FP32 bars."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300.pipeline import ForwardAdjoint, PlainPerProjection
from synth import small_workload
from tests import oracle_chain
from tests.gpu_util import dev, gset, host, rel_l2, views

pytestmark = pytest.mark.gpu

# unit roundoff of the storage format (round to nearest even)
UNIT = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -11, torch.float32: 2.0 ** -24}
FMT = {torch.bfloat16: "bf16", torch.float16: "f16"}


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


def _rounding_interval(x, dt):
    """[round(x - d), round(x + d)] in the storage format, d the fp32 error
    allowed before storing: 1e-5 of the largest magnitude (the FP32 parity bar,
    as for the voxel checks) plus 8 fp32 units of x."""
    x = np.asarray(x, dtype=np.float64)
    d = 1e-5 * np.abs(x).max() + 8 * 2.0 ** -24 * np.abs(x)
    return oracle.round_storage(x - d, FMT[dt]), oracle.round_storage(x + d, FMT[dt])


@pytest.fixture(scope="module")
def wl_k5():
    """The small workload with the truncation radius raised to kappa = 5: a
    truncation tie then moves a voxel by at most max|value| e^{-12.5}, so the
    comparisons below see the storage rounding and the arithmetic alone."""
    wl = small_workload()
    wl.kappa = 5.0
    return wl


def _other_rounding(x, dt):
    """x rounded to the storage format, except that every element whose fp32
    error band (see _rounding_interval) straddles a rounding midpoint takes the
    other neighbour: the largest set of storage roundings in which a kernel
    that rounds its fp32 value can differ from the oracle's."""
    lo, hi = _rounding_interval(x, dt)
    r = oracle.round_storage(x, FMT[dt])
    return np.where(lo != r, lo, np.where(hi != r, hi, r))


@pytest.mark.parametrize("w_same", [False, True], ids=["W-fp32", "W-reduced"])
@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_storage_only_per_stage_error(wl_k5, dt, w_same):
    """The oracle rounds V and E (and W) to the storage format where the path
    stores them, so the stage errors below leave out the cost of storage.  The
    kernel rounds its fp32 value and the oracle its fp64 value, so a stored
    element is unique only up to the rounding of the fp32 error band around the
    oracle's value: every stored V and E element must lie in that interval, and
    the fraction rounded the other way is printed.  Those straddles then move
    every later stage a little; the oracle measures how much by rounding every
    straddle-able element the other way (a second oracle chain).  The
    projections and every gradient must hold the FP32 bars (1e-5 relative L2
    and 1e-3); W, which carries the straddles of V and E voxel by voxel, 1e-5
    plus that sensitivity (and the projections too when W itself is stored
    reduced)."""
    wl = wl_k5
    loss, grads, f = oracle_chain.step(wl, wl.measured, kind=2, storage=(FMT[dt], w_same))
    _, grads_alt, f_alt = oracle_chain.step(wl, wl.measured, kind=2,
                                            storage=(FMT[dt], w_same, lambda x: _other_rounding(x, dt)))
    step = _run(wl, dt, w_dtype=dt if w_same else torch.float32)
    e = stage_errors(wl, step, grads, f)
    # the same per-stage metrics between the two oracle chains: the straddle sensitivity
    sens = {k: rel_l2(a, b) for k, (a, b) in {
        "W": (f_alt["W"], f["W"]), "Y": (f_alt["Y"], f["Y"]), "dW": (grads_alt["dW"], grads["dW"]),
        "dV": (grads_alt["dV"], grads["dV"]), "dE": (grads_alt["dE"], grads["dE"]),
        "d_coeff": (grads_alt["coeff"], grads["coeff"]), "d_ref_mean": (grads_alt["ref"][0], grads["ref"][0]),
        "d_mbc_value": (grads_alt["mbc"][0][3], grads["mbc"][0][3])}.items()}
    straddles = {}
    for name, got, key in (("V", host(step.V[0]), "V"), ("E", host(step.E), "E")):
        lo, hi = _rounding_interval(f[key + "_unrounded"].reshape(got.shape), dt)
        assert np.all((lo <= got) & (got <= hi)), name
        straddles[name] = float(np.mean(got != f[key].reshape(got.shape)))
    print(FMT[dt], step.W.dtype, {k: f"{v:.2e}" for k, v in e.items()},
          "| stored elements rounded the other way", {k: f"{v:.1e}" for k, v in straddles.items()},
          "| straddle sensitivity", {k: f"{v:.1e}" for k, v in sens.items()})
    # W carries the straddles of V and E directly (and its own when it is stored
    # reduced); projections and gradients hold the plain FP32 bars
    assert e["W"] <= 1e-5 + sens["W"]
    assert e["Y"] <= 1e-5 + (sens["Y"] if w_same else 0.0)
    for k in ("dW", "dV", "dE", "d_coeff", "d_ref_mean", "d_mbc_value"):
        assert e[k] <= 1e-3, k


def test_plain_per_projection_path_without_truncation_ties(wl_k5):
    """fp32 storage at kappa = 5: every stage over all elements within the FP32
    bar (the kappa = 3 test above includes the truncation ties of V)."""
    loss, grads, f = oracle_chain.step(wl_k5, wl_k5.measured, kind=2)
    e = stage_errors(wl_k5, _run(wl_k5, torch.float32, PlainPerProjection), grads, f)
    print("plain f32, kappa 5", {k: f"{v:.2e}" for k, v in e.items()})
    for k in ("V", "E", "W", "Y"):
        assert e[k] <= 1e-5, k
    for k in ("dW", "dV", "dE", "d_coeff", "d_ref_mean", "d_mbc_value"):
        assert e[k] <= 1e-3, k
