"""GPU parity of the Stage-1 X-ray rasterizer (Eq. 8-9) against the FP64 oracle
through the C ABI: whole projections at small sizes (several 16x16 tiles,
ragged detector edges, kappa = 3 and no truncation), sampled pixels and
sampled Gaussians' gradients at the paper scale (100,000 Gaussians, 512x384,
32 views), and the edge cases (empty sets, Gaussians behind the source or off
the detector, list overflow, reproducibility).  Forward bar: relative L2
<= 1e-5; gradients <= 1e-3."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from synth import Detector, Grid, circular_views, gaussian_set, paper_workload, select_batch, small_workload
from tests.gpu_util import dev, gset, host, pixel_views, rel_l2, views

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOLG = 1e-3


def _oracle(det, vw, gs, kappa):
    return oracle.splat(det.nu, det.nv, vw, gs.mean, gs.scale, gs.quat, gs.value, kappa)


@pytest.mark.parametrize("kappa", [3.0, float("inf")])
def test_rasterize_small_workload_matches_oracle(kappa):
    wl = small_workload(with_measured=False)  # 2,000 Gaussians, 8 views of 128^2
    Y = pmf.gs_rasterize(wl.det, views(wl.views), gset(wl.ref, kappa))
    assert rel_l2(host(Y), _oracle(wl.det, wl.views, wl.ref, kappa)) <= TOL32


def _edge_set():
    """Gaussians inside a small volume plus one behind the source of view 0,
    one far off every detector and one straddling the detector edge."""
    grid = Grid(40, 36, 30, 2.0, 2.0, 2.0)
    gs = gaussian_set(np.random.default_rng(21), grid, 300, 0.7, 3.0)
    vw = circular_views(3, 300.0, 450.0, 37, 29, 1.4, 1.4, start=0.3)
    extra = np.array([vw[0, 0:3] * 1.3, [900.0, -900.0, 0.0], [0.0, 0.0, 14.0]], dtype=np.float32)
    gs.mean = np.concatenate([gs.mean, extra]).astype(np.float32)
    gs.scale = np.concatenate([gs.scale, np.full((3, 3), 3.0, np.float32)])
    gs.quat = np.concatenate([gs.quat, np.tile(np.float32([1, 0, 0, 0]), (3, 1))])
    gs.value = np.concatenate([gs.value, np.ones((3, 1), np.float32)])
    return gs, vw, Detector(37, 29, 1.0)


def test_rasterize_ragged_detector_and_edge_gaussians():
    gs, vw, det = _edge_set()
    Y = pmf.gs_rasterize(det, views(vw), gset(gs, 3.0))
    assert rel_l2(host(Y), _oracle(det, vw, gs, 3.0)) <= TOL32


def test_rasterize_empty_and_zero_views():
    gs, vw, det = _edge_set()
    empty = pmf.Gaussians(torch.zeros((0, 3), device="cuda"), torch.zeros((0, 3), device="cuda"),
                          torch.zeros((0, 4), device="cuda"), torch.zeros((0, 1), device="cuda"), 3.0)
    Y = pmf.gs_rasterize(det, views(vw), empty)
    assert torch.equal(Y, torch.zeros_like(Y))
    Y0 = pmf.gs_rasterize(det, views(vw[:0]), gset(gs, 3.0))
    assert Y0.shape == (0, det.nv, det.nu)


def test_rasterize_list_overflow_and_reproducibility():
    """A pair list far too small: every tile scans all Gaussians (same bits,
    counted); and two launches give identical bits (integer pixel sums)."""
    wl = small_workload(with_measured=False)
    g = gset(wl.ref, 3.0)
    vw = views(wl.views)
    a = pmf.gs_rasterize(wl.det, vw, g)
    b = pmf.gs_rasterize(wl.det, vw, g)
    assert torch.equal(a, b)
    pmf.device_counters(reset=True)
    c = pmf.gs_rasterize(wl.det, vw, g, pair_capacity=1)
    assert torch.equal(a, c)
    assert pmf.device_counters()["raster_list_overflow"] > 0
    pmf.device_counters(reset=True)


def test_rasterize_nonfinite_parameter_poisons_its_views():
    gs, vw, det = _edge_set()
    g = gset(gs, 3.0)
    g.scale[5, 1] = float("nan")
    pmf.device_counters(reset=True)
    Y = pmf.gs_rasterize(det, views(vw), g)
    assert torch.isnan(Y).all()
    assert pmf.device_counters()["nonfinite"] > 0
    with pytest.raises(pmf.PmfError):
        pmf.device_status()
    pmf.device_counters(reset=True)


@pytest.mark.parametrize("kappa", [3.0, float("inf")])
def test_rasterize_backward_matches_oracle(kappa):
    gs, vw, det = _edge_set()
    dY = np.random.default_rng(22).normal(size=(len(vw), det.nv, det.nu)).astype(np.float32)
    got = pmf.gs_rasterize_backward(det, views(vw), gset(gs, kappa), dev(dY))
    ref = oracle.splat_backward(det.nu, det.nv, vw, gs.mean, gs.scale, gs.quat, gs.value, dY, kappa)
    for name, a, b in zip(("mean", "scale", "quat", "value"), got, ref):
        assert rel_l2(host(a).reshape(b.shape), b) <= TOLG, name
    # the value gradient is a plain weighted pixel sum
    assert rel_l2(host(got[3]).reshape(-1), ref[3]) <= TOL32


def test_rasterize_backward_accumulates_and_is_reproducible():
    gs, vw, det = _edge_set()
    g = gset(gs, 3.0)
    dY = dev(np.random.default_rng(23).normal(size=(len(vw), det.nv, det.nu)))
    a = pmf.gs_rasterize_backward(det, views(vw), g, dY)
    b = pmf.gs_rasterize_backward(det, views(vw), g, dY)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    base = [torch.full_like(t, 0.5) for t in a]
    pmf.gs_rasterize_backward(det, views(vw), g, dY, grads=base, accumulate=True)
    for x, y in zip(base, a):
        assert torch.allclose(x, y + 0.5, rtol=0, atol=1e-5 * (1 + float(y.abs().max())))


@pytest.fixture(scope="module")
def paper():
    wl = paper_workload(p=660)
    idx = select_batch(wl.p, 32, 0)
    return wl, wl.views[idx]


def test_rasterize_paper_scale_sampled_pixels(paper):
    """The benchmark's Stage-1 launch (100,000 Gaussians, 32 views of 512x384):
    64 sampled pixels against the oracle, one 1x1 view per pixel."""
    wl, vw = paper
    Y = host(pmf.gs_rasterize(wl.det, views(vw), gset(wl.ref, wl.kappa)))
    rng = np.random.default_rng(24)
    pix = [(int(rng.integers(0, 32)), int(rng.integers(0, wl.det.nv)), int(rng.integers(0, wl.det.nu)))
           for _ in range(64)]
    ref = oracle.splat(1, 1, pixel_views(vw, wl.det.nu, wl.det.nv, pix), wl.ref.mean, wl.ref.scale, wl.ref.quat,
                       wl.ref.value, wl.kappa)[:, 0, 0]
    got = np.array([Y[p, b, a] for p, b, a in pix])
    assert rel_l2(got, ref) <= TOL32


def test_rasterize_paper_scale_gradients(paper):
    """The adjoint at the paper scale: <dY, Y> = sum_g rho_g dL/drho_g (Y is
    linear in the densities) over the whole batch, and 48 sampled Gaussians'
    gradients against the oracle (a Gaussian's gradient depends only on its own
    parameters and dY)."""
    wl, vw = paper
    g = gset(wl.ref, wl.kappa)
    Y = pmf.gs_rasterize(wl.det, views(vw), g)
    dY = torch.randn(Y.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(25))
    grads = pmf.gs_rasterize_backward(wl.det, views(vw), g, dY)
    lhs = float((dY.double() * Y.double()).sum())
    rhs = float((g.value.double().reshape(-1) * grads[3].double().reshape(-1)).sum())
    assert rhs == pytest.approx(lhs, rel=1e-5)
    sel = np.random.default_rng(26).choice(wl.ref.mean.shape[0], 48, replace=False)
    ref = oracle.splat_backward(wl.det.nu, wl.det.nv, vw, wl.ref.mean[sel], wl.ref.scale[sel], wl.ref.quat[sel],
                                wl.ref.value[sel], host(dY), wl.kappa)
    for name, a, b in zip(("mean", "scale", "quat", "value"), grads, ref):
        assert rel_l2(host(a)[sel].reshape(b.shape), b) <= TOLG, name
