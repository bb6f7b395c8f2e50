"""Uneven batched launches: volumes of different grids, detectors and view
counts in one persistent projector (and adjoint) launch give exactly the
per-volume results, and match the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from synth import Detector, Grid, circular_views
from tests.gpu_util import dev, host, rel_l2, views

pytestmark = pytest.mark.gpu


def _items(dtype=torch.float32):
    rng = np.random.default_rng(90)
    spec = [(Grid(20, 18, 14, 2.0, 2.0, 2.5), Detector(37, 23, 1.0), 3, False),
            (Grid(32, 32, 16, 2.0, 2.0, 2.0), Detector(48, 40, 1.0), 5, True),
            (Grid(24, 20, 12, 3.0, 2.0, 2.0), Detector(20, 52, 1.2), 2, False),
            (Grid(16, 16, 16, 1.0, 1.0, 1.0), Detector(16, 16, 0.5), 1, False)]
    items = []
    for k, (g, d, P, shared) in enumerate(spec):
        vw = circular_views(P, 300.0 + 50 * k, 450.0 + 60 * k, d.nu, d.nv, 1.7, 1.9, start=0.2 * k)
        vol = rng.random(g.shape if shared else (P,) + g.shape).astype(np.float32)
        items.append((g, d, vw, vol, shared))
    return items


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_batched_projection_equals_per_volume_launches(dt):
    items = _items()
    batched = pmf.ops.conebeam_project_batched([(g, d, views(vw), dev(vol).to(dt), sh) for g, d, vw, vol, sh in items])
    for (g, d, vw, vol, sh), yb in zip(items, batched):
        ys = pmf.conebeam_project(g, d, views(vw), dev(vol).to(dt), shared=sh)
        assert torch.equal(yb, ys)
        if dt == torch.float32:
            assert rel_l2(host(yb), oracle.project(g, d.nu, d.nv, d.step_mm, vw, vol, shared=sh)) <= 1e-5


def test_batched_projection_mixed_staging_and_empty_items():
    """fp32 batches take bulk-copy staging only when every item's rows are
    16-byte multiples: one item with nx = 21 sends the whole batch to plain
    staging, and an item with no views is skipped; both give the per-volume
    results bit for bit."""
    items = _items()
    rng = np.random.default_rng(92)
    g = Grid(21, 15, 11, 2.0, 2.0, 2.0)
    d = Detector(30, 26, 1.0)
    vw = circular_views(3, 320.0, 470.0, d.nu, d.nv, 1.7, 1.9, start=0.4)
    items.append((g, d, vw, rng.random((3,) + g.shape).astype(np.float32), False))
    for batch in (items, items[:2] + [(items[2][0], items[2][1], items[2][2][:0], items[2][3][:0], False)]):
        got = pmf.ops.conebeam_project_batched([(g_, d_, views(vw_), dev(vol), sh) for g_, d_, vw_, vol, sh in batch])
        for (g_, d_, vw_, vol, sh), yb in zip(batch, got):
            if vw_.shape[0] == 0:
                assert yb.numel() == 0
                continue
            assert torch.equal(yb, pmf.conebeam_project(g_, d_, views(vw_), dev(vol), shared=sh))


def test_batched_backprojection_equals_per_volume_launches():
    items = _items()
    rng = np.random.default_rng(91)
    dys = [rng.normal(size=(vw.shape[0], d.nv, d.nu)).astype(np.float32) for g, d, vw, vol, sh in items]
    batched = pmf.ops.conebeam_project_backward_batched(
        [(g, d, views(vw), dev(dy), sh) for (g, d, vw, vol, sh), dy in zip(items, dys)])
    for (g, d, vw, vol, sh), dy, gb in zip(items, dys, batched):
        gs = pmf.conebeam_project_backward(g, d, views(vw), dev(dy), shared=sh)
        assert torch.equal(gb, gs)
        ref = oracle.project_backward(g, d.nu, d.nv, d.step_mm, vw, dy, shared=sh)
        assert rel_l2(host(gb), ref) <= 1e-5


def test_batched_rejects_too_many_items():
    items = _items()[:1] * 17
    with pytest.raises(pmf.ops._lib.PmfError):
        pmf.ops.conebeam_project_batched([(g, d, views(vw), dev(vol), sh) for g, d, vw, vol, sh in items])
