"""The native training-step plan (pmf_plan_*), its CUDA-graph mode, the launch-form
autotuner and the device diagnostics, on the small workload (64^3 @ 4 mm, 2,000
reference Gaussians, one MBC level, 8 views of 128^2).  The plan composes the
same entry points as pipeline.ForwardAdjoint, so its outputs must equal that
step's bit for bit, whatever the launch forms; the step itself is checked
against the oracle by the parity tests."""
import numpy as np
import pytest
import torch

import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300.pipeline import ForwardAdjoint
from synth import small_workload
from tests.gpu_util import dev, gset, views

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wl():
    return small_workload()


def _sets(wl):
    return gset(wl.ref, wl.kappa), [gset(m, wl.kappa) for m in wl.mbc]


def _batch(wl, shift=0):
    idx = (np.arange(wl.p) + shift) % wl.p
    return views(wl.views[idx]), dev(wl.coeff[idx]), dev(wl.measured[idx])


def _plan_outputs(plan):
    t = plan.tensors()
    out = {k: t[k].clone() for k in ("V", "E", "W", "Y", "dW", "dV", "dE")}
    out["loss"] = plan.loss.clone()
    out["d_coeff"] = plan.d_coeff.clone()
    for k, g in enumerate(plan.g_ref):
        out[f"ref{k}"] = g.clone()
    for l, gl in enumerate(plan.g_mbc):
        for k, g in enumerate(gl):
            out[f"mbc{l}_{k}"] = g.clone()
    return out


def _assert_same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("dt,wdt", [(torch.float32, torch.float32), (torch.bfloat16, torch.float32),
                                     (torch.bfloat16, torch.bfloat16)])
def test_plan_step_equals_forward_adjoint(wl, dt, wdt):
    ref, mbc = _sets(wl)
    args = _batch(wl)
    step = ForwardAdjoint(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=dt, w_dtype=wdt)
    loss = step.run(*args).clone()
    plan = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=dt, w_dtype=wdt)
    got = plan.step(*args)
    torch.cuda.synchronize()
    assert torch.equal(got, loss)
    t = plan.tensors()
    assert t["W"].dtype == wdt
    assert torch.equal(t["V"], step.V[0]) and torch.equal(t["E"], step.E) and torch.equal(t["W"], step.W)
    assert torch.equal(t["Y"], step.Y) and torch.equal(t["dW"], step.dW)
    for a, b in zip(plan.g_ref, step.g_ref):
        assert torch.equal(a, b)
    for ga, gb in zip(plan.g_mbc, step.g_mbc):
        for a, b in zip(ga, gb):
            assert torch.equal(a, b)
    assert torch.equal(plan.d_coeff, step.g_wc[2])
    assert torch.equal(t["dV"], step.g_wc[0]) and torch.equal(t["dE"], step.g_wc[1])
    plan.close()


def test_graph_plan_replays_the_eager_step(wl):
    """Two different batches through a graph-captured plan equal the eager plan's
    results for the same batches."""
    ref, mbc = _sets(wl)
    eager = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.bfloat16)
    graph = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.bfloat16, use_graph=True)
    for shift in (0, 3):
        b = _batch(wl, shift)
        eager.step(*b)
        graph.step(*b)
        torch.cuda.synchronize()
        _assert_same(_plan_outputs(eager), _plan_outputs(graph))
    eager.close()
    graph.close()


def _shape(txt):
    return tuple(int(x) for x in txt.split("=")[1].split(","))


def test_autotune_cache_selects_launch_shapes(wl, tmp_path):
    """The autotuner records one shape per direction; a plan reads it back.
    Launch forms (grid or persistent) give bit-identical results; brick length
    and rays per CTA move only the last bits (chunk anchors, per-CTA fixed-point
    scales), so every forced shape stays within 1e-6 of the default plan's
    volumes and projections and within 1e-4 of its gradients (a tenth of the
    gradient bar: the quaternion gradient sums terms of both signs); the
    default itself is pinned to the oracle by the parity tests."""
    ref, mbc = _sets(wl)
    b = _batch(wl)
    cache = tmp_path / "tune.txt"
    pmf.autotune(wl.grid, wl.det, ref, mbc, wl.p, str(cache), dtype=torch.float32, views=b[0], coeff=b[1],
                 meas=b[2])
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and " proj=" in lines[0] and " backproj=" in lines[0] and " vox=" in lines[0]
    key, fp_txt, bp_txt, vox_txt = lines[0].split(" ")
    tuned = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.float32, tune_cache=str(cache))
    assert tuned.launch_forms() == (_shape(fp_txt), _shape(bp_txt))
    tiles = [tuple(int(v) for v in t.split("x")) for t in vox_txt[len("vox="):].split(",")]
    assert tuned.voxel_tiles() == tiles and len(tiles) == 1 + len(mbc)
    assert all(t in pmf.ops.VOXEL_TILES for t in tiles)
    default = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.float32)
    assert default.launch_forms() == ((0, 48, 256), (0, 48, 128))
    assert default.voxel_tiles() == [(8, 8, 8)] * (1 + len(mbc))
    # the tiled voxelizer gives the same bits, so the tuned plan's voxel tiles
    # alone change nothing: force the tuned tiles with the default launch shapes
    cache_t = tmp_path / "tiles.txt"
    cache_t.write_text(f"{key} proj=0,48,256 backproj=0,48,128 {vox_txt}\n")
    tiled = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.float32, tune_cache=str(cache_t))
    assert tiled.voxel_tiles() == tiles
    default.step(*b)
    torch.cuda.synchronize()
    base = _plan_outputs(default)
    tiled.step(*b)
    torch.cuda.synchronize()
    _assert_same(base, _plan_outputs(tiled))
    tiled.close()
    for fp, bp in [((2, 48, 256), (3, 48, 128)), ((0, 16, 256), (0, 64, 128)), ((4, 32, 128), (1, 16, 256))]:
        cache.write_text(f"other-key proj=1,32,256 backproj=1,32,256\n{key} proj={','.join(map(str, fp))} "
                         f"backproj={','.join(map(str, bp))}\n")
        forced = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.float32, tune_cache=str(cache))
        assert forced.launch_forms() == (fp, bp)
        forced.step(*b)
        torch.cuda.synchronize()
        got = _plan_outputs(forced)
        if fp[1:] == (48, 256) and bp[1:] == (48, 128):
            _assert_same(base, got)  # forms alone: bit-identical
        else:
            for k in base:
                d = (got[k].double() - base[k].double()).norm() / max(base[k].double().norm(), 1e-30)
                assert d <= (1e-6 if k in ("V", "E", "W", "Y", "loss") else 1e-4), (k, fp, bp, float(d))
        forced.close()
    # a second autotune of the same key replaces its line and keeps the others
    pmf.autotune(wl.grid, wl.det, ref, mbc, wl.p, str(cache), dtype=torch.float32, views=b[0], coeff=b[1],
                 meas=b[2])
    lines = cache.read_text().splitlines()
    assert len(lines) == 2 and lines[0].startswith("other-key ") and lines[1].startswith(key + " ")
    for p in (default, tuned):
        p.close()


def test_device_counters_and_status(wl):
    pmf.device_counters(reset=True)
    assert all(v == 0 for v in pmf.device_counters().values())
    ref, _ = _sets(wl)
    # a pair list far too small: every tile scans all Gaussians (same result, counted)
    full = pmf.gs_voxelize(wl.grid, ref)
    small = pmf.gs_voxelize(wl.grid, ref, pair_capacity=1)
    assert torch.equal(full, small)
    c = pmf.device_counters()
    assert c["voxelize_list_overflow"] > 0 and c["nonfinite"] == 0
    pmf.device_status()  # no error: overflow is a slow path, not a failure
    # a NaN in the projection adjoint's input: the output is NaN and the status reports it
    dY = torch.zeros((1, wl.det.nv, wl.det.nu), device="cuda")
    dY[0, 5, 7] = float("nan")
    out = pmf.conebeam_project_backward(wl.grid, wl.det, views(wl.views[:1]), dY, shared=False)
    assert torch.isnan(out).all()
    assert pmf.device_counters()["nonfinite"] >= 1
    with pytest.raises(pmf.PmfError, match="NaN or infinite"):
        pmf.device_status()
    pmf.device_counters(reset=True)
    pmf.device_status()


def test_box_fallback_counters(wl):
    """Pixels far larger than voxels overflow the shared box (the geometry of the
    fallback parity test): both projector directions count their fallbacks."""
    from synth import Detector, Grid, circular_views
    grid = Grid(40, 40, 40, 0.5, 0.5, 0.5)
    vw = circular_views(2, 60.0, 90.0, 18, 17, 12.0, 12.0, start=0.3)
    det = Detector(18, 17, 0.25)
    vol = torch.rand(grid.shape, device="cuda")
    pmf.device_counters(reset=True)
    Y = pmf.conebeam_project(grid, det, views(vw), vol, shared=True)
    pmf.conebeam_project_backward(grid, det, views(vw), torch.ones_like(Y), shared=True)
    c = pmf.device_counters(reset=True)
    assert c["project_box_fallback"] > 0 and c["backproject_box_fallback"] > 0
    assert c["nonfinite"] == 0


def test_eq14_plan_equals_forward_adjoint_and_replays_new_crops(wl):
    """The Eq. 14 objective through the native plan (eager and graph-captured)
    equals the Python step bit for bit, with the TV crop moving every step."""
    ref, mbc = _sets(wl)
    q = dict(data_range=float(wl.measured.max() - wl.measured.min()), tv_size=32)
    step = ForwardAdjoint(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.bfloat16, kind="eq14", eq14=q)
    eager = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.bfloat16, kind="eq14", eq14=q)
    graph = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=wl.p, dtype=torch.bfloat16, kind="eq14", eq14=q,
                     use_graph=True)
    for shift, origin in ((0, (3, 9, 27)), (2, (30, 1, 12))):
        b = _batch(wl, shift)
        o = torch.tensor(origin, dtype=torch.int32, device="cuda")
        loss = step.run(*b, tv_origin=o).clone()
        eager.step(*b, tv_origin=o)
        graph.step(*b, tv_origin=o)
        torch.cuda.synchronize()
        assert torch.equal(eager.loss, loss) and torch.equal(graph.loss, loss)
        for a, c in zip(eager.g_ref, step.g_ref):
            assert torch.equal(a, c)
        for ga, gc in zip(eager.g_mbc, step.g_mbc):
            for a, c in zip(ga, gc):
                assert torch.equal(a, c)
        assert torch.equal(eager.d_coeff, step.g_wc[2])
        _assert_same(_plan_outputs(eager), _plan_outputs(graph))
    for p in (eager, graph):
        p.close()
