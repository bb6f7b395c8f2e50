"""CPU-side checks of the plan, workspace, geometry and diagnostics entry points:
the ctypes structs match the header as gcc lays it out, the circular-scan helper
reproduces the Table I / Sec. 2.3.3 trajectory, the workspace dispatcher agrees
with every per-op query, and invalid plan descriptors are rejected on the host
before any CUDA call."""
import ctypes as ct
import os
import subprocess

import numpy as np
import pytest

import paper_2503_22139_gb300.ops as ops
from paper_2503_22139_gb300 import _lib
from synth import circular_views

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_PROBE = r"""
#include <stdio.h>
#include <stddef.h>
#include "pmf.h"
#define S(T) printf(#T " %zu\n", sizeof(T))
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
    S(pmf_view); S(pmf_grid); S(pmf_detector); S(pmf_gaussians); S(pmf_project_item); S(pmf_backproject_item);
    S(pmf_ws_args); S(pmf_batch_desc); S(pmf_plan_tensors);
    O(pmf_ws_args, n); O(pmf_ws_args, count); O(pmf_ws_args, channels); O(pmf_ws_args, P);
    O(pmf_batch_desc, det); O(pmf_batch_desc, dtype); O(pmf_batch_desc, levels); O(pmf_batch_desc, ref);
    O(pmf_batch_desc, mbc); O(pmf_batch_desc, views); O(pmf_batch_desc, loss); O(pmf_batch_desc, d_ref);
    O(pmf_batch_desc, d_mbc); O(pmf_batch_desc, d_coeff); O(pmf_batch_desc, use_graph);
    O(pmf_batch_desc, tune_cache); O(pmf_batch_desc, lambda_ssim); O(pmf_batch_desc, ssim_range);
    O(pmf_batch_desc, tv_size); O(pmf_batch_desc, tv_origin); O(pmf_batch_desc, w_dtype);
    O(pmf_plan_tensors, dE);
    O(pmf_project_item, views); O(pmf_project_item, vol_stride); O(pmf_backproject_item, vol_stride);
    return 0;
}
"""


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text(_PROBE)
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def test_ctypes_structs_match_gcc_layout(c_layout):
    pairs = {"pmf_view": _lib.PmfView, "pmf_grid": _lib.PmfGrid, "pmf_detector": _lib.PmfDetector,
             "pmf_gaussians": _lib.PmfGaussians, "pmf_project_item": _lib.PmfProjectItem,
             "pmf_backproject_item": _lib.PmfBackprojectItem, "pmf_ws_args": _lib.PmfWsArgs,
             "pmf_batch_desc": _lib.PmfBatchDesc, "pmf_plan_tensors": _lib.PmfPlanTensors}
    for cname, cls in pairs.items():
        assert ct.sizeof(cls) == c_layout[cname], cname
    for key, off in c_layout.items():
        if "." not in key:
            continue
        cname, field = key.split(".")
        assert getattr(pairs[cname], field).offset == off, key


def test_circular_views_match_the_scan_protocol():
    """SAD/SDD 1000/1500 mm, 512 x 384 at 0.776 mm, 660 views over 360 degrees."""
    got = ops.pmf_circular_views(660, 1000.0, 1500.0, 0.776, 0.776, 512, 384).numpy()
    ref = circular_views(660, 1000.0, 1500.0, 512, 384, 0.776, 0.776)
    assert got.shape == (660, 12)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)
    # geometry invariants: |src| = SAD, |det| = SDD - SAD, du and dv orthogonal to the central ray
    assert np.allclose(np.linalg.norm(got[:, 0:3], axis=1), 1000.0)
    assert np.allclose(np.linalg.norm(got[:, 3:6], axis=1), 500.0)
    assert np.allclose(np.einsum("pi,pi->p", got[:, 6:9], got[:, 0:3]), 0.0, atol=1e-9)
    assert np.allclose(got[:, 9:12], [0.0, 0.0, 0.776])


def test_circular_views_reject_bad_geometry():
    L = _lib.load()
    arr = (_lib.PmfView * 2)()
    assert L.pmf_circular_views(2, 1500.0, 1000.0, 1.0, 1.0, 8, 8, arr) == -1  # SDD < SAD
    assert L.pmf_circular_views(2, 1000.0, 1500.0, 0.0, 1.0, 8, 8, arr) == -1
    assert L.pmf_circular_views(2, 1000.0, 1500.0, 1.0, 1.0, 0, 8, arr) == -1


def test_workspace_dispatcher_agrees_with_each_query():
    g = (200, 200, 100, 2.0, 2.0, 2.0)
    L = _lib.load()
    G = ops._grid(g)

    def direct(fn, *args):
        return ops._size(fn, *args)

    assert ops.pmf_workspace_size("voxelize", g, n=100000, pair_capacity=10**6) == \
        direct(L.gs_voxelize_workspace, ct.byref(G), 100000, 10**6)
    assert ops.pmf_workspace_size("voxelize_backward", g, n=8000, channels=3) == \
        direct(L.gs_voxelize_backward_workspace, ct.byref(G), 8000, 3)
    assert ops.pmf_workspace_size("combine_backward", g, L=3, P=32) == \
        direct(L.mbc_combine_backward_workspace, ct.byref(G), 3, 32)
    assert ops.pmf_workspace_size("warp_backward", g, P=32) == direct(L.warp_volume_backward_workspace, ct.byref(G), 32)
    assert ops.pmf_workspace_size("warp_combine_backward", g, L=3, P=32) == \
        direct(L.warp_combine_backward_workspace, ct.byref(G), 3, 32)
    assert ops.pmf_workspace_size("project_backward", g, P=32, vol_stride=4_000_000) == \
        direct(L.conebeam_project_backward_workspace, ct.byref(G), 32, 4_000_000)
    assert ops.pmf_workspace_size("loss", g, count=32 * 512 * 384) == \
        direct(L.projection_loss_workspace, 32 * 512 * 384)
    a = _lib.PmfWsArgs(G, 0, 0, 0, 0, 0, 0, 0)
    n = ct.c_size_t(0)
    assert L.pmf_workspace_size(99, ct.byref(a), ct.byref(n)) == -1
    assert b"unknown workspace op" in L.pmf_last_error()


def _desc(**over):
    d = _lib.PmfBatchDesc()
    d.grid = _lib.PmfGrid(16, 16, 16, 4.0, 4.0, 4.0)
    d.det = _lib.PmfDetector(32, 32, 2.0)
    d.dtype, d.batch, d.loss_kind, d.levels = 0, 4, 2, 1
    fake = 1 << 20  # never dereferenced: validation rejects the descriptor first
    d.ref = _lib.PmfGaussians(10, 1, 3.0, fake, fake, fake, fake)
    d.mbc[0] = _lib.PmfGaussians(4, 3, 3.0, fake, fake, fake, fake)
    for k in range(4):
        d.d_ref[k] = fake
        d.d_mbc[0][k] = fake
    d.views = d.coeff = d.meas = d.loss = d.d_coeff = fake
    for k, v in over.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value,msg", [
    ("batch", 0, b"batch"), ("loss_kind", 0, b"loss_kind"), ("levels", 0, b"levels"), ("levels", 9, b"levels"),
    ("dtype", 7, b"dtype"), ("views", None, b"null batch pointer"), ("loss_kind", 4, b"loss_kind"),
    ("w_dtype", 1, b"w_dtype"), ("w_dtype", 5, b"w_dtype"),
])
def test_plan_rejects_bad_descriptors_on_the_host(field, value, msg):
    L = _lib.load()
    h = ct.c_void_p(123)
    d = _desc(**{field: value})
    assert L.pmf_plan_create(ct.byref(d), ct.byref(h)) == -1
    assert h.value is None
    assert msg in L.pmf_last_error()


def test_plan_rejects_wrong_channel_counts():
    L = _lib.load()
    d = _desc()
    d.mbc[0] = _lib.PmfGaussians(4, 1, 3.0, 1 << 20, 1 << 20, 1 << 20, 1 << 20)
    h = ct.c_void_p(0)
    assert L.pmf_plan_create(ct.byref(d), ct.byref(h)) == -1
    assert b"channels" in L.pmf_last_error()


def test_autotune_needs_a_cache_path():
    L = _lib.load()
    d = _desc()
    assert L.pmf_autotune(ct.byref(d), b"") == -1
    assert L.pmf_autotune(ct.byref(d), None) == -1


def test_destroying_a_null_plan_is_a_no_op():
    assert _lib.load().pmf_plan_destroy(None) == 0


def test_plan_rejects_incomplete_eq14_descriptors():
    L = _lib.load()
    for field, value, msg in [("ssim_range", 0.0, b"ssim_range"), ("tv_size", 1, b"tv_size"),
                              ("tv_size", 17, b"tv_size"), ("tv_origin", None, b"tv_origin")]:
        d = _desc(loss_kind=3, lambda_ssim=0.25, lambda_mbc=1.0, lambda_tv=0.05, ssim_range=100.0, tv_size=8,
                  tv_origin=1 << 20)
        setattr(d, field, value)
        h = ct.c_void_p(0)
        assert L.pmf_plan_create(ct.byref(d), ct.byref(h)) == -1
        assert msg in L.pmf_last_error()
