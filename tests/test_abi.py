"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point include/pmf.h declares, its structs match the header, and
host-side validation rejects bad arguments before any device work."""
import ctypes as ct
import math
import os
import re

import pytest

from paper_2503_22139_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pmf.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["gs_voxelize", "gs_voxelize_backward", "mbc_combine", "mbc_combine_backward", "warp_volume",
                 "warp_volume_backward", "conebeam_project", "conebeam_project_backward", "projection_loss",
                 "warp_combine", "warp_combine_backward"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert b"sm_103a" in L.pmf_version()


def test_struct_layouts_match_header():
    assert ct.sizeof(_lib.PmfGrid) == 24
    assert ct.sizeof(_lib.PmfView) == 96
    assert ct.sizeof(_lib.PmfDetector) == 12
    assert ct.sizeof(_lib.PmfGaussians) == 48
    assert _lib.PmfGaussians.mean.offset == 16


def test_every_symbol_has_a_python_binding_of_the_same_name():
    import paper_2503_22139_gb300.ops as ops
    for n in _declared():
        if n.startswith("pmf_") or n.endswith("_workspace"):
            continue
        assert hasattr(ops, n), n


def _status(name, *args):
    L = _lib.load()
    return getattr(L, name)(*args)


def test_workspace_queries_are_host_only():
    g = _lib.PmfGrid(200, 200, 100, 2.0, 2.0, 2.0)
    n = ct.c_size_t(0)
    assert _status("gs_voxelize_workspace", ct.byref(g), 100000, 10**6, ct.byref(n)) == 0
    assert n.value >= 4 * 10**6
    assert _status("conebeam_project_backward_workspace", ct.byref(g), 32, 4_000_000, ct.byref(n)) == 0
    assert n.value >= 8 * 32 * 4_000_000
    assert _status("warp_combine_backward_workspace", ct.byref(g), 3, 32, ct.byref(n)) == 0
    assert _status("projection_loss_workspace", 1000, ct.byref(n)) == 0


@pytest.mark.parametrize("grid", [(0, 4, 4, 1, 1, 1), (4, 4, 4, 0, 1, 1), (4, -1, 4, 1, 1, 1)])
def test_bad_grids_are_rejected_before_launch(grid):
    g = _lib.PmfGrid(*grid)
    d = _lib.PmfDetector(8, 8, 1.0)
    rc = _status("conebeam_project", ct.byref(g), ct.byref(d), 1, ct.c_void_p(16), 0, ct.c_void_p(16), 0,
                 ct.c_void_p(16), None)
    assert rc == -1
    assert b"grid" in _lib.load().pmf_last_error() or b"voxel" in _lib.load().pmf_last_error()


def test_bad_arguments_are_rejected_before_launch():
    g = _lib.PmfGrid(8, 8, 8, 1.0, 1.0, 1.0)
    d = _lib.PmfDetector(8, 8, -1.0)
    assert _status("conebeam_project", ct.byref(g), ct.byref(d), 1, ct.c_void_p(16), 0, ct.c_void_p(16), 0,
                   ct.c_void_p(16), None) == -1
    d = _lib.PmfDetector(8, 8, 1.0)
    assert _status("conebeam_project", ct.byref(g), ct.byref(d), 1, ct.c_void_p(16), 7, ct.c_void_p(16), 0,
                   ct.c_void_p(16), None) == -1
    gs = _lib.PmfGaussians(10, 1, 0.0, 16, 16, 16, 16)  # kappa = 0
    assert _status("gs_voxelize", ct.byref(g), ct.byref(gs), 0, ct.c_void_p(16), ct.c_void_p(256), 1 << 20,
                   None) == -1
    gs = _lib.PmfGaussians(10, 9, 3.0, 16, 16, 16, 16)  # too many channels
    assert _status("gs_voxelize", ct.byref(g), ct.byref(gs), 0, ct.c_void_p(16), ct.c_void_p(256), 1 << 20,
                   None) == -5
    gs = _lib.PmfGaussians(10, 1, math.inf, 16, 16, 16, 16)
    # workspace far too small
    assert _status("gs_voxelize", ct.byref(g), ct.byref(gs), 0, ct.c_void_p(16), ct.c_void_p(256), 16, None) == -3
    # misaligned workspace
    assert _status("gs_voxelize", ct.byref(g), ct.byref(gs), 0, ct.c_void_p(16), ct.c_void_p(264), 1 << 20,
                   None) == -3
    assert _status("projection_loss", 3, 1, 4, ct.c_void_p(16), ct.c_void_p(16), ct.c_void_p(16), None,
                   ct.c_void_p(256), 1 << 16, None) == -1
    assert _status("mbc_combine", ct.byref(g), 9, 1, 0, ct.c_void_p(16), ct.c_void_p(16), ct.c_void_p(16),
                   None) == -1


def test_rasterizer_workspace_and_host_validation():
    d = _lib.PmfDetector(512, 384, 1.0)
    n0, n1 = ct.c_size_t(0), ct.c_size_t(0)
    assert _status("gs_rasterize_workspace", ct.byref(d), 32, 100000, 0, ct.byref(n0)) == 0
    assert _status("gs_rasterize_workspace", ct.byref(d), 32, 100000, 10**6, ct.byref(n1)) == 0
    # 32 bytes per projected Gaussian and 16 per pixel box, 4 per list entry
    assert n0.value >= 32 * 100000 * 48 and n1.value - n0.value >= 4 * 10**6 - 256
    fake = ct.c_void_p(256)
    gs = _lib.PmfGaussians(10, 3, 3.0, 16, 16, 16, 16)  # three channels: not a density set
    assert _status("gs_rasterize", ct.byref(d), 1, fake, ct.byref(gs), fake, fake, 1 << 30, None) == -1
    assert b"one channel" in _lib.load().pmf_last_error()
    gs = _lib.PmfGaussians(10, 1, 0.0, 16, 16, 16, 16)  # kappa = 0
    assert _status("gs_rasterize", ct.byref(d), 1, fake, ct.byref(gs), fake, fake, 1 << 30, None) == -1
    gs = _lib.PmfGaussians(10, 1, 3.0, 16, 16, 16, 16)
    assert _status("gs_rasterize", ct.byref(d), 1, None, ct.byref(gs), fake, fake, 1 << 30, None) == -1
    assert _status("gs_rasterize", ct.byref(d), 1, fake, ct.byref(gs), fake, fake, 16, None) == -3
    bad = _lib.PmfDetector(0, 384, 1.0)
    assert _status("gs_rasterize", ct.byref(bad), 1, fake, ct.byref(gs), fake, fake, 1 << 30, None) == -1
    assert _status("gs_rasterize_backward", ct.byref(d), 1, fake, ct.byref(gs), fake, None, fake, fake, fake, 0,
                   fake, 1 << 30, None) == -1


def test_density_control_host_validation():
    fake = ct.c_void_p(256)
    gs = _lib.PmfGaussians(10, 1, 3.0, 16, 16, 16, 16)
    n = ct.c_size_t(0)
    assert _status("gs_density_control_workspace", 1000, ct.byref(n)) == 0 and n.value >= 1000 * 9
    # output capacity below 2 n
    assert _status("gs_density_control", ct.byref(gs), fake, 1.0, fake, 0.1, 1.0, 0.01, 1.6, fake, fake, fake, fake,
                   19, fake, fake, 1 << 20, None) == -1
    assert b"out_capacity" in _lib.load().pmf_last_error()
    assert _status("gs_density_control", ct.byref(gs), fake, 1.0, fake, 0.1, 1.0, 0.01, 0.0, fake, fake, fake, fake,
                   20, fake, fake, 1 << 20, None) == -1
    assert _status("gs_density_control", ct.byref(gs), None, 1.0, fake, 0.1, 1.0, 0.01, 1.6, fake, fake, fake, fake,
                   20, fake, fake, 1 << 20, None) == -1


def test_tiled_voxelizer_and_threshold_host_validation():
    g = _lib.PmfGrid(40, 36, 30, 2.0, 2.0, 2.0)
    fake = ct.c_void_p(256)
    gs = _lib.PmfGaussians(10, 1, 3.0, 16, 16, 16, 16)
    n8, n4 = ct.c_size_t(0), ct.c_size_t(0)
    t8 = (ct.c_int32 * 3)(8, 8, 8)
    t4 = (ct.c_int32 * 3)(8, 8, 4)
    bad = (ct.c_int32 * 3)(8, 8, 2)
    assert _status("gs_voxelize_tiled_workspace", ct.byref(g), 1000, 0, t8, ct.byref(n8)) == 0
    assert _status("gs_voxelize_tiled_workspace", ct.byref(g), 1000, 0, t4, ct.byref(n4)) == 0
    # twice the tiles: the per-tile counters and offsets grow
    assert n4.value > n8.value
    ref = ct.c_size_t(0)
    assert _status("gs_voxelize_workspace", ct.byref(g), 1000, 0, ct.byref(ref)) == 0 and ref.value == n8.value
    assert _status("gs_voxelize_tiled_workspace", ct.byref(g), 1000, 0, bad, ct.byref(n8)) == -5
    assert b"not supported" in _lib.load().pmf_last_error()
    assert _status("gs_voxelize_tiled", ct.byref(g), ct.byref(gs), 0, bad, fake, fake, 1 << 20, None) == -5
    assert _status("gs_voxelize_tiled", ct.byref(g), ct.byref(gs), 0, None, fake, fake, 1 << 20, None) == -1
    # the densification threshold: rank in [0, n), n >= 1, finite scale
    for n, rank, scale in ((10, 10, 1.0), (10, -1, 1.0), (0, 0, 1.0), (10, 3, math.inf)):
        assert _status("gs_density_threshold", n, fake, scale, rank, fake, None) == -1, (n, rank, scale)
    assert _status("gs_density_threshold", 10, None, 1.0, 3, fake, None) == -1


def test_fused_bound_entry_points_need_their_bound_pointer():
    """conebeam_project_backward_absmax and warp_combine_backward_bounded
    reject a null bound pointer on the host, before any device work."""
    g = _lib.PmfGrid(8, 8, 8, 1.0, 1.0, 1.0)
    d = _lib.PmfDetector(8, 8, 1.0)
    fake = ct.c_void_p(256)
    assert _status("conebeam_project_backward_absmax", ct.byref(g), ct.byref(d), 1, fake, fake, fake, 512, 0, fake,
                   1 << 20, None, None) == -1
    assert b"absmax" in _lib.load().pmf_last_error()
    assert _status("warp_combine_backward_bounded", ct.byref(g), 3, 2, 0, fake, fake, fake, fake, None, fake, fake,
                   fake, 0, fake, 1 << 20, None) == -1
    assert b"absmax" in _lib.load().pmf_last_error()
