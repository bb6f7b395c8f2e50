"""ctypes loader for the in-tree sm_103a library (libpmf.so) and its C structs.

There is no fallback: if the library cannot be built or loaded, every entry
point raises.  The structs mirror include/pmf.h field for field.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None


class PmfGrid(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32),
                ("vx", ct.c_float), ("vy", ct.c_float), ("vz", ct.c_float)]


class PmfView(ct.Structure):
    _fields_ = [("src", ct.c_double * 3), ("det", ct.c_double * 3), ("du", ct.c_double * 3), ("dv", ct.c_double * 3)]


class PmfDetector(ct.Structure):
    _fields_ = [("nu", ct.c_int32), ("nv", ct.c_int32), ("step_mm", ct.c_float)]


class PmfGaussians(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("channels", ct.c_int32), ("kappa", ct.c_float),
                ("mean", ct.c_void_p), ("scale", ct.c_void_p), ("quat", ct.c_void_p), ("value", ct.c_void_p)]


class PmfProjectItem(ct.Structure):
    _fields_ = [("grid", PmfGrid), ("det", PmfDetector), ("P", ct.c_int32), ("views", ct.c_void_p),
                ("vol", ct.c_void_p), ("vol_stride", ct.c_int64), ("proj", ct.c_void_p)]


class PmfBackprojectItem(ct.Structure):
    _fields_ = [("grid", PmfGrid), ("det", PmfDetector), ("P", ct.c_int32), ("views", ct.c_void_p),
                ("d_proj", ct.c_void_p), ("d_vol", ct.c_void_p), ("vol_stride", ct.c_int64)]


PMF_MAX_LEVELS = 8
PMF_DIAG_COUNT = 8
DIAG_NAMES = ("voxelize_list_overflow", "project_box_fallback", "backproject_box_fallback", "warp_halo_exit",
              "nonfinite", "timeout", "raster_list_overflow", "bounds")
PMF_OPS = {"voxelize": 1, "voxelize_backward": 2, "combine_backward": 3, "warp_backward": 4,
           "warp_combine_backward": 5, "project_backward": 6, "loss": 7}


class PmfWsArgs(ct.Structure):
    _fields_ = [("grid", PmfGrid), ("n", ct.c_int64), ("pair_capacity", ct.c_int64), ("vol_stride", ct.c_int64),
                ("count", ct.c_int64), ("channels", ct.c_int32), ("L", ct.c_int32), ("P", ct.c_int32)]


class PmfBatchDesc(ct.Structure):
    _fields_ = [("grid", PmfGrid), ("det", PmfDetector), ("dtype", ct.c_int), ("batch", ct.c_int32),
                ("loss_kind", ct.c_int32), ("levels", ct.c_int32), ("ref", PmfGaussians),
                ("mbc", PmfGaussians * PMF_MAX_LEVELS), ("views", ct.c_void_p), ("coeff", ct.c_void_p),
                ("meas", ct.c_void_p), ("loss", ct.c_void_p), ("d_ref", ct.c_void_p * 4),
                ("d_mbc", (ct.c_void_p * 4) * PMF_MAX_LEVELS), ("d_coeff", ct.c_void_p), ("use_graph", ct.c_int32),
                ("tune_cache", ct.c_char_p), ("lambda_ssim", ct.c_float), ("lambda_mbc", ct.c_float),
                ("lambda_tv", ct.c_float), ("ssim_range", ct.c_float), ("tv_size", ct.c_int32),
                ("tv_origin", ct.c_void_p), ("w_dtype", ct.c_int)]


class PmfPlanTensors(ct.Structure):
    _fields_ = [(n, ct.c_void_p) for n in ("V", "E", "W", "Y", "dY", "dW", "dV", "dE")]


PMF_OK = 0
STATUS = {0: "PMF_OK", -1: "PMF_EINVAL", -2: "PMF_ECUDA", -3: "PMF_EWORKSPACE", -4: "PMF_ETIMEOUT",
          -5: "PMF_EUNSUPPORTED"}
DTYPE_CODES = {"f32": 0, "bf16": 1, "f16": 2}

_P = ct.c_void_p
_G = ct.POINTER(PmfGrid)
_SZ = ct.POINTER(ct.c_size_t)
_I32 = ct.c_int32
_I64 = ct.c_int64

# name -> argtypes (every entry point returns pmf_status as int)
SIGNATURES = {
    "gs_voxelize_workspace": [_G, _I64, _I64, _SZ],
    "gs_voxelize_count": [_G, ct.POINTER(PmfGaussians), _P, _P, ct.c_size_t, _P],
    "gs_voxelize": [_G, ct.POINTER(PmfGaussians), ct.c_int, _P, _P, ct.c_size_t, _P],
    "gs_voxelize_tiled_workspace": [_G, _I64, _I64, ct.POINTER(ct.c_int32), _SZ],
    "gs_voxelize_tiled_count": [_G, ct.POINTER(PmfGaussians), ct.POINTER(ct.c_int32), _P, _P, ct.c_size_t, _P],
    "gs_voxelize_tiled": [_G, ct.POINTER(PmfGaussians), ct.c_int, ct.POINTER(ct.c_int32), _P, _P, ct.c_size_t, _P],
    "gs_voxelize_backward_workspace": [_G, _I64, _I32, _SZ],
    "pmf_shift_means": [_I64, _P, _P, _P, _P],
    "gs_grad_norm_accumulate": [_I64, _P, _P, _P],
    "gs_density_control_workspace": [_I64, _SZ],
    "gs_density_control": [ct.POINTER(PmfGaussians), _P, ct.c_float, _P, ct.c_float, ct.c_float, ct.c_float,
                           ct.c_float, _P, _P, _P, _P, _I64, _P, _P, ct.c_size_t, _P],
    "gs_rasterize_workspace": [ct.POINTER(PmfDetector), _I32, _I64, _I64, _SZ],
    "gs_rasterize_count": [ct.POINTER(PmfDetector), _I32, _P, ct.POINTER(PmfGaussians), _P, _P, ct.c_size_t, _P],
    "gs_rasterize": [ct.POINTER(PmfDetector), _I32, _P, ct.POINTER(PmfGaussians), _P, _P, ct.c_size_t, _P],
    "gs_rasterize_backward": [ct.POINTER(PmfDetector), _I32, _P, ct.POINTER(PmfGaussians), _P, _P, _P, _P, _P,
                              ct.c_int, _P, ct.c_size_t, _P],
    "gs_voxelize_backward": [_G, ct.POINTER(PmfGaussians), _P, _P, _P, _P, _P, ct.c_int, _P, ct.c_size_t, _P],
    "mbc_combine": [_G, _I32, _I32, ct.c_int, _P, _P, _P, _P],
    "mbc_combine_backward_workspace": [_G, _I32, _I32, _SZ],
    "mbc_combine_backward": [_G, _I32, _I32, ct.c_int, _P, _P, _P, _P, _P, ct.c_int, _P, ct.c_size_t, _P],
    "mbc_combine_backward_noalloc": [_G, _I32, _I32, ct.c_int, _P, _P, _P, _P, _P, ct.c_int, _P],
    "warp_volume": [_G, _I32, ct.c_int, _P, _P, _P, _P],
    "warp_volume_backward_workspace": [_G, _I32, _SZ],
    "warp_volume_backward": [_G, _I32, ct.c_int, _P, _P, _P, _P, _P, ct.c_int, _P, ct.c_size_t, _P],
    "warp_combine": [_G, _I32, _I32, ct.c_int, _P, _P, _P, _P, _P],
    "warp_combine_mixed": [_G, _I32, _I32, ct.c_int, _P, _P, _P, ct.c_int, _P, _P],
    "warp_combine_backward_workspace": [_G, _I32, _I32, _SZ],
    "warp_combine_backward": [_G, _I32, _I32, ct.c_int, _P, _P, _P, _P, _P, _P, _P, ct.c_int, _P, ct.c_size_t, _P],
    "warp_combine_backward_bounded": [_G, _I32, _I32, ct.c_int, _P, _P, _P, _P, _P, _P, _P, _P, ct.c_int, _P, ct.c_size_t,
                                      _P],
    "conebeam_project": [_G, ct.POINTER(PmfDetector), _I32, _P, ct.c_int, _P, _I64, _P, _P],
    "conebeam_project_backward_workspace": [_G, _I32, _I64, _SZ],
    "conebeam_project_backward": [_G, ct.POINTER(PmfDetector), _I32, _P, _P, _P, _I64, ct.c_int, _P, ct.c_size_t, _P],
    "conebeam_project_backward_absmax": [_G, ct.POINTER(PmfDetector), _I32, _P, _P, _P, _I64, ct.c_int, _P, ct.c_size_t,
                                         _P, _P],
    "conebeam_project_batched": [_I32, ct.POINTER(PmfProjectItem), ct.c_int, _P],
    "conebeam_project_backward_batched_workspace": [_I32, ct.POINTER(PmfBackprojectItem), _SZ],
    "conebeam_project_backward_batched": [_I32, ct.POINTER(PmfBackprojectItem), ct.c_int, _P, ct.c_size_t, _P],
    "projection_loss_workspace": [_I64, _SZ],
    "projection_loss": [_I32, _I32, _I64, _P, _P, _P, _P, _P, ct.c_size_t, _P],
    "projection_dssim_workspace": [_I32, _I32, _I32, _SZ],
    "projection_dssim": [_I32, _I32, _I32, _P, _P, ct.c_float, ct.c_float, _P, _P, ct.c_int, _P, ct.c_size_t, _P],
    "tv_loss_workspace": [_I32, _SZ],
    "tv_loss": [_G, ct.c_int, _P, _I32, _P, ct.c_float, _P, _P, ct.c_int, _P, ct.c_size_t, _P],
    "mbc_normality_workspace": [_I32, _SZ],
    "mbc_normality": [_G, _I32, ct.c_int, _P, ct.c_float, _P, _P, ct.c_int, _P, ct.c_size_t, _P],
    "pmf_adam_step": [_I64, _P, _P, _P, _P, ct.c_float, ct.c_float, ct.c_float, ct.c_float, _I32, _P],
    "pmf_circular_views": [_I32, ct.c_double, ct.c_double, ct.c_double, ct.c_double, _I32, _I32, ct.POINTER(PmfView)],
    "pmf_workspace_size": [_I32, ct.POINTER(PmfWsArgs), _SZ],
    "pmf_device_counters": [ct.POINTER(ct.c_uint64), _I32],
    "pmf_device_status": [_P],
    "gs_density_threshold": [_I64, _P, ct.c_float, _I64, _P, _P],
    "pmf_debug_stall_bulk_copies": [_I32],
    "pmf_plan_create": [ct.POINTER(PmfBatchDesc), ct.POINTER(ct.c_void_p)],
    "pmf_plan_step": [_P, _P],
    "pmf_plan_tensors_get": [_P, ct.POINTER(PmfPlanTensors)],
    "pmf_plan_launch_forms": [_P, ct.POINTER(_I32), ct.POINTER(_I32)],
    "pmf_plan_voxel_tiles": [_P, ct.POINTER(_I32)],
    "pmf_plan_destroy": [_P],
    "pmf_autotune": [ct.POINTER(PmfBatchDesc), ct.c_char_p],
}


class PmfError(RuntimeError):
    pass


def variant() -> str:
    """Which build this process loads: "debug" (the bounds-checked
    libpmf_debug.so) when PMF_LIB_VARIANT=debug, else the normal libpmf.so."""
    return "debug" if os.environ.get("PMF_LIB_VARIANT", "") == "debug" else "release"


def load():
    """Build (if stale) and load libpmf.so (or, see variant(), the debug
    build); raises if either fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(debug=variant() == "debug")
            if not os.path.exists(path):
                raise PmfError(f"libpmf.so missing at {path}")
            L = ct.CDLL(path)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ct.c_int
            L.pmf_version.restype = ct.c_char_p
            L.pmf_last_error.restype = ct.c_char_p
            L.pmf_status_string.restype = ct.c_char_p
            L.pmf_status_string.argtypes = [ct.c_int]
            _lib = L
    return _lib


def check(status: int, what: str) -> None:
    if status != PMF_OK:
        msg = load().pmf_last_error().decode(errors="replace")
        raise PmfError(f"{what}: {STATUS.get(status, status)}: {msg}")


def library_path() -> str:
    return _build.LIB
