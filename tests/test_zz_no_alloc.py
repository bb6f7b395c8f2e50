"""The no-allocation variant of the combine adjoint, called through the C ABI
with caller-owned outputs only, must reproduce the allocating entry point.

Some callers cannot allocate device memory on the call path (all device memory
belongs to their own pool, or they must avoid the synchronization that
allocating can cause); mbc_combine_backward_noalloc serves them from a fixed
array compiled into the library.  This file is collected last on purpose."""
import ctypes as ct

import numpy as np
import pytest
import torch

import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300 import _lib
from synth import Grid

pytestmark = pytest.mark.gpu


def _inputs(P, L, seed):
    grid = Grid(23, 19, 17, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(seed)
    E = torch.as_tensor(rng.normal(0, 2.0, (L, 3) + grid.shape), dtype=torch.float32, device="cuda")
    w = torch.as_tensor(rng.uniform(-1, 1, (P, L, 3)), dtype=torch.float32, device="cuda")
    dD = torch.as_tensor(rng.normal(size=(P, 3) + grid.shape), dtype=torch.float32, device="cuda")
    return grid, E, w, dD


def _call_c(grid, E, w, dD, dE, dw):
    L = _lib.load()
    g = _lib.PmfGrid(grid.nx, grid.ny, grid.nz, grid.vx, grid.vy, grid.vz)
    return L.mbc_combine_backward_noalloc(ct.byref(g), int(w.shape[1]), int(w.shape[0]), 0,
                                          ct.c_void_p(E.data_ptr()), ct.c_void_p(w.data_ptr()),
                                          ct.c_void_p(dD.data_ptr()), ct.c_void_p(dE.data_ptr()),
                                          ct.c_void_p(dw.data_ptr()), 0,
                                          ct.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_allocating_entry_point_twice(gpu_lib):
    grid, E, w, dD = _inputs(P=32, L=3, seed=101)
    ref_dE, ref_dw = pmf.mbc_combine_backward(grid, E, w, dD)
    for _ in range(2):  # the second call reuses the shared scratch left by the first
        dE = torch.full_like(ref_dE, float("nan"))
        dw = torch.full_like(ref_dw, float("nan"))
        assert _call_c(grid, E, w, dD, dE, dw) == 0, _lib.load().pmf_last_error()
        torch.cuda.synchronize()
        torch.testing.assert_close(dE, ref_dE, rtol=1e-6, atol=1e-6)
        torch.testing.assert_close(dw, ref_dw, rtol=1e-6, atol=1e-6)


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu_lib):
    grid, E, w, dD = _inputs(P=43, L=3, seed=102)  # P*L = 129 > 128
    dE = torch.empty_like(E)
    dw = torch.empty_like(w)
    assert _call_c(grid, E, w, dD, dE, dw) == -3
    assert b"no-allocation" in _lib.load().pmf_last_error()
