"""The back-projector's fused abs-max and the bounded warp adjoint.

conebeam_project_backward_absmax writes max |d_vol| (the float bits with the
sign cleared) from the kernel that converts its accumulator;
warp_combine_backward_bounded takes that value as the bound of its fixed-point
dV instead of a pass of its own over dW.  With the exact maximum both give the
unfused calls' bits."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from synth import Detector, Grid, circular_views
from tests.gpu_util import dev, host, rel_l2, views

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib_loaded(gpu_lib):
    return gpu_lib


def _bits(t: torch.Tensor) -> int:
    """abs bits of max |t| (finite t)."""
    return int(t.abs().max().reshape(1).view(torch.int32).item())


def _bp_problem(seed=22, P=3):
    grid = Grid(20, 18, 14, 2.0, 2.0, 2.5)
    rng = np.random.default_rng(seed)
    vw = circular_views(P, 400.0, 600.0, 29, 21, 1.8, 1.9, start=0.1)
    dY = rng.normal(size=(P, 21, 29)).astype(np.float32)
    return grid, Detector(29, 21, 1.0), vw, dY


@pytest.mark.parametrize("shared,accumulate", [(False, False), (True, False), (False, True)])
def test_backproject_absmax_is_the_max_of_what_it_writes(shared, accumulate):
    grid, det, vw, dY = _bp_problem()
    shape = grid.shape if shared else (3,) + grid.shape
    base = torch.randn(shape, device="cuda") * 0.1 if accumulate else None
    plain = pmf.conebeam_project_backward(grid, det, views(vw), dev(dY), shared=shared, accumulate=accumulate,
                                          out=base.clone() if accumulate else None)
    bits = torch.full((1,), -1, dtype=torch.int32, device="cuda")  # the call sets it, whatever it held
    got = pmf.conebeam_project_backward_absmax(grid, det, views(vw), dev(dY), bits, shared=shared,
                                               accumulate=accumulate, out=base.clone() if accumulate else None)
    assert torch.equal(got, plain)
    assert int(bits.item()) == _bits(got)
    if not accumulate:
        assert rel_l2(host(got), oracle.project_backward(grid, 29, 21, 1.0, vw, dY, shared=shared)) <= TOL32


def test_backproject_absmax_of_a_zero_gradient_is_zero():
    grid, det, vw, dY = _bp_problem()
    bits = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    got = pmf.conebeam_project_backward_absmax(grid, det, views(vw), dev(np.zeros_like(dY)), bits)
    assert not torch.any(got) and int(bits.item()) == 0


def _warp_problem(seed, L, P, grid):
    rng = np.random.default_rng(seed)
    V = rng.random(grid.shape).astype(np.float32)
    E = rng.normal(0, 2.0, (L, 3) + grid.shape).astype(np.float32)
    w = rng.uniform(-1, 1, (P, L, 3)).astype(np.float32)
    dW = rng.normal(size=(P,) + grid.shape).astype(np.float32)
    return V, E, w, dW


@pytest.mark.parametrize("L,P,dt", [(3, 6, torch.float32), (2, 5, torch.bfloat16), (6, 3, torch.float32)])
def test_warp_adjoint_bounded_by_the_exact_max_is_bit_identical(L, P, dt):
    """The tile path (L <= 4) and the grid-stride path (L = 6), fp32 and bf16
    grids: the exact max gives the unbounded call's bits; a bound four times
    larger (fewer low-order bits of dV) stays within the fp32 tolerance."""
    grid = Grid(35, 9, 7, 2.0, 2.0, 2.0)
    V, E, w, dW = _warp_problem(60 + L, L, P, grid)
    Vd, Ed = dev(V).to(dt), dev(E).to(dt)
    dWd = dev(dW)
    a = pmf.warp_combine_backward(grid, Vd, Ed, dev(w), dWd)
    bits = torch.tensor([_bits(dWd)], dtype=torch.int32, device="cuda")
    b = pmf.warp_combine_backward_bounded(grid, Vd, Ed, dev(w), dWd, bits)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    loose = (dWd.abs().max() * 4).reshape(1).view(torch.int32).clone()
    c = pmf.warp_combine_backward_bounded(grid, Vd, Ed, dev(w), dWd, loose)
    assert rel_l2(host(c[0]), host(a[0])) <= TOL32
    assert torch.equal(c[1], a[1]) and torch.equal(c[2], a[2])  # dE and the coefficients do not use the bound


def test_back_projector_bound_feeds_the_warp_adjoint():
    """The chain as the training step runs it: dW and its max from the
    back-projector, then the bounded warp adjoint, equal the unfused chain bit
    for bit."""
    grid, det, vw, dY = _bp_problem(31, P=4)
    V, E, w, _ = _warp_problem(32, 3, 4, grid)
    bits = torch.zeros(1, dtype=torch.int32, device="cuda")
    dW1 = pmf.conebeam_project_backward(grid, det, views(vw), dev(dY))
    dW2 = pmf.conebeam_project_backward(grid, det, views(vw), dev(dY), absmax=bits)
    assert torch.equal(dW1, dW2)
    a = pmf.warp_combine_backward(grid, dev(V), dev(E), dev(w), dW1)
    b = pmf.warp_combine_backward(grid, dev(V), dev(E), dev(w), dW2, d_out_absmax=bits)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("shared", [False, True])
def test_conversion_paths_agree_for_any_output_alignment(shared):
    """The accumulator conversion reads and writes four values at a time when
    the output is 16-byte aligned, element by element otherwise; a grid of
    21 x 17 x 13 voxels (not a multiple of 4) also takes the tail path.  Both
    give the same bits and the same maximum."""
    grid = Grid(21, 17, 13, 2.0, 2.0, 2.5)
    rng = np.random.default_rng(41)
    vw = circular_views(3, 400.0, 600.0, 29, 21, 1.8, 1.9, start=0.3)
    dY = dev(rng.normal(size=(3, 21, 29)).astype(np.float32))
    det = Detector(29, 21, 1.0)
    shape = grid.shape if shared else (3,) + grid.shape
    n = int(np.prod(shape))
    b1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    b2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    aligned = pmf.conebeam_project_backward(grid, det, views(vw), dY, shared=shared, absmax=b1)
    assert aligned.data_ptr() % 16 == 0
    buf = torch.empty(n + 1, device="cuda")
    off = buf[1:].view(shape)  # 4 bytes past a 16-byte boundary
    got = pmf.conebeam_project_backward(grid, det, views(vw), dY, shared=shared, out=off, absmax=b2)
    assert got.data_ptr() % 16 == 4
    assert torch.equal(got, aligned) and int(b1.item()) == int(b2.item()) == _bits(aligned)
    acc_a = pmf.conebeam_project_backward(grid, det, views(vw), dY, shared=shared, accumulate=True,
                                          out=aligned.clone())
    acc_o = pmf.conebeam_project_backward(grid, det, views(vw), dY, shared=shared, accumulate=True, out=off)
    assert torch.equal(acc_o, acc_a)
