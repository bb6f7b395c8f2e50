"""GPU parity: every stage of the CUDA path (called through the C ABI) against
the FP64 oracle on the same seeded inputs.  FP32 bar: relative L2 <= 1e-5
(tighter where the arithmetic allows); gradients <= 1e-3 relative."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from synth import Detector, Grid, circular_views, small_workload, fd_subproblem, gaussian_set, mbc_levels
from tests import oracle_chain
from tests.gpu_util import assert_voxels_match, dev, gset, host, pixel_views, rel_l2, tie_band, views

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib_loaded(gpu_lib):
    return gpu_lib


def _rand_gaussians(seed, grid, G, lo, hi, C, std=None):
    return gaussian_set(np.random.default_rng(seed), grid, G, lo, hi, channels=C, value_std=std)


# ------------------------------------------------------------- voxelizer

@pytest.mark.parametrize("kappa", [3.0, float("inf")])
def test_voxelize_ragged_grid(kappa):
    grid = Grid(13, 11, 9, 2.0, 2.5, 3.0)  # several 8^3 tiles with ragged edges
    gs = _rand_gaussians(1, grid, 60, 0.7, 3.0, 1)
    got = host(pmf.gs_voxelize(grid, gset(gs, kappa)))
    ref = oracle.voxelize(grid, gs.mean, gs.scale, gs.quat, gs.value, kappa)
    amb, _ = tie_band(grid, gs, kappa)
    assert_voxels_match(got, ref, amb, TOL32)


@pytest.mark.parametrize("kappa", [3.0, 5.0])
def test_voxelize_small_workload_reference_and_mbc(kappa):
    """At the workloads' kappa = 3 the voxels outside the binary32 tie band hold
    1e-5 and the rest their tie mass; the number of pairs in the band and of
    voxels where a tie actually went the other way are printed.  At kappa = 5
    a flipped tie moves a voxel by at most max|value| e^{-12.5}, so every voxel
    of the volume, ties included, holds 1e-5."""
    wl = small_workload(with_measured=False)
    for gs in (wl.ref, wl.mbc[0]):
        got = host(pmf.gs_voxelize(wl.grid, gset(gs, kappa)))
        ref = oracle.voxelize(wl.grid, gs.mean, gs.scale, gs.quat, gs.value, kappa)
        amb, npairs = tie_band(wl.grid, gs, kappa)
        assert got.shape == (gs.channels,) + wl.grid.shape
        sure, flipped = assert_voxels_match(got, ref, amb, TOL32)
        print(f"kappa {kappa} C={gs.channels}: all-voxel rel-L2 {rel_l2(got, ref):.2e}, {npairs} pairs in the tie "
              f"band, {int((amb > 0).sum())} voxels touched, {flipped} decided the other way")
        assert sure > (0.999 if kappa == 3.0 else 0.99)
        if kappa == 5.0:
            assert rel_l2(got, ref) <= TOL32  # all voxels, ties included


@pytest.mark.parametrize("tile", [(16, 8, 8), (8, 8, 4), (16, 8, 4)])
@pytest.mark.parametrize("C,kappa", [(1, 3.0), (3, 3.0), (3, float("inf"))])
def test_voxelize_bin_tiles_give_the_same_bits(tile, C, kappa):
    """Every bin tile sums the same exactly-rounded terms, so the volume is the
    default tile's bit for bit -- on a ragged grid, through the pair lists and
    through the overflow path that scans every Gaussian -- and it matches the
    oracle like the default."""
    grid = Grid(37, 22, 13, 2.0, 2.0, 2.5)
    gs = _rand_gaussians(5 + C, grid, 120, 0.7, 3.5, C, 2.0 if C == 3 else None)
    g = gset(gs, kappa)
    base = pmf.gs_voxelize(grid, g)
    got = pmf.gs_voxelize_tiled(grid, g, tile)
    assert torch.equal(base, got)
    assert torch.equal(base, pmf.gs_voxelize(grid, g, tile=tile, pair_capacity=11))
    ref = oracle.voxelize(grid, gs.mean, gs.scale, gs.quat, gs.value, kappa)
    amb, _ = tie_band(grid, gs, kappa)
    assert_voxels_match(host(got), ref, amb, TOL32)
    # the pair count depends on the tile: a tile made of whole 8^3 tiles lists
    # each Gaussian in at most as many tiles, one that subdivides 8^3 in at least
    n8 = pmf.gs_voxelize_count(grid, g)
    nt = pmf.gs_voxelize_tiled_count(grid, g, tile)
    if all(t >= 8 for t in tile):
        assert nt <= n8
    elif all(t <= 8 for t in tile):
        assert nt >= n8
    assert nt > 0


def test_voxelize_list_overflow_falls_back_correctly():
    """A pair capacity far below the overlap count routes tiles through the
    scan-everything path; the result must not change by a bit."""
    grid = Grid(24, 20, 17, 2.0, 2.0, 2.0)
    gs = gset(_rand_gaussians(2, grid, 300, 0.7, 4.0, 3, 2.0), 3.0)
    full = pmf.gs_voxelize(grid, gs)
    small = pmf.gs_voxelize(grid, gs, pair_capacity=37)
    zero = pmf.gs_voxelize(grid, gs, pair_capacity=0)
    torch.testing.assert_close(full, small, rtol=0, atol=0)
    torch.testing.assert_close(full, zero, rtol=0, atol=0)


def test_voxelize_edge_cases():
    grid = Grid(9, 8, 7, 2.0, 2.0, 2.0)
    empty = pmf.Gaussians(dev(np.zeros((0, 3))), dev(np.ones((0, 3))), dev(np.ones((0, 4))), dev(np.zeros((0, 1))))
    assert float(pmf.gs_voxelize(grid, empty).abs().max()) == 0.0
    # entirely outside the volume
    far = pmf.Gaussians(dev([[500.0, 0, 0]]), dev([[1.0, 1, 1]]), dev([[1.0, 0, 0, 0]]), dev([[1.0]]), 3.0)
    assert float(pmf.gs_voxelize(grid, far).abs().max()) == 0.0
    # one voxel grid
    g1 = Grid(1, 1, 1, 1.0, 1.0, 1.0)
    one = pmf.Gaussians(dev([[0.0, 0, 0]]), dev([[1.0, 1, 1]]), dev([[1.0, 0, 0, 0]]), dev([[2.0]]), 3.0)
    assert float(pmf.gs_voxelize(g1, one).item()) == pytest.approx(2.0, rel=1e-7)


def test_voxelize_is_bit_reproducible():
    wl = small_workload(with_measured=False)
    gs = gset(wl.mbc[0], wl.kappa)
    a = pmf.gs_voxelize(wl.grid, gs)
    b = pmf.gs_voxelize(wl.grid, gs)
    assert torch.equal(a, b)


@pytest.mark.parametrize("C,kappa", [(1, float("inf")), (3, float("inf")), (1, 3.0), (3, 2.5)])
def test_voxelize_backward_matches_oracle(C, kappa):
    grid = Grid(12, 10, 11, 2.0, 2.0, 2.0)
    gs = _rand_gaussians(3 + C, grid, 40, 0.8, 3.0, C, 2.0 if C == 3 else None)
    rng = np.random.default_rng(7)
    d_out = rng.normal(size=(C,) + grid.shape).astype(np.float32)
    got = pmf.gs_voxelize_backward(grid, gset(gs, kappa), dev(d_out))
    ref = oracle.voxelize_backward(grid, gs.mean, gs.scale, gs.quat, gs.value, d_out, kappa)
    for name, g_, r_ in zip(("mean", "scale", "quat", "value"), got, ref):
        assert rel_l2(host(g_), r_) <= 1e-4, name


@pytest.mark.parametrize("C", [2, 4])
def test_voxelize_two_and_four_channels(C):
    """The two- and four-channel forms against the oracle: the forward on the
    default and the widest bin tile (same bits; at four channels its staged
    records need more than 48 KB of shared memory) and the adjoint."""
    grid = Grid(21, 18, 15, 2.0, 2.0, 2.0)
    gs = _rand_gaussians(40 + C, grid, 80, 0.7, 3.0, C, 1.5)
    g = gset(gs, 3.0)
    base = pmf.gs_voxelize(grid, g)
    assert torch.equal(base, pmf.gs_voxelize_tiled(grid, g, (16, 8, 8)))
    ref = oracle.voxelize(grid, gs.mean, gs.scale, gs.quat, gs.value, 3.0)
    amb, _ = tie_band(grid, gs, 3.0)
    assert_voxels_match(host(base), ref, amb, TOL32)
    d_out = np.random.default_rng(60 + C).normal(size=(C,) + grid.shape).astype(np.float32)
    got = pmf.gs_voxelize_backward(grid, gset(gs, float("inf")), dev(d_out))
    refb = oracle.voxelize_backward(grid, gs.mean, gs.scale, gs.quat, gs.value, d_out, float("inf"))
    for name, g_, r_ in zip(("mean", "scale", "quat", "value"), got, refb):
        assert rel_l2(host(g_), r_) <= 1e-4, name


def test_voxelize_backward_vector_loads_give_the_same_bits():
    """With several channels on 16-byte rows the adjoint reads the upstream
    gradient 16 bytes at a time; the same values at a pointer off the 16-byte
    boundary take scalar loads.  The voxels visited and their order are the
    same, so the gradients are too, bit for bit, and they match the oracle."""
    grid = Grid(24, 14, 11, 2.0, 2.0, 2.0)
    gs = _rand_gaussians(71, grid, 60, 0.8, 4.0, 3, 2.0)
    d_out = np.random.default_rng(72).normal(size=(3,) + grid.shape).astype(np.float32)
    aligned = dev(d_out)
    buf = torch.zeros(aligned.numel() + 1, device="cuda")
    buf[1:] = aligned.reshape(-1)
    shifted = buf[1:].view(aligned.shape)  # 4 bytes past a 16-byte boundary
    assert shifted.data_ptr() % 16 != 0 and aligned.data_ptr() % 16 == 0
    g = gset(gs, 3.0)
    got_v = pmf.gs_voxelize_backward(grid, g, aligned)
    got_s = pmf.gs_voxelize_backward(grid, g, shifted)
    for a, b in zip(got_v, got_s):
        assert torch.equal(a, b)
    ref = oracle.voxelize_backward(grid, gs.mean, gs.scale, gs.quat, gs.value, d_out, 3.0)
    for name, g_, r_ in zip(("mean", "scale", "quat", "value"), got_v, ref):
        assert rel_l2(host(g_), r_) <= 1e-4, name


def test_voxelize_backward_accumulates():
    grid = Grid(8, 8, 8, 2.0, 2.0, 2.0)
    gs = gset(_rand_gaussians(9, grid, 10, 1.0, 2.0, 1), 3.0)
    d_out = dev(np.random.default_rng(1).normal(size=(1,) + grid.shape))
    a = pmf.gs_voxelize_backward(grid, gs, d_out)
    b = pmf.gs_voxelize_backward(grid, gs, d_out, grads=tuple(t.clone() for t in a), accumulate=True)
    for x, y in zip(a, b):
        torch.testing.assert_close(2 * x, y, rtol=1e-6, atol=1e-6)


# --------------------------------------------------- combine and warp

def _mbc_and_ref(grid, seed, L=3, P=5):
    rng = np.random.default_rng(seed)
    V = rng.random(grid.shape).astype(np.float32)
    E = rng.normal(0, 2.0, (L, 3) + grid.shape).astype(np.float32)
    w = rng.uniform(-1, 1, (P, L, 3)).astype(np.float32)
    return V, E, w


def test_combine_and_warp_match_oracle():
    grid = Grid(21, 17, 13, 2.0, 2.0, 2.0)
    V, E, w = _mbc_and_ref(grid, 11)
    D = pmf.mbc_combine(grid, dev(E), dev(w))
    Dref = oracle.combine(E, w)
    assert rel_l2(host(D), Dref) <= 1e-6
    W = pmf.warp_volume(grid, dev(V), D)
    Wref = oracle.warp(grid, V, host(D))
    assert rel_l2(host(W), Wref) <= TOL32
    Wf = pmf.warp_combine(grid, dev(V), dev(E), dev(w))
    assert rel_l2(host(Wf), oracle.warp(grid, V, Dref)) <= TOL32


@pytest.mark.parametrize("L,dt", [(2, torch.bfloat16), (3, torch.float16), (6, torch.bfloat16)])
def test_warp_combine_fp32_output_from_reduced_grids(L, dt):
    """warp_combine_mixed: bf16 / fp16 V and E, fp32 W (the 8x8x4 tile kernel
    for L <= 4, the per-voxel kernel above).  W is the fp32 warp of the stored
    grids' values, and rounding it to the grids' format gives the same-format
    entry point's output bit for bit (both round the same fp32 sum once)."""
    grid = Grid(37, 11, 9, 2.0, 2.0, 2.0)
    V, E, w = _mbc_and_ref(grid, 50 + L, L=L, P=3)
    Vd, Ed = dev(V).to(dt), dev(E).to(dt)
    W32 = torch.empty((3,) + grid.shape, device="cuda")
    pmf.warp_combine(grid, Vd, Ed, dev(w), out=W32)
    Vq, Eq = host(Vd).astype(np.float64), host(Ed).astype(np.float64)
    assert rel_l2(host(W32), oracle.warp(grid, Vq, oracle.combine(Eq, w))) <= TOL32
    Wn = pmf.warp_combine(grid, Vd, Ed, dev(w))
    assert Wn.dtype == dt and torch.equal(W32.to(dt), Wn)


def test_zero_dvf_warp_is_bitwise_identity():
    grid = Grid(9, 8, 7, 2.0, 2.0, 2.0)
    V = dev(np.random.default_rng(3).random(grid.shape))
    W = pmf.warp_volume(grid, V, torch.zeros((2, 3) + grid.shape, device="cuda"))
    assert torch.equal(W[0], V) and torch.equal(W[1], V)


def test_combine_and_warp_backward_match_oracle():
    grid = Grid(19, 15, 12, 2.0, 2.0, 2.0)
    V, E, w = _mbc_and_ref(grid, 12, L=3, P=4)
    rng = np.random.default_rng(13)
    dW = rng.normal(size=(4,) + grid.shape).astype(np.float32)
    Dref = oracle.combine(E, w)
    dV_ref, dD_ref = oracle.warp_backward(grid, V, Dref, dW)
    dE_ref, dw_ref = oracle.combine_backward(E, w, dD_ref)
    D = pmf.mbc_combine(grid, dev(E), dev(w))
    dV, dD = pmf.warp_volume_backward(grid, dev(V), D, dev(dW))
    assert rel_l2(host(dV), dV_ref) <= TOL32
    assert rel_l2(host(dD), dD_ref) <= 1e-4
    dE, dw = pmf.mbc_combine_backward(grid, dev(E), dev(w), dev(dD_ref.astype(np.float32)))
    dE_r2, dw_r2 = oracle.combine_backward(E, w, dD_ref.astype(np.float32))
    assert rel_l2(host(dE), dE_r2) <= 1e-6
    assert rel_l2(host(dw), dw_r2) <= 1e-5
    fdV, fdE, fdw = pmf.warp_combine_backward(grid, dev(V), dev(E), dev(w), dev(dW))
    assert rel_l2(host(fdV), dV_ref) <= TOL32
    assert rel_l2(host(fdE), dE_ref) <= 1e-4
    assert rel_l2(host(fdw), dw_ref) <= 1e-4


@pytest.mark.parametrize("L", [1, 2, 4])
def test_fused_warp_tile_kernels_every_level_count(L):
    """The tile kernels (8x8x4 forward, 8x16x4 adjoint) are instantiated per level count (L <= 4); each
    reduces its 3 L coefficient-gradient values per view across the warp by
    halving exchange, whose slot layout depends on 3 L.  Forward and adjoint of
    every instance against the oracle on a ragged grid."""
    grid = Grid(35, 9, 7, 2.0, 2.0, 2.0)
    V, E, w = _mbc_and_ref(grid, 90 + L, L=L, P=6)
    D = oracle.combine(E, w)
    W = host(pmf.warp_combine(grid, dev(V), dev(E), dev(w)))
    assert rel_l2(W, oracle.warp(grid, V, D)) <= TOL32
    dW = np.random.default_rng(95 + L).normal(size=(6,) + grid.shape).astype(np.float32)
    dV_ref, dD_ref = oracle.warp_backward(grid, V, D, dW)
    dE_ref, dw_ref = oracle.combine_backward(E, w, dD_ref)
    dV, dE, dw = pmf.warp_combine_backward(grid, dev(V), dev(E), dev(w), dev(dW))
    assert rel_l2(host(dV), dV_ref) <= TOL32
    assert rel_l2(host(dE), dE_ref) <= 1e-4
    assert rel_l2(host(dw), dw_ref) <= 1e-4


def test_fused_warp_displacements_beyond_the_staged_halo():
    """MBC vectors of 12 mm std on 2 mm voxels: many displaced samples leave
    the tile's staged 4-voxel halo (the kernels then read and scatter through
    global memory), some leave the grid, and one voxel's displacement is 10^30
    mm (outside the range of the fast floor; zero padding).  Forward and
    adjoint still match the oracle."""
    grid = Grid(45, 13, 10, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(71)
    L, P = 2, 3
    V = rng.random(grid.shape).astype(np.float32)
    E = rng.normal(0, 12.0, (L, 3) + grid.shape).astype(np.float32)
    E[0, 1, 4, 6, 20] = 1e30
    w = rng.uniform(-1, 1, (P, L, 3)).astype(np.float32)
    w[:, 0, 1] = np.abs(w[:, 0, 1]) + 0.1
    D = oracle.combine(E, w)
    far = np.abs(D) / 2.0 > 4.0
    assert far.any(axis=1).mean() > 0.2
    W = host(pmf.warp_combine(grid, dev(V), dev(E), dev(w)))
    Wref = oracle.warp(grid, V, D)
    assert np.all(W[:, 4, 6, 20] == 0.0) and np.all(Wref[:, 4, 6, 20] == 0.0)
    assert rel_l2(W, Wref) <= TOL32
    dW = rng.normal(size=(P,) + grid.shape).astype(np.float32)
    dW[:, 4, 6, 20] = 0.0  # the 10^30 voxel has no finite DVF gradient to compare
    dV_ref, dD_ref = oracle.warp_backward(grid, V, D, dW)
    dE_ref, dw_ref = oracle.combine_backward(E, w, dD_ref)
    dV, dE, dw = pmf.warp_combine_backward(grid, dev(V), dev(E), dev(w), dev(dW))
    assert rel_l2(host(dV), dV_ref) <= TOL32
    assert rel_l2(host(dE), dE_ref) <= 1e-4
    assert rel_l2(host(dw), dw_ref) <= 1e-4


def test_warp_backward_is_bit_reproducible():
    grid = Grid(19, 15, 12, 2.0, 2.0, 2.0)
    V, E, w = _mbc_and_ref(grid, 14, L=3, P=4)
    dW = dev(np.random.default_rng(15).normal(size=(4,) + grid.shape))
    a = pmf.warp_combine_backward(grid, dev(V), dev(E), dev(w), dW)
    b = pmf.warp_combine_backward(grid, dev(V), dev(E), dev(w), dW)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


# ------------------------------------------------------------ projector

@pytest.mark.parametrize("nu,nv", [(37, 23), (16, 16)])
def test_project_ragged_detector(nu, nv):
    grid = Grid(20, 18, 14, 2.0, 2.0, 2.5)
    rng = np.random.default_rng(21)
    vol = rng.random((3,) + grid.shape).astype(np.float32)
    vw = circular_views(3, 400.0, 600.0, nu, nv, 1.8, 1.9, start=0.37)
    got = host(pmf.conebeam_project(grid, Detector(nu, nv, 1.0), views(vw), dev(vol)))
    ref = oracle.project(grid, nu, nv, 1.0, vw, vol)
    assert rel_l2(got, ref) <= TOL32


@pytest.mark.parametrize("shared", [False, True])
def test_project_bulk_copy_staging_equals_plain_staging(shared):
    """fp32 volumes whose rows are whole 16-byte lines get their shared-memory
    boxes by bulk tensor copies; bf16 volumes by plain loads.  On values that
    bf16 holds exactly both forms must give the same projections bit for bit
    (the samples and their order do not depend on how the box was filled),
    and no bulk copy may time out."""
    grid = Grid(48, 44, 36, 2.0, 2.0, 2.0)
    P = 4
    vol = np.random.default_rng(23).random((P,) + grid.shape).astype(np.float32)
    vb = dev(vol).to(torch.bfloat16)
    src = vb[0] if shared else vb
    vw = circular_views(P, 500.0, 750.0, 70, 54, 2.2, 2.2, start=0.2)
    det = Detector(70, 54, 1.0)
    pmf.device_counters(reset=True)
    y32 = pmf.conebeam_project(grid, det, views(vw), src.float(), shared=shared)
    y16 = pmf.conebeam_project(grid, det, views(vw), src, shared=shared)
    assert torch.equal(y32, y16)
    assert pmf.device_counters()["timeout"] == 0
    pmf.device_status()
    ref = oracle.project(grid, 70, 54, 1.0, vw, host(src), shared=shared)
    assert rel_l2(host(y32), ref) <= TOL32


def test_bulk_copy_wait_timeout_is_reported_and_recovers():
    """The failure path of the bulk-copy projector's bounded wait, without a
    fault: the test hook arms each chunk's mbarrier but issues no copy, so every
    CTA that stages a box gives up after its short limit with nothing in flight.
    Its pixels are NaN (the others equal a clean launch), the timeout counter
    rises and pmf_device_status reports PMF_ETIMEOUT; once the hook is off, the
    next launch equals a clean one bit for bit and the status is OK again."""
    grid = Grid(48, 44, 36, 2.0, 2.0, 2.0)
    P = 3
    vol = dev(np.random.default_rng(24).random(grid.shape).astype(np.float32))
    vw = views(circular_views(P, 500.0, 750.0, 70, 54, 2.2, 2.2, start=0.3))
    det = Detector(70, 54, 1.0)
    pmf.device_counters(reset=True)
    clean = pmf.conebeam_project(grid, det, vw, vol, shared=True)
    pmf.device_status()
    try:
        pmf.ops.pmf_debug_stall_bulk_copies(True)
        stalled = pmf.conebeam_project(grid, det, vw, vol, shared=True)
        torch.cuda.synchronize()
    finally:
        pmf.ops.pmf_debug_stall_bulk_copies(False)
    # a CTA that stages a box times out and writes NaN to all its pixels; one
    # whose every chunk takes the global-gather fallback computes as usual
    nan = torch.isnan(stalled)
    assert bool(torch.equal(stalled[~nan], clean[~nan]))
    hit = clean != 0
    assert float(nan[hit].float().mean()) > 0.5
    assert pmf.device_counters()["timeout"] > 0
    with pytest.raises(pmf.PmfError, match="ETIMEOUT"):
        pmf.device_status()
    pmf.device_counters(reset=True)
    again = pmf.conebeam_project(grid, det, vw, vol, shared=True)
    assert torch.equal(again, clean)
    assert pmf.device_counters()["timeout"] == 0
    pmf.device_status()


def test_project_small_workload_voxelized_reference():
    wl = small_workload(with_measured=False)
    V = pmf.gs_voxelize(wl.grid, gset(wl.ref, wl.kappa))[0]
    Vh = host(V)
    got = host(pmf.conebeam_project(wl.grid, wl.det, views(wl.views), V, shared=True))
    ref = oracle.project(wl.grid, wl.det.nu, wl.det.nv, wl.det.step_mm, wl.views, Vh)
    assert rel_l2(got, ref) <= TOL32


def test_project_shared_volume_and_rays_that_miss():
    grid = Grid(16, 16, 16, 2.0, 2.0, 2.0)
    vol = np.random.default_rng(4).random(grid.shape).astype(np.float32)
    vw = circular_views(2, 300.0, 450.0, 40, 40, 2.0, 2.0)  # outer pixels miss the volume
    got = host(pmf.conebeam_project(grid, Detector(40, 40, 1.0), views(vw), dev(vol), shared=True))
    ref = oracle.project(grid, 40, 40, 1.0, vw, vol)
    assert rel_l2(got, ref) <= TOL32
    assert np.all(got[ref == 0] == 0)


@pytest.mark.parametrize("shared", [False, True])
def test_backproject_matches_oracle_and_is_reproducible(shared):
    grid = Grid(20, 18, 14, 2.0, 2.0, 2.5)
    rng = np.random.default_rng(22)
    vw = circular_views(3, 400.0, 600.0, 29, 21, 1.8, 1.9, start=0.1)
    dY = rng.normal(size=(3, 21, 29)).astype(np.float32)
    det = Detector(29, 21, 1.0)
    got = pmf.conebeam_project_backward(grid, det, views(vw), dev(dY), shared=shared)
    again = pmf.conebeam_project_backward(grid, det, views(vw), dev(dY), shared=shared)
    assert torch.equal(got, again)
    ref = oracle.project_backward(grid, 29, 21, 1.0, vw, dY, shared=shared)
    assert rel_l2(host(got), ref) <= TOL32


def test_marchers_with_boxes_wider_than_32_voxels():
    """Samples one voxel apart, so a 48-sample chunk spans about 48 voxels
    along the rays and x-major tiles have boxes wider than 32 voxels: the plain
    staging and the adjoint hold them with rows 65 words apart (no chunk falls
    back), while the bulk copies, 44 voxels wide, gather those chunks from
    global memory instead.  Both staging forms still agree bit for bit and both
    directions match the oracle."""
    grid = Grid(64, 48, 24, 1.0, 1.0, 1.0)
    P, nu, nv = 4, 40, 24
    vw = circular_views(P, 300.0, 450.0, nu, nv, 0.2, 0.2, start=0.05)
    det = Detector(nu, nv, 1.0)
    vol = np.random.default_rng(81).random((P,) + grid.shape).astype(np.float32)
    vb = dev(vol).to(torch.bfloat16)
    pmf.device_counters(reset=True)
    y16 = pmf.conebeam_project(grid, det, views(vw), vb)  # plain staging
    assert pmf.device_counters(reset=True)["project_box_fallback"] == 0
    y32 = pmf.conebeam_project(grid, det, views(vw), vb.float())  # bulk copies
    assert pmf.device_counters(reset=True)["project_box_fallback"] > 0
    assert torch.equal(y32, y16)
    ref = oracle.project(grid, nu, nv, 1.0, vw, host(vb.float()))
    assert rel_l2(host(y32), ref) <= TOL32
    dY = np.random.default_rng(82).normal(size=(P, nv, nu)).astype(np.float32)
    got = pmf.conebeam_project_backward(grid, det, views(vw), dev(dY))
    assert pmf.device_counters(reset=True)["backproject_box_fallback"] == 0
    refb = oracle.project_backward(grid, nu, nv, 1.0, vw, dY)
    assert rel_l2(host(got), refb) <= TOL32


def test_loss_matches_oracle():
    rng = np.random.default_rng(5)
    a, b = rng.normal(size=(3, 17, 29)).astype(np.float32), rng.normal(size=(3, 17, 29)).astype(np.float32)
    for kind in (1, 2):
        loss, g = pmf.projection_loss(kind, dev(a), dev(b))
        lref, gref = oracle.loss(kind, a, b)
        assert float(loss.item()) == pytest.approx(lref, rel=1e-6)
        assert rel_l2(host(g), gref) <= 1e-6
        # arrays off the 16-byte grid (the kernel's scalar form)
        ua, ub = torch.zeros(a.size + 1, device="cuda"), torch.zeros(b.size + 1, device="cuda")
        ua[1:] = dev(a).reshape(-1)
        ub[1:] = dev(b).reshape(-1)
        loss_u, g_u = pmf.projection_loss(kind, ua[1:].reshape(a.shape), ub[1:].reshape(b.shape))
        assert float(loss_u.item()) == pytest.approx(lref, rel=1e-6)
        assert rel_l2(host(g_u), gref) <= 1e-6


def test_loss_at_the_paper_batch_size():
    """32 projections of 512x384 (the vectorised form over many grid-stride
    rounds) against a float64 sum."""
    rng = np.random.default_rng(6)
    a = rng.normal(size=(32, 384, 512)).astype(np.float32)
    b = rng.normal(size=(32, 384, 512)).astype(np.float32)
    for kind in (1, 2):
        loss, g = pmf.projection_loss(kind, dev(a), dev(b))
        lref, gref = oracle.loss(kind, a, b)
        assert float(loss.item()) == pytest.approx(lref, rel=1e-6)
        assert rel_l2(host(g), gref) <= 1e-6


# ------------------------------------------------------------- the chain

def _gpu_step(wl, meas, kind=2):
    g, det = wl.grid, wl.det
    ref = gset(wl.ref, wl.kappa)
    mbcs = [gset(m, wl.kappa) for m in wl.mbc]
    V = pmf.gs_voxelize(g, ref)[0]
    E = torch.stack([pmf.gs_voxelize(g, m) for m in mbcs])
    w = dev(wl.coeff)
    vt = views(wl.views)
    W = pmf.warp_combine(g, V, E, w)
    Y = pmf.conebeam_project(g, det, vt, W, shared=False)
    loss, dY = pmf.projection_loss(kind, Y, dev(meas))
    dW = pmf.conebeam_project_backward(g, det, vt, dY, shared=False)
    dV, dE, dw = pmf.warp_combine_backward(g, V, E, w, dW)
    gref = pmf.gs_voxelize_backward(g, ref, dV.reshape(1, *g.shape))
    gmbc = [pmf.gs_voxelize_backward(g, m, dE[l]) for l, m in enumerate(mbcs)]
    return loss, Y, dict(coeff=dw, ref=gref, mbc=gmbc, dV=dV, dE=dE, dW=dW)


@pytest.mark.parametrize("kind", [2, 1])
def test_full_chain_forward_and_gradients_match_oracle(kind):
    wl = fd_subproblem()
    meas = wl.measured
    loss, Y, grads = _gpu_step(wl, meas, kind)
    lref, gref, fref = oracle_chain.step(wl, meas, kind=kind)
    assert rel_l2(host(Y), fref["Y"]) <= TOL32
    assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
    assert rel_l2(host(grads["coeff"]), gref["coeff"]) <= 1e-3
    for i in range(4):
        assert rel_l2(host(grads["ref"][i]), gref["ref"][i]) <= 1e-3
        for l in range(3):
            assert rel_l2(host(grads["mbc"][l][i]), gref["mbc"][l][i]) <= 1e-3


def test_small_workload_chain_forward_matches_oracle():
    wl = small_workload()
    loss, Y, _ = _gpu_step(wl, wl.measured)
    f = oracle_chain.forward(wl)
    assert rel_l2(host(Y), f["Y"]) <= TOL32


def test_projector_box_fallback_paths_match_oracle():
    """Pixels far larger than voxels make each chunk's voxel box exceed shared
    memory, forcing the global-memory paths of both projector and adjoint."""
    grid = Grid(40, 40, 40, 0.5, 0.5, 0.5)
    rng = np.random.default_rng(31)
    vol = rng.random(grid.shape).astype(np.float32)
    vw = circular_views(2, 60.0, 90.0, 18, 17, 12.0, 12.0, start=0.3)
    det = Detector(18, 17, 0.25)
    got = host(pmf.conebeam_project(grid, det, views(vw), dev(vol), shared=True))
    ref = oracle.project(grid, 18, 17, 0.25, vw, vol)
    assert rel_l2(got, ref) <= TOL32
    dY = rng.normal(size=(2, 17, 18)).astype(np.float32)
    gb = host(pmf.conebeam_project_backward(grid, det, views(vw), dev(dY), shared=True))
    assert rel_l2(gb, oracle.project_backward(grid, 18, 17, 0.25, vw, dY, shared=True)) <= TOL32


def test_projector_source_inside_volume():
    """Samples start at m = 0 when the source sits inside the padded volume."""
    grid = Grid(24, 24, 16, 2.0, 2.0, 2.0)
    vol = np.random.default_rng(32).random(grid.shape).astype(np.float32)
    vw = circular_views(3, 10.0, 60.0, 20, 14, 3.0, 3.0, start=0.2)
    det = Detector(20, 14, 1.0)
    got = host(pmf.conebeam_project(grid, det, views(vw), dev(vol), shared=True))
    assert rel_l2(got, oracle.project(grid, 20, 14, 1.0, vw, vol)) <= TOL32
    dY = np.random.default_rng(33).normal(size=(3, 14, 20)).astype(np.float32)
    gb = host(pmf.conebeam_project_backward(grid, det, views(vw), dev(dY), shared=True))
    assert rel_l2(gb, oracle.project_backward(grid, 20, 14, 1.0, vw, dY, shared=True)) <= TOL32


@pytest.mark.parametrize("L,std", [(3, 6.0), (1, 1.0), (4, 3.0)])
def test_fused_warp_tiles_with_large_displacements(L, std):
    """Ragged tiles (8x8x4 forward, 8x16x4 adjoint) and displacements well past the 4-voxel shared-memory
    halo (std 6 mm at 2 mm voxels): both the box and the direct scatter paths."""
    grid = Grid(37, 9, 7, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(40 + L)
    V = rng.random(grid.shape).astype(np.float32)
    E = rng.normal(0, std, (L, 3) + grid.shape).astype(np.float32)
    w = rng.uniform(-1, 1, (5, L, 3)).astype(np.float32)
    dW = rng.normal(size=(5,) + grid.shape).astype(np.float32)
    D = oracle.combine(E, w)
    assert rel_l2(host(pmf.warp_combine(grid, dev(V), dev(E), dev(w))), oracle.warp(grid, V, D)) <= TOL32
    dV_ref, dD_ref = oracle.warp_backward(grid, V, D, dW)
    dE_ref, dw_ref = oracle.combine_backward(E, w, dD_ref)
    dV, dE, dw = pmf.warp_combine_backward(grid, dev(V), dev(E), dev(w), dev(dW))
    assert rel_l2(host(dV), dV_ref) <= TOL32
    assert rel_l2(host(dE), dE_ref) <= 1e-4
    assert rel_l2(host(dw), dw_ref) <= 1e-4


def test_voxelize_backward_unsplit_many_gaussians():
    """Enough Gaussians that each is handled by a single warp (no slab split)."""
    grid = Grid(40, 36, 30, 2.0, 2.0, 2.0)
    gs = _rand_gaussians(55, grid, 24000, 0.5, 2.0, 1)
    d_out = np.random.default_rng(56).normal(size=(1,) + grid.shape).astype(np.float32)
    got = pmf.gs_voxelize_backward(grid, gset(gs, 3.0), dev(d_out))
    ref = oracle.voxelize_backward(grid, gs.mean, gs.scale, gs.quat, gs.value, d_out, 3.0)
    for name, g_, r_ in zip(("mean", "scale", "quat", "value"), got, ref):
        assert rel_l2(host(g_), r_) <= 1e-4, name
