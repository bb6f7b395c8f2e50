"""The paper-scale scan at 1 mm voxels (400x400x200, 32 million voxels; Sec. 4's
batch-8 case): the voxelizer on sampled 8^3 crops against the oracle (the
oracle voxelizes each crop exactly, with the means shifted to the crop's
centre), the projector on sampled pixels of the voxelized volume against the
oracle's ray sums, the projector pair by the adjoint identity, and the whole
batch-8 training step (finite, bit-reproducible, within the paper's memory)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300.pipeline import ForwardAdjoint
from synth import Grid, paper_workload_1mm, select_batch
from tests.gpu_util import assert_voxels_match, dev, gset, host, pixel_views, rel_l2, tie_band, views

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wl():
    return paper_workload_1mm(p=660)


@pytest.fixture(scope="module")
def V(wl):
    return pmf.gs_voxelize(wl.grid, gset(wl.ref, wl.kappa))[0]


def test_1mm_voxelization_on_sampled_crops(wl, V):
    g = wl.grid
    rng = np.random.default_rng(81)
    D = 8
    Vh = host(V)
    m = wl.ref
    for _ in range(6):
        o = rng.integers(0, [g.nx - D, g.ny - D, g.nz - D])
        c = np.array([(o[k] + D / 2 - n / 2) * 1.0 for k, n in enumerate((g.nx, g.ny, g.nz))])
        crop = Grid(D, D, D, 1.0, 1.0, 1.0)
        sh = m.mean.astype(np.float64) - c
        ref = oracle.voxelize(crop, sh, m.scale, m.quat, m.value, wl.kappa)
        amb, _ = tie_band(crop, m, wl.kappa, offset=c, mean=sh)
        got = Vh[o[2]:o[2] + D, o[1]:o[1] + D, o[0]:o[0] + D][None]
        assert_voxels_match(got, ref, amb, 1e-5)


def test_1mm_projection_on_sampled_pixels(wl, V):
    g, det = wl.grid, wl.det
    vw = wl.views[select_batch(wl.p, 8, 0)]
    Y = host(pmf.conebeam_project(g, det, views(vw), V, shared=True))
    Vh = host(V)
    rng = np.random.default_rng(82)
    pix = [(int(rng.integers(0, 8)), int(rng.integers(0, det.nv)), int(rng.integers(0, det.nu))) for _ in range(24)]
    ref = oracle.project(g, 1, 1, det.step_mm, pixel_views(vw, det.nu, det.nv, pix), Vh)[:, 0, 0]
    got = np.array([Y[p, b, a] for p, b, a in pix])
    assert rel_l2(got, ref) <= 1e-5


def test_1mm_projector_adjoint_identity(wl):
    g, det = wl.grid, wl.det
    vw = views(wl.views[select_batch(wl.p, 2, 0)])
    gen = torch.Generator("cuda").manual_seed(83)
    x = torch.rand((2,) + g.shape, device="cuda", generator=gen)
    y = torch.randn((2, det.nv, det.nu), device="cuda", generator=gen)
    Px = pmf.conebeam_project(g, det, vw, x, shared=False)
    Pty = pmf.conebeam_project_backward(g, det, vw, y, shared=False)
    lhs = float((Px.double() * y.double()).sum())
    rhs = float((x.double() * Pty.double()).sum())
    assert rhs == pytest.approx(lhs, rel=1e-5)


def test_1mm_training_step_batch_8(wl):
    """The batch-8 step at 1 mm (bf16 V and E, fp32 W): finite and bit-reproducible,
    and its device memory stays well inside the paper's 65 GB."""
    torch.cuda.reset_peak_memory_stats()
    idx = select_batch(wl.p, 8, 0)
    meas = np.random.default_rng(84).random((8, wl.det.nv, wl.det.nu)).astype(np.float32) * 400
    step = ForwardAdjoint(wl.grid, wl.det, gset(wl.ref, wl.kappa), [gset(m, wl.kappa) for m in wl.mbc], batch=8,
                          dtype=torch.bfloat16)
    args = (views(wl.views[idx]), dev(wl.coeff[idx]), dev(meas))
    l1 = step.run(*args).clone()
    g1 = [t.clone() for t in step.g_ref + step.g_wc]
    l2 = step.run(*args)
    torch.cuda.synchronize()
    assert torch.equal(l1, l2) and torch.isfinite(l1).all()
    for a, b in zip(g1, step.g_ref + step.g_wc):
        assert torch.equal(a, b) and torch.isfinite(a).all()
    peak = torch.cuda.max_memory_allocated() / 2 ** 30
    print(f"1 mm, batch 8: peak device memory {peak:.1f} GiB")
    assert peak < 65.0
