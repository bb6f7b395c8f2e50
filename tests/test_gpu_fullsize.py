"""Parity at the paper-scale sizes the benchmark runs (200x200x100 @ 2 mm,
100,000 reference Gaussians, MBC levels 500/2,000/8,000, 512x384 detector,
batch of 32 views), in the benchmark's launch configuration.  Each stage is fed
oracle-side inputs; where the oracle is too slow for whole outputs it is
evaluated on sampled pixels, and the adjoints are also checked by the
dot-product identity over the full batch."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300.pipeline import ForwardAdjoint
from synth import paper_workload, select_batch
from tests.gpu_util import assert_voxels_match, dev, gset, host, pixel_views, rel_l2, tie_band, views

pytestmark = pytest.mark.gpu

B = 32


@pytest.fixture(scope="module")
def wl():
    return paper_workload(p=660)


@pytest.fixture(scope="module")
def oracle_volumes(wl):
    g = wl.grid
    V = oracle.voxelize(g, wl.ref.mean, wl.ref.scale, wl.ref.quat, wl.ref.value, wl.kappa)[0]
    E = np.stack([oracle.voxelize(g, m.mean, m.scale, m.quat, m.value, wl.kappa) for m in wl.mbc])
    return V, E


def _batch(wl):
    idx = select_batch(wl.p, B, 0)
    return wl.views[idx], wl.coeff[idx]


def test_fullsize_voxelization(wl, oracle_volumes):
    V, E = oracle_volumes
    g = wl.grid
    got = host(pmf.gs_voxelize(g, gset(wl.ref, wl.kappa)))
    amb, npairs = tie_band(g, wl.ref, wl.kappa)
    sure, flipped = assert_voxels_match(got, V[None], amb, 1e-5)
    print(f"reference set: {npairs} pairs in the tie band, {flipped} voxels decided the other way")
    assert sure > 0.999
    for l, m in enumerate(wl.mbc):
        got = host(pmf.gs_voxelize(g, gset(m, wl.kappa)))
        amb, npairs = tie_band(g, m, wl.kappa)
        sure, flipped = assert_voxels_match(got, E[l], amb, 1e-5)
        print(f"MBC level {l}: {npairs} pairs in the tie band, {flipped} voxels decided the other way")
        assert sure > 0.999


def test_fullsize_warp_and_sampled_projection(wl, oracle_volumes):
    V, E = oracle_volumes
    g, det = wl.grid, wl.det
    vw, coeff = _batch(wl)
    Vd, Ed = dev(V), dev(E)
    W = pmf.warp_combine(g, Vd, Ed, dev(coeff))  # the whole batch, as the benchmark launches it
    rng = np.random.default_rng(77)
    Vf, Ef = V.astype(np.float32), E.astype(np.float32)
    Y = host(pmf.conebeam_project(g, det, views(vw), W, shared=False))
    for p in (0, 17):
        Wref = oracle.warp(g, Vf, oracle.combine(Ef, coeff[p:p + 1].astype(np.float64)))[0]
        assert rel_l2(host(W[p]), Wref) <= 1e-5
        pix = [(p, int(rng.integers(0, det.nv)), int(rng.integers(0, det.nu))) for _ in range(16)]
        for (_, b, a), v1 in zip(pix, pixel_views(vw, det.nu, det.nv, pix)):
            yref = oracle.project(g, 1, 1, det.step_mm, v1[None], Wref)[0, 0, 0]
            assert Y[p, b, a] == pytest.approx(yref, rel=2e-5, abs=1e-6 * np.abs(Y).max())


def test_fullsize_backprojection_one_view(wl):
    g, det = wl.grid, wl.det
    vw, _ = _batch(wl)
    dY = np.random.default_rng(78).normal(size=(1, det.nv, det.nu)).astype(np.float32)
    got = host(pmf.conebeam_project_backward(g, det, views(vw[:1]), dev(dY), shared=False))
    ref = oracle.project_backward(g, det.nu, det.nv, det.step_mm, vw[:1], dY)
    assert rel_l2(got, ref) <= 1e-5


def _adjoint_gap(Ax, y, x, Aty):
    """|<Ax, y> - <x, A^T y>| relative to ||Ax|| ||y|| (the Cauchy-Schwarz
    scale of the inner product; random-sign y makes the sum itself small)."""
    lhs = float((Ax.double() * y.double()).sum())
    rhs = float((x.double() * Aty.double()).sum())
    return abs(lhs - rhs) / (float(Ax.double().norm()) * float(y.double().norm()))


def test_fullsize_adjoint_identities(wl, oracle_volumes):
    """<A x, y> = <x, A^T y> over the whole batch for the projector and the
    fused warp (x random, y random), at the benchmark's sizes."""
    g, det = wl.grid, wl.det
    vw, coeff = _batch(wl)
    V, E = oracle_volumes
    gen = torch.Generator("cuda").manual_seed(5)
    x = torch.rand((B,) + g.shape, device="cuda", generator=gen)
    y = torch.randn((B, det.nv, det.nu), device="cuda", generator=gen)
    vt = views(vw)
    gap = _adjoint_gap(pmf.conebeam_project(g, det, vt, x, shared=False), y, x,
                       pmf.conebeam_project_backward(g, det, vt, y, shared=False))
    assert gap <= 1e-6
    Ed, cd = dev(E), dev(coeff)
    u = torch.rand(g.shape, device="cuda", generator=gen)
    yw = torch.randn((B,) + g.shape, device="cuda", generator=gen)
    d_ref, _, _ = pmf.warp_combine_backward(g, u, Ed, cd, yw)
    assert _adjoint_gap(pmf.warp_combine(g, u, Ed, cd), yw, u, d_ref) <= 1e-6


def test_fullsize_warp_adjoint_four_views(wl, oracle_volumes):
    """The fused warp adjoint on four views of the paper-scale grid against the
    oracle's warp and combine adjoints (oracle-side V, E and a seeded dW)."""
    g = wl.grid
    V, E = oracle_volumes
    _, coeff = _batch(wl)
    w4 = coeff[:4]
    Vf, Ef = V.astype(np.float32), E.astype(np.float32)
    dW = np.random.default_rng(80).normal(size=(4,) + g.shape).astype(np.float32)
    dV, dE, dw = pmf.warp_combine_backward(g, dev(Vf), dev(Ef), dev(w4), dev(dW))
    D = oracle.combine(Ef, w4.astype(np.float64))
    dV_ref, dD_ref = oracle.warp_backward(g, Vf, D, dW)
    dE_ref, dw_ref = oracle.combine_backward(Ef, w4.astype(np.float64), dD_ref)
    assert rel_l2(host(dV), dV_ref) <= 1e-5
    assert rel_l2(host(dE), dE_ref) <= 1e-4
    # the DVF gradient jumps where a sample crosses a voxel face, and fp32 and
    # fp64 positions pick different sides for a few voxels; the coefficient
    # gradient sums those over the whole grid, so it gets the gradient bar
    assert rel_l2(host(dw), dw_ref) <= 1e-3


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_fullsize_training_step_runs_and_is_reproducible(wl, dt):
    """The benchmark's step (B = 32) twice on the same batch: bit-identical
    loss and gradients, finite everywhere."""
    vw, coeff = _batch(wl)
    meas = np.random.default_rng(79).random((B, wl.det.nv, wl.det.nu)).astype(np.float32) * 400
    step = ForwardAdjoint(wl.grid, wl.det, gset(wl.ref, wl.kappa), [gset(m, wl.kappa) for m in wl.mbc], batch=B,
                          dtype=dt)
    args = (views(vw), dev(coeff), dev(meas))
    l1 = step.run(*args).clone()
    g1 = [t.clone() for t in step.g_ref + step.g_wc]
    l2 = step.run(*args)
    assert torch.equal(l1, l2)
    for a, b in zip(g1, step.g_ref + step.g_wc):
        assert torch.equal(a, b)
        assert torch.isfinite(a).all()
