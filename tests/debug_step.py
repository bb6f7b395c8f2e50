"""One forward + adjoint pass of the small workload, and one Stage-1
rasterizer pass, through the bounds-checked debug build of the library (test
infrastructure; run as `python -m tests.debug_step` with PMF_LIB_VARIANT=debug
by tests/test_gpu_debug_build.py, in a process of its own).

Every output and workspace the caller hands the library sits between guard
bands of a canary bit pattern; after the calls, no bounds check may have
failed (PMF_DIAG_BOUNDS), every canary must be intact, and the results must
match the FP64 oracle as in the parity tests.  Prints DEBUG-STEP-OK."""
from __future__ import annotations

import numpy as np
import torch

import paper_2503_22139_gb300 as pmf
from paper_2503_22139_gb300 import _lib, ops
from synth import small_workload
from tests import oracle_chain

GUARD_BYTES = 4096  # a multiple of 256: the guarded buffer keeps the allocation's alignment
CANARY = 0x5A


class Guarded:
    """Byte buffers with guard bands on both sides; `view(shape, dtype)` is the
    part the library sees."""

    def __init__(self):
        self.bufs = []

    def bytes(self, nbytes: int) -> torch.Tensor:
        full = torch.full((nbytes + 2 * GUARD_BYTES,), CANARY, dtype=torch.uint8, device="cuda")
        self.bufs.append((full, nbytes))
        return full[GUARD_BYTES:GUARD_BYTES + nbytes]

    def view(self, shape, dtype=torch.float32) -> torch.Tensor:
        n = int(np.prod(shape))
        esz = torch.tensor([], dtype=dtype).element_size()
        return self.bytes(n * esz).view(dtype).view(*shape)

    def intact(self) -> bool:
        torch.cuda.synchronize()
        for full, nbytes in self.bufs:
            head, tail = full[:GUARD_BYTES], full[GUARD_BYTES + nbytes:]
            if not (bool((head == CANARY).all()) and bool((tail == CANARY).all())):
                return False
        return True


def rel(a, b) -> float:
    a = a.detach().double().cpu().numpy().reshape(np.shape(b))
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def main() -> None:
    assert _lib.variant() == "debug" and b"debug" in _lib.load().pmf_version(), "not the debug build"
    torch.cuda.set_device(0)
    wl = small_workload()
    g, det, P = wl.grid, wl.det, wl.p
    G = Guarded()
    dev = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    sets = [wl.ref] + list(wl.mbc)
    gsets = [pmf.Gaussians(dev(s.mean), dev(s.scale), dev(s.quat), dev(s.value), wl.kappa) for s in sets]
    views, coeff, meas = pmf.views_tensor(wl.views, "cuda"), dev(wl.coeff), dev(wl.measured)
    shape, N, Lv, Q = g.shape, g.n, len(wl.mbc), det.nu * det.nv
    pmf.device_counters(reset=True)

    # forward: voxelize every set (every bin tile for the reference set), warp, project, loss
    vols = []
    for gs in gsets:
        cap = pmf.gs_voxelize_count(g, gs)
        out = G.view((gs.channels,) + shape)
        vols.append(pmf.gs_voxelize(g, gs, out=out, ws=G.bytes(ops.gs_voxelize_workspace(g, gs.n, cap))))
    for tile in ops.VOXEL_TILES[1:]:
        cap = pmf.gs_voxelize_tiled_count(g, gsets[0], tile)
        t = pmf.gs_voxelize(g, gsets[0], out=G.view((1,) + shape), tile=tile,
                            ws=G.bytes(ops.gs_voxelize_workspace(g, gsets[0].n, cap, tile)))
        assert torch.equal(t, vols[0]), tile
    V, E = vols[0][0], torch.stack([v for v in vols[1:]])
    W = pmf.warp_combine(g, V, E, coeff, out=G.view((P,) + shape))
    Y = pmf.conebeam_project(g, det, views, W, shared=False, out=G.view((P, det.nv, det.nu)))
    loss, dY = G.view((1,)), G.view((P, det.nv, det.nu))
    wsl = G.bytes(ops.pmf_workspace_size("loss", g, count=P * Q))
    ops.check(_lib.load().projection_loss(2, P, Q, ops._p(Y), ops._p(meas), ops._p(loss), ops._p(dY), ops._p(wsl),
                                          wsl.numel(), ops._stream()), "projection_loss")
    # adjoint: back-project, warp + combine adjoint, voxelizer adjoints
    dW = pmf.conebeam_project_backward(g, det, views, dY, shared=False, out=G.view((P,) + shape),
                                       ws=G.bytes(ops.pmf_workspace_size("project_backward", g, vol_stride=N, P=P)))
    wc = (G.view(shape), G.view((Lv, 3) + shape), G.view((P, Lv, 3)))
    dV, dE, dco = pmf.warp_combine_backward(g, V, E, coeff, dW, grads=wc,
                                            ws=G.bytes(ops.pmf_workspace_size("warp_combine_backward", g, L=Lv, P=P)))
    grads = []
    for i, gs in enumerate(gsets):
        d_out = dV[None] if i == 0 else dE[i - 1]
        gr = (G.view((gs.n, 3)), G.view((gs.n, 3)), G.view((gs.n, 4)), G.view((gs.n, gs.channels)))
        grads.append(pmf.gs_voxelize_backward(g, gs, d_out, grads=gr,
                                              ws=G.bytes(ops.gs_voxelize_backward_workspace(g, gs.n, gs.channels))))
    # Stage-1 rasterizer (Eq. 8-9) on the reference set, forward and adjoint
    rcap = pmf.gs_rasterize_count(det, views, gsets[0])
    R = pmf.gs_rasterize(det, views, gsets[0], out=G.view((P, det.nv, det.nu)),
                         ws=G.bytes(ops.gs_rasterize_workspace(det, P, gsets[0].n, rcap)))
    rg = (G.view((gsets[0].n, 3)), G.view((gsets[0].n, 3)), G.view((gsets[0].n, 4)), G.view((gsets[0].n, 1)))
    pmf.gs_rasterize_backward(det, views, gsets[0], dY, grads=rg,
                              ws=G.bytes(ops.gs_rasterize_workspace(det, P, gsets[0].n, 0)))
    torch.cuda.synchronize()

    counters = pmf.device_counters()
    assert counters["bounds"] == 0, counters
    pmf.device_status()
    assert G.intact(), "a guard band around a caller buffer was overwritten"
    lref, gref, fref = oracle_chain.step(wl, wl.measured, kind=2)
    errs = {"Y": rel(Y, fref["Y"]), "loss": abs(float(loss.item()) - lref) / abs(lref),
            "coeff": rel(dco, gref["coeff"]), "ref_mean": rel(grads[0][0], gref["ref"][0]),
            "mbc_value": rel(grads[1][3], gref["mbc"][0][3])}
    assert errs["Y"] <= 1e-5 and errs["loss"] <= 1e-5, errs
    assert max(errs["coeff"], errs["ref_mean"], errs["mbc_value"]) <= 1e-3, errs
    assert bool(torch.isfinite(R).all()) and float(R.abs().max()) > 0
    print("counters", counters, "errors", {k: f"{v:.2e}" for k, v in errs.items()})
    print("DEBUG-STEP-OK")


if __name__ == "__main__":
    main()
