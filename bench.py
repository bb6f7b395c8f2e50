#!/usr/bin/env python3
"""Throughput of the PMF-STGR forward model + adjoint on GB300.

One step = one training batch (default 32 projections, the paper's Stage-2
batch, Sec. 2.3.2) of the paper-scale workload (200x200x100 at 2 mm, 100,000
reference Gaussians, three MBC levels of 500/2,000/8,000 Gaussians, 512x384
detector, 660 views over 360 degrees): voxelize the reference and MBC
Gaussians, combine + warp, cone-beam project, loss, and the full adjoint down
to every Gaussian parameter and temporal coefficient.  Metric: projections/s
(forward + adjoint).  Inputs are seeded synthetic stand-ins for the XCAT and
patient scans.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f32|bf16|f16]
    python bench.py --impl reference ...    # FP64 CPU oracle on host cores
    python bench.py --rasterizer --batch B  # the Stage-1 rasterizer alone (for profiling)
    python bench.py --uneven                # the uneven four-volume batch alone (for profiling)

Under torchrun every rank runs independent batches (no data-path collective);
the timed region is bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "projections/s fwd+adjoint at 1 GB300; batched BF16 vs plain FP32; % HBM roofline"
UNIT = "projections/s"
WORKLOAD = "PMF-STGR fwd+adjoint, 200x200x100 @2mm, 100k ref Gaussians, MBC 500/2000/8000, 512x384 det, 660 views"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--dtype", choices=["f32", "bf16", "f16"], default="bf16",
                    help="storage type of V and E (all arithmetic and gradients are fp32)")
    ap.add_argument("--w-dtype", choices=["f32", "same"], default="f32",
                    help="storage type of the warped volumes W: fp32, or the same as V and E")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the batched-fp32 and plain per-projection fp32 comparison runs")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--kind", type=int, default=2, help="1 = L1 loss, 2 = L2 loss")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--small", action="store_true", help="the 64^3 / 2k-Gaussian / 128^2 case (for profiling)")
    ap.add_argument("--rasterizer", action="store_true",
                    help="time only the Stage-1 rasterizer (gs_rasterize + gs_rasterize_backward) on --batch views")
    ap.add_argument("--uneven", action="store_true",
                    help="time only the uneven four-volume batch (128^2x64 .. 256^2x128, 17 / 40 / 64 / 96 views): one batched launch each way vs "
                         "one launch pair per volume")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, enabled: bool = True):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.enabled = enabled
        self.skip = 0

    def start(self):
        if not self.enabled:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts only once the sampler is writing (its start-up
        # takes a few hundred ms); the samples before it are dropped in stop()
        t_end = time.time() + 3.0
        while time.time() < t_end and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.02)
        self.skip = sum(1 for _ in open(self.path))

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for n, line in enumerate(open(self.path)):
            if n < self.skip:
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        maxmhz = max(r[1] for r in rows)
        load = [r[0] for r in rows if r[2] > 0.25 * max(x[2] for x in rows)] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": maxmhz, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- helpers

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, or None if the
    kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(kernel)
    if not d or workload not in d.get("workloads", []):
        return None
    srcs = [os.path.join(ROOT, f) for f in d.get("sources", [d.get("source", "")])]
    if not all(os.path.exists(f) for f in srcs):
        return None
    h = hashlib.sha256()
    for f in srcs:
        h.update(open(f, "rb").read())
    if h.hexdigest()[:16] != d.get("source_sha"):
        return None
    return float(d["dram_bytes_per_launch"])


def onchip_for(kernel: str):
    """The on-chip resource that binds a projector kernel, per sample, from the
    committed ncu counts (profiles/onchip.json), or None if the kernel's sources
    changed since they were taken."""
    path = os.path.join(ROOT, "profiles", "onchip.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(kernel)
    if not d:
        return None
    h = hashlib.sha256()
    for f in d["sources"]:
        fp = os.path.join(ROOT, f)
        if not os.path.exists(fp):
            return None
        h.update(open(fp, "rb").read())
    return d if h.hexdigest()[:16] == d.get("source_sha") else None


def build_workload(small: bool):
    import numpy as np
    import synth
    if small:
        wl = synth.small_workload(with_measured=True)
        return wl, wl.measured
    wl = synth.paper_workload(p=660)
    meas = synth.measured_projections(np.random.default_rng(synth.seeds_for("paper")["measured"]), wl.p, wl.det.nu,
                                      wl.det.nv, 400.0)
    return wl, meas


def algorithmic_bytes(stage: str, B: int, n: int, q: int, L: int, esz: int, wsz: int) -> float:
    """Bytes each stage must move at least once per launch (B projections);
    esz: bytes per element of V and E, wsz: of the warped volumes W."""
    if stage == "conebeam_project":
        return B * (n * wsz + q * 4 + 96)
    if stage == "conebeam_project_backward":
        return B * (q * 4 + n * 4 + 96)
    if stage == "warp_combine":
        return L * 3 * n * esz + n * esz + B * n * wsz
    if stage == "warp_combine_backward":
        return B * n * 4 + L * 3 * n * esz + n * esz + n * 4 + L * 3 * n * 4
    if stage == "projection_loss":
        return B * q * 12
    return 0.0


# Algorithmic fp32 flops per ray sample (counted from the definition, Eq. 6):
# forward: 3 position FMAs (6) + 7 linear blends of 3 flops (21) + accumulate (1);
# adjoint: 3 position FMAs (6) + the 8 trilinear weights (3 complements, 4 pair
# products, 8 products: 15) + 8 weighted adds into the volume gradient (16).
FLOPS_PER_SAMPLE = {"conebeam_project": 28.0, "conebeam_project_backward": 37.0}
KERNEL_OF = {"conebeam_project": "k_project", "conebeam_project_backward": "k_backproject",
             "warp_combine": "k_wc_fwd_tile", "warp_combine_backward": "k_wc_bwd_tile",
             "gs_voxelize": "k_render", "gs_voxelize_backward": "k_vox_bwd", "projection_loss": "k_loss"}


def sm_clock_mhz():
    """The maximum SM clock the pool measured (MEASURED_PEAKS.json), else GB300's 2070 MHz."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path)).get("sm_max_mhz", 2070.0)), "measured"
    return 2070.0, "fallback"


def fp32_peak(sms: int):
    """Non-tensor fp32 FMA peak: SMs (queried from the device) x 128 lanes x 2
    flops x the maximum SM clock."""
    mhz, how = sm_clock_mhz()
    return (round(sms * 128 * 2 * mhz * 1e6 / 1e12, 3),
            f"derived: {sms} SMs (device query) x 128 FP32 lanes x 2 x {mhz:.0f} MHz ({how} clock)")


def samples_per_view(grid, det, views):
    """Ray samples per view that fall inside the zero-padded volume (the terms
    the line-integral sum of Eq. 6 actually has), counted exactly per ray."""
    import numpy as np
    n = np.array([grid.nx, grid.ny, grid.nz], dtype=np.float64)
    v = np.array([grid.vx, grid.vy, grid.vz], dtype=np.float64)
    a = np.arange(det.nu) + 0.5 - det.nu / 2.0
    b = np.arange(det.nv) + 0.5 - det.nv / 2.0
    out = np.zeros(len(views))
    for i, vw in enumerate(np.asarray(views, dtype=np.float64)):
        src, dc, du, dv = vw[0:3], vw[3:6], vw[6:9], vw[9:12]
        d = dc + b[:, None, None] * dv + a[None, :, None] * du - src
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        us = src / v + n / 2 - 0.5
        st = det.step_mm * d / v
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (-1.0 - us) / st
            t2 = (n - us) / st
        lo = np.nanmax(np.where(st != 0, np.minimum(t1, t2), -np.inf), axis=-1)
        hi = np.nanmin(np.where(st != 0, np.maximum(t1, t2), np.inf), axis=-1)
        inside = np.all((st != 0) | ((us > -1) & (us < n)), axis=-1)
        cnt = np.ceil(hi) - np.maximum(np.floor(lo) + 1.0, 0.0)
        out[i] = np.where(inside & (cnt > 0), cnt, 0.0).sum()
    return out


# ------------------------------------------------------------ native arm

def run_native(a):
    import numpy as np
    import torch
    import torch.distributed as tdist

    import paper_2503_22139_gb300 as pmf
    from paper_2503_22139_gb300 import ops
    from paper_2503_22139_gb300.pipeline import ForwardAdjoint
    import synth

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[a.dtype]
    wdt = torch.float32 if a.w_dtype == "f32" else dt
    wl, meas_np = build_workload(a.small)
    B = min(a.batch, wl.p)
    perm = synth.select_batch(wl.p, wl.p, 0)  # one permutation of the scan; batches are its slices
    nbatch = wl.p // B

    def d(x, t=torch.float32):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=t, device="cuda")

    views_all = d(wl.views[perm], torch.float64)
    coeff_all = d(wl.coeff[perm])

    def gset(s):
        return pmf.Gaussians(d(s.mean), d(s.scale), d(s.quat), d(s.value), wl.kappa)

    ref = gset(wl.ref)
    mbc = [gset(m) for m in wl.mbc]
    if wl.gt is not None:
        # targets: the ground-truth Gaussian set through the same forward model
        # (fp32, before timing), B views at a time
        gt = gset(wl.gt)
        Vgt = pmf.gs_voxelize(wl.grid, gt)[0]
        Egt = torch.stack([pmf.gs_voxelize(wl.grid, m) for m in mbc])
        meas_all = torch.empty((wl.p, wl.det.nv, wl.det.nu), dtype=torch.float32, device="cuda")
        for s in range(0, wl.p, B):
            Wgt = pmf.warp_combine(wl.grid, Vgt, Egt, coeff_all[s:s + B])
            meas_all[s:s + B] = pmf.conebeam_project(wl.grid, wl.det, views_all[s:s + B], Wgt, shared=False)
        del gt, Vgt, Egt, Wgt
        torch.cuda.synchronize()
    else:
        meas_all = d(meas_np[perm])
    step = ForwardAdjoint(wl.grid, wl.det, ref, mbc, batch=B, dtype=dt, kind=a.kind, w_dtype=wdt)

    stage_names = ["gs_voxelize", "warp_combine", "conebeam_project", "projection_loss",
                   "conebeam_project_backward", "warp_combine_backward", "gs_voxelize_backward"]

    def batch(k):
        s = ((rank * 7919 + k) % nbatch) * B
        return views_all[s:s + B], coeff_all[s:s + B], meas_all[s:s + B]

    # warm-up
    for k in range(a.warmup):
        step.run(*batch(k))
    torch.cuda.synchronize()

    # per-stage events on the launching stream, over the timed steps
    stream = torch.cuda.current_stream()
    ev = {s: [] for s in stage_names}
    orig = {s: getattr(ops, s) for s in stage_names}

    def timed(name):
        f = orig[name]

        def w(*args, **kw):
            # on the stream the call is launched on (the step runs the Gaussian
            # sets' voxelizer calls on side streams, so those stages overlap)
            cur = torch.cuda.current_stream()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            r = f(*args, **kw)
            e1.record(cur)
            ev[name].append((e0, e1))
            return r
        return w

    clocks = ClockSampler(local, enabled=not a.no_clocks)
    clocks.start()
    for s in stage_names:
        setattr(ops, s, timed(s))
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(a.steps):
        loss = step.run(*batch(a.warmup + k))
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    for s in stage_names:
        setattr(ops, s, orig[s])
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    if world > 1:
        tt = torch.tensor([elapsed], device="cuda")
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        elapsed = float(tt.item())
    total_proj = B * a.steps * world
    value = total_proj / elapsed
    stage_ms = {s: sum(e0.elapsed_time(e1) for e0, e1 in ev[s]) / a.steps for s in stage_names if ev[s]}

    # rooflines: the projector stages are bound by arithmetic issue (every sample is
    # a trilinear gather or scatter), the streaming stages by HBM
    n, q, L = wl.grid.n, wl.det.q, wl.levels
    esz = torch.tensor([], dtype=dt).element_size()
    wsz = torch.tensor([], dtype=wdt).element_size()
    hbm_peak, hsrc = peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    f32_peak, fsrc = fp32_peak(sms)
    mhz, _ = sm_clock_mhz()
    timed_views = np.concatenate([wl.views[perm][((rank * 7919 + a.warmup + k) % nbatch) * B:
                                                 ((rank * 7919 + a.warmup + k) % nbatch) * B + B]
                                  for k in range(a.steps)])
    # per launch (B views): exact counts on up to 64 of the timed views, scaled
    sub = timed_views[np.linspace(0, len(timed_views) - 1, min(64, len(timed_views))).astype(int)]
    samples = float(samples_per_view(wl.grid, wl.det, sub).mean()) * B
    workload_tag = f"{'small' if a.small else 'paper'}-{a.dtype}{'-wf32' if wdt != dt else ''}-B{B}"
    kernel_of = dict(KERNEL_OF)
    if wdt == torch.float32:  # fp32 volumes: the box is staged with bulk tensor copies
        kernel_of["conebeam_project"] = "k_project_tma"
    stage_roof = {}
    for st, ms in stage_ms.items():
        per_launch_ms = ms / max(1, len(ev[st]) // a.steps)
        sec = per_launch_ms / 1e3
        alg_b = algorithmic_bytes(st, B, n, q, L, esz, wsz)
        ent = {"avg_launch_ms": round(per_launch_ms, 4)}
        if alg_b:
            ent.update({"hbm_achieved_gbs": round(alg_b / sec / 1e9, 2), "hbm_frac": round(alg_b / sec / 1e9 / hbm_peak, 5),
                        "algorithmic_bytes": alg_b})
        oc = onchip_for(kernel_of.get(st, KERNEL_OF.get(st, st))) if st in FLOPS_PER_SAMPLE else None
        if oc is not None:
            ach = oc["per_sample"] * samples / sec
            # the resource's rate per SM per clock x the device's SMs x the maximum clock
            pk = oc["per_sm_per_clock"] * sms * mhz * 1e6
            ent["onchip"] = {"resource": oc["resource"], "achieved_per_s": round(ach, 1),
                             "peak_per_s": pk, "frac": round(ach / pk, 4), "per_sample": oc["per_sample"]}
        if st in FLOPS_PER_SAMPLE:
            fl = samples * FLOPS_PER_SAMPLE[st]
            ent.update({"bound": "alu", "achieved": round(fl / sec / 1e12, 3), "peak": f32_peak, "unit": "TFLOP/s",
                        "frac": round(fl / sec / 1e12 / f32_peak, 5), "algorithmic_flops": fl,
                        "samples_per_launch": samples})
        elif alg_b:
            ent.update({"bound": "hbm", "achieved": ent["hbm_achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                        "frac": ent["hbm_frac"]})
        stage_roof[st] = ent
    dom = max(stage_ms, key=stage_ms.get)
    d = stage_roof[dom]
    roof = {"kernel": kernel_of.get(dom, dom), "stage": dom, "bound": d.get("bound"), "achieved": d.get("achieved"),
            "peak": d.get("peak"), "unit": d.get("unit"), "frac": d.get("frac"),
            "peak_source": (f"{fsrc}" if d.get("unit") == "TFLOP/s" else f"{hsrc} hbm_gbs"),
            "traffic": traffic_for(kernel_of.get(dom, dom), workload_tag),
            "hbm_frac": d.get("hbm_frac"), "avg_launch_ms": d["avg_launch_ms"], "onchip": d.get("onchip")}

    # end to end, through the C ABI: pinned host inputs -> device -> one
    # pmf_plan_step (the native step plan, replayed from a CUDA graph) ->
    # gradients and loss back to pinned host.  Every step copies its own inputs
    # (the Gaussian sets' parameters and the batch) in and its gradients and
    # loss out inside the timed region; as a data loader would, a copy stream
    # moves step k+1's inputs (and step k-1's results) while step k computes,
    # through two device staging sets.  The parameters live in one flat buffer
    # and the plan's outputs in another (grads_flat), so each moves as one copy.
    e2e = None
    if not a.no_e2e:
        sets_in = [ref] + mbc
        par_ts = [t for m in sets_in for t in (m.mean, m.scale, m.quat, m.value)]
        offs, tot = [], 0
        for t in par_ts:
            offs.append(tot)
            tot += (t.numel() + 63) // 64 * 64  # 256-byte boundaries
        par_flat = torch.zeros(tot, dtype=torch.float32, device="cuda")
        pv = [par_flat[o:o + t.numel()].view(t.shape) for o, t in zip(offs, par_ts)]
        for v_, t in zip(pv, par_ts):
            v_.copy_(t)
        esets = [pmf.Gaussians(*pv[4 * i:4 * i + 4], m.kappa) for i, m in enumerate(sets_in)]
        eplan = pmf.Plan(wl.grid, wl.det, esets[0], esets[1:], batch=B, dtype=dt, kind=a.kind, use_graph=True,
                         w_dtype=wdt)
        params = [par_flat]
        h_par = [par_flat.cpu().pin_memory()]
        h_views = views_all.cpu().pin_memory()
        h_coeff = coeff_all.cpu().pin_memory()
        h_meas = meas_all.cpu().pin_memory()
        outs = [eplan.grads_flat]  # every gradient and the loss
        h_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
        st_par = [[torch.empty_like(t) for t in params] for _ in range(2)]
        st_in = [(torch.empty((B, 12), dtype=torch.float64, device="cuda"), torch.empty((B, L, 3), device="cuda"),
                  torch.empty((B, wl.det.nv, wl.det.nu), device="cuda")) for _ in range(2)]
        st_out = [[torch.empty_like(t) for t in outs] for _ in range(2)]
        h2d = sum(t.numel() * t.element_size() for t in h_par) + B * (12 * 8 + L * 3 * 4 + wl.det.q * 4)
        d2h = sum(t.numel() * t.element_size() for t in h_out)
        cstream = torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_res = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def h2d_step(k):  # on the copy stream
            s0 = ((rank * 7919 + k) % nbatch) * B
            i = k % 2
            for dst, src_ in zip(st_par[i], h_par):
                dst.copy_(src_, non_blocking=True)
            for dst, src_ in zip(st_in[i], (h_views, h_coeff, h_meas)):
                dst.copy_(src_[s0:s0 + B], non_blocking=True)
            ev_in[i].record(cstream)

        def run_e2e(k0, n):
            with torch.cuda.stream(cstream):
                cstream.wait_stream(stream)
                h2d_step(k0)
            for k in range(k0, k0 + n):
                i = k % 2
                if k + 1 < k0 + n:
                    with torch.cuda.stream(cstream):
                        h2d_step(k + 1)  # after the copy stream's D2H of step k - 1: staging i ^ 1 is free
                stream.wait_event(ev_in[i])
                for dst, src_ in zip(params, st_par[i]):
                    dst.copy_(src_, non_blocking=True)
                eplan.step(*st_in[i])
                if k - 2 >= k0:
                    stream.wait_event(ev_out[i])  # step k - 2's results have left staging i
                for dst, src_ in zip(st_out[i], outs):
                    dst.copy_(src_, non_blocking=True)
                ev_res[i].record(stream)
                with torch.cuda.stream(cstream):
                    cstream.wait_event(ev_res[i])
                    for h, t in zip(h_out, st_out[i]):
                        h.copy_(t, non_blocking=True)
                    ev_out[i].record(cstream)
            stream.wait_stream(cstream)

        run_e2e(0, a.warmup)
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_e2e(a.warmup, a.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        te = e0.elapsed_time(e1) / 1e3
        if world > 1:
            tt = torch.tensor([te], device="cuda")
            tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
            te = float(tt.item())
        e2e = {"value": round(total_proj / te, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "path": "pmf_plan_step (C ABI, CUDA graph)",
               "overlap": "copy stream, double-buffered staging"}
        eplan.close()
        del eplan

    launches = step.launches_per_step * a.steps
    variants = {}
    if not a.no_variants:
        from paper_2503_22139_gb300.pipeline import GraphedStep
        gstep = GraphedStep(step, *batch(0))
        for k in range(2):
            gstep.run(*batch(k))
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for k in range(a.steps):
            gstep.run(*batch(a.warmup + k))
        g1.record(stream)
        torch.cuda.synchronize()
        tg = g0.elapsed_time(g1) / 1e3
        if world > 1:
            tt = torch.tensor([tg], device="cuda")
            tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
            tg = float(tt.item())
        variants[f"graph_replay_{a.dtype}"] = round(B * a.steps * world / tg, 3)
        del gstep
        # the native plan (C++ step, captured into a CUDA graph on its own stream)
        plan = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=B, dtype=dt, kind=a.kind, use_graph=True, w_dtype=wdt)
        for k in range(2):
            plan.step(*batch(k))
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
        g0.record(stream)
        for k in range(a.steps):
            plan.step(*batch(a.warmup + k))
        g1.record(stream)
        torch.cuda.synchronize()
        tg = g0.elapsed_time(g1) / 1e3
        if world > 1:
            tt = torch.tensor([tg], device="cuda")
            tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
            tg = float(tt.item())
        variants[f"native_plan_graph_{a.dtype}"] = round(B * a.steps * world / tg, 3)
        plan.close()
        del plan
        # the same plan with the autotuner's launch shapes for this workload
        with tempfile.TemporaryDirectory() as td:
            cache = os.path.join(td, "tune.txt")
            pmf.autotune(wl.grid, wl.det, ref, mbc, B, cache, dtype=dt, kind=a.kind, views=batch(0)[0],
                         coeff=batch(0)[1], meas=batch(0)[2], w_dtype=wdt)
            plan = pmf.Plan(wl.grid, wl.det, ref, mbc, batch=B, dtype=dt, kind=a.kind, use_graph=True,
                            tune_cache=cache, w_dtype=wdt)
        for k in range(2):
            plan.step(*batch(k))
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
        g0.record(stream)
        for k in range(a.steps):
            plan.step(*batch(a.warmup + k))
        g1.record(stream)
        torch.cuda.synchronize()
        tg = g0.elapsed_time(g1) / 1e3
        if world > 1:
            tt = torch.tensor([tg], device="cuda")
            tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
            tg = float(tt.item())
        variants[f"native_plan_graph_autotuned_{a.dtype}"] = round(B * a.steps * world / tg, 3)
        fp_shape, bp_shape = plan.launch_forms()
        variants["autotuned_shapes"] = {"proj": list(fp_shape), "backproj": list(bp_shape),
                                        "fields": ["form (0 grid, k persistent CTAs/SM)", "chunk", "rays"],
                                        "voxel_tiles": ["x".join(map(str, t)) for t in plan.voxel_tiles()]}
        plan.close()
        del plan
        from paper_2503_22139_gb300.pipeline import PlainPerProjection
        main_dt = a.dtype
        del step
        torch.cuda.empty_cache()
        kv = max(2, min(a.steps, 6))
        for name, cls, vdt in (("batched_f32", ForwardAdjoint, "f32"),
                               ("plain_per_projection_f32", PlainPerProjection, "f32")):
            if name == "batched_f32" and main_dt == "f32":
                variants[name] = round(value, 3)
                continue
            vstep = cls(wl.grid, wl.det, ref, mbc, batch=B, dtype=torch.float32, kind=a.kind)
            for k in range(2):
                vstep.run(*batch(k))
            torch.cuda.synchronize()
            if world > 1:
                tdist.barrier()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for k in range(kv):
                vstep.run(*batch(a.warmup + k))
            v1.record(stream)
            torch.cuda.synchronize()
            tv = v0.elapsed_time(v1) / 1e3
            if world > 1:
                tt = torch.tensor([tv], device="cuda")
                tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
                tv = float(tt.item())
            variants[name] = round(B * kv * world / tv, 3)
            del vstep
            torch.cuda.empty_cache()
        variants[f"batched_{main_dt}_over_plain_f32"] = round(value / variants["plain_per_projection_f32"], 3)

        def timed_steps(run, n, views=B):
            for k in range(2):
                run(k)
            torch.cuda.synchronize()
            if world > 1:
                tdist.barrier()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for k in range(n):
                run(a.warmup + k)
            v1.record(stream)
            torch.cuda.synchronize()
            tv = v0.elapsed_time(v1) / 1e3
            if world > 1:
                tt = torch.tensor([tv], device="cuda")
                tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
                tv = float(tt.item())
            return views * n * world / tv

        # the Stage 2-3 objective of Eq. 14 (L1 + 0.25 D-SSIM + L_MBC + 0.05 TV on a
        # 32^3 crop drawn per step from a seeded generator)
        drange = float((meas_all.max() - meas_all.min()).item())
        tv_rng = np.random.default_rng(4242)
        n_orig = 64
        origins = torch.tensor(np.stack([tv_rng.integers(0, [wl.grid.nx - 31, wl.grid.ny - 31, wl.grid.nz - 31])
                                         for _ in range(n_orig)]), dtype=torch.int32, device="cuda")
        estep = ForwardAdjoint(wl.grid, wl.det, ref, mbc, batch=B, dtype=dt, kind="eq14",
                               eq14=dict(data_range=drange), w_dtype=wdt)
        variants[f"eq14_objective_{a.dtype}"] = round(
            timed_steps(lambda k: estep.run(*batch(k), tv_origin=origins[k % n_orig]), a.steps), 3)
        del estep
        torch.cuda.empty_cache()
        # Stage 1 (Eq. 10-11): the reference Gaussians rasterized by Gaussian
        # splatting (Eq. 8-9), L1 + 0.25 D-SSIM, 0.05 TV of a voxelized 32^3 crop
        # drawn per step; batches of B views and of one view (the paper's Stage-1
        # batch size)
        from paper_2503_22139_gb300.pipeline import GraphedStage1, Stage1Step
        centres = [Stage1Step.crop_centre(wl.grid, o.tolist(), 32).cuda() for o in origins.cpu()]
        for vb in (B, 1):
            s1 = Stage1Step(wl.grid, wl.det, ref, batch=vb, data_range=drange)
            variants[f"stage1_rasterizer_B{vb}_views"] = round(timed_steps(
                lambda k: s1.run(batch(k)[0][:vb], batch(k)[2][:vb], centres[k % n_orig]), a.steps, views=vb), 3)
            # the same step replayed from a CUDA graph (inputs copied into its
            # static buffers each step)
            gs1 = GraphedStage1(s1, batch(0)[0][:vb], batch(0)[2][:vb], centres[0])
            variants[f"stage1_rasterizer_B{vb}_views_graph"] = round(timed_steps(
                lambda k: gs1.run(batch(k)[0][:vb], batch(k)[2][:vb], centres[k % n_orig]), a.steps, views=vb), 3)
            del s1, gs1
        torch.cuda.empty_cache()
        # the two resolution levels of Stages 2 and 3 (Sec. 2.3.2): Stage 2 on the
        # half-resolution grid (100x100x50 at 4 mm, 2 mm march step) with batches
        # of 32, Stage 3 on the full grid with batches of 8
        g2 = (wl.grid.nx // 2, wl.grid.ny // 2, wl.grid.nz // 2, 2 * wl.grid.vx, 2 * wl.grid.vy, 2 * wl.grid.vz)
        d2 = (wl.det.nu, wl.det.nv, 2 * wl.det.step_mm)
        for name, gg, dd, vb in (("stage2_halfres_B32", g2, d2, B), ("stage3_fullres_B8", wl.grid, wl.det, 8)):
            st = ForwardAdjoint(gg, dd, ref, mbc, batch=vb, dtype=dt, kind=a.kind, w_dtype=wdt)
            variants[f"{name}_{a.dtype}"] = round(timed_steps(
                lambda k: st.run(batch(k)[0][:vb], batch(k)[1][:vb], batch(k)[2][:vb]), a.steps, views=vb), 3)
            del st
        torch.cuda.empty_cache()
        # 1 mm voxels (400x400x200, the same Gaussian sets; Sec. 4's batch-8 case):
        # throughput of the batch-8 step and its peak device memory
        w1 = synth.paper_workload_1mm(p=wl.p)
        torch.cuda.reset_peak_memory_stats()
        base_mem = torch.cuda.memory_allocated()
        step1 = ForwardAdjoint(w1.grid, w1.det, ref, mbc, batch=8, dtype=dt, kind=a.kind, w_dtype=wdt)
        m1 = torch.as_tensor(synth.measured_projections(np.random.default_rng(4343), 8, w1.det.nu, w1.det.nv, 400.0),
                             dtype=torch.float32, device="cuda")
        variants[f"step_1mm_B8_{a.dtype}"] = round(timed_steps(
            lambda k: step1.run(batch(k)[0][:8], batch(k)[1][:8], m1), max(2, min(a.steps, 5)), views=8), 3)
        variants["step_1mm_B8_peak_gib"] = round((torch.cuda.max_memory_allocated() - base_mem) / 2 ** 30, 2)
        del step1, m1
        torch.cuda.empty_cache()
        # 100 optimisation iterations (B projections each, Adam on every Gaussian
        # parameter of copies of the sets); throughput and the loss trajectory
        def clone_set(gs):
            return pmf.Gaussians(gs.mean.clone(), gs.scale.clone(), gs.quat.clone(), gs.value.clone(), gs.kappa)
        tref, tmbc = clone_set(ref), [clone_set(m) for m in mbc]
        tstep = ForwardAdjoint(wl.grid, wl.det, tref, tmbc, batch=B, dtype=dt, kind=a.kind, w_dtype=wdt)
        params, lrs = [], []
        for gs in [tref] + tmbc:
            params += [gs.mean, gs.scale, gs.quat, gs.value]
            lrs += [0.02, 0.005, 0.002, 0.002 if gs.channels == 1 else 0.01]
        opt = pmf.Adam(params, lr=lrs)
        grads_of = lambda: [g for gl in [tstep.g_ref] + tstep.g_mbc for g in gl]
        traj = []

        def train(k):
            loss_k = tstep.run(*batch(k))
            opt.step(grads_of())
            if k in (a.warmup, a.warmup + 99):
                traj.append(loss_k.clone())

        variants[f"train_100_iterations_{a.dtype}"] = round(timed_steps(train, 100), 3)
        variants["train_loss_first_last"] = [round(float(t.item()), 3) for t in traj]
        del tstep, opt
        torch.cuda.empty_cache()
        if not a.small:
            # the uneven batch: four volumes of different grids (128^2x64 .. 256^2x128,
            # each its reference set voxelized in fp32) with 17 / 40 / 64 / 96 views,
            # projected and back-projected as one persistent launch each way, plain
            # and replayed from a CUDA graph, against one launch pair per volume
            items, dys = [], []
            for u in synth.uneven_volumes():
                ug = pmf.Gaussians(*(torch.as_tensor(x, device="cuda") for x in
                                     (u.ref.mean, u.ref.scale, u.ref.quat, u.ref.value)), u.kappa)
                vol = pmf.gs_voxelize(u.grid, ug)[0]
                uv = torch.as_tensor(u.views, dtype=torch.float64, device="cuda")
                items.append((u.grid, u.det, uv, vol, True))
                dys.append(torch.ones((u.p, u.det.nv, u.det.nu), device="cuda"))
            nviews = sum(it[2].shape[0] for it in items)
            ys = [torch.empty((it[2].shape[0], it[1].nv, it[1].nu), device="cuda") for it in items]
            gs_out = [torch.empty(it[0].shape, device="cuda") for it in items]

            def uneven_batched(k):
                ops.conebeam_project_batched(items, out=ys)
                ops.conebeam_project_backward_batched([(it[0], it[1], it[2], dy, True) for it, dy in zip(items, dys)],
                                                      out=gs_out)

            def uneven_per_volume(k):
                for it, dy, y, go in zip(items, dys, ys, gs_out):
                    ops.conebeam_project(it[0], it[1], it[2], it[3], shared=True, out=y)
                    ops.conebeam_project_backward(it[0], it[1], it[2], dy, shared=True, out=go)

            variants["config3_uneven_batched_f32"] = round(timed_steps(uneven_batched, 5, views=nviews), 3)
            uneven_batched(0)
            torch.cuda.synchronize()
            ug_graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(ug_graph):
                uneven_batched(0)
            variants["config3_uneven_batched_graph_f32"] = round(timed_steps(lambda k: ug_graph.replay(), 5,
                                                                             views=nviews), 3)
            variants["config3_per_volume_f32"] = round(timed_steps(uneven_per_volume, 5, views=nviews), 3)
            del items, dys, ys, gs_out, ug_graph
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(wl, meas_np, small=a.small)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(elapsed * 1e3 / a.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": ("synthetic: seeded Gaussian sets; targets are a seeded ground-truth Gaussian set's projections "
                 "through the same forward" if wl.gt is not None else "synthetic"),
        "config": {"workload": WORKLOAD if not a.small else "small: 64^3 @4mm, 2k Gaussians, 128^2 det, 8 views",
                   "batch_projections": B, "loss": "L2" if a.kind == 2 else "L1", "storage_dtype": a.dtype,
                   "warped_volume_dtype": "f32" if wdt == torch.float32 else a.dtype,
                   "accumulate_dtype": "f32", "l2_policy": "working set > L2 (E 144 MB, W and dW 512 MB each)",
                   "parallelism": f"replicas{world}", "sm_count": sms},
        "roofline": roof, "stage_ms_per_step": {k: round(v, 4) for k, v in stage_ms.items()},
        "stage_rooflines": stage_roof,
        "variants_projections_per_s": variants or None,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches,
        "loss": float(loss.item()),
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()


# ------------------------------------------------------------- CPU oracle

def oracle_sample(wl, meas_np, view_idx, kind=2):
    """One projection's forward + adjoint of the workload with the FP64 oracle,
    voxelization of all Gaussians and its adjoint included; returns seconds."""
    import numpy as np
    import oracle
    g, det = wl.grid, wl.det
    t = time.perf_counter()
    V = oracle.voxelize(g, wl.ref.mean, wl.ref.scale, wl.ref.quat, wl.ref.value, wl.kappa)[0]
    E = np.stack([oracle.voxelize(g, m.mean, m.scale, m.quat, m.value, wl.kappa) for m in wl.mbc])
    w = wl.coeff[view_idx:view_idx + 1].astype(np.float64)
    vw = wl.views[view_idx:view_idx + 1]
    D = oracle.combine(E, w)
    W = oracle.warp(g, V, D)
    Y = oracle.project(g, det.nu, det.nv, det.step_mm, vw, W, shared=False)
    _, dY = oracle.loss(kind, Y, meas_np[view_idx:view_idx + 1])
    dW = oracle.project_backward(g, det.nu, det.nv, det.step_mm, vw, dY, shared=False)
    dV, dD = oracle.warp_backward(g, V, D, dW)
    dE, dw = oracle.combine_backward(E, w, dD)
    oracle.voxelize_backward(g, wl.ref.mean, wl.ref.scale, wl.ref.quat, wl.ref.value, dV, wl.kappa)
    for l, m in enumerate(wl.mbc):
        oracle.voxelize_backward(g, m.mean, m.scale, m.quat, m.value, dE[l], wl.kappa)
    return time.perf_counter() - t


def cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo; the machine type elsewhere)."""
    import platform
    arm = {}
    try:
        for line in open("/proc/cpuinfo"):
            key, _, val = line.partition(":")
            key, val = key.strip().lower(), val.strip()
            if key in ("model name", "cpu model") and val:
                return val
            if key in ("cpu implementer", "cpu part") and val:
                arm.setdefault(key, val)
    except OSError:
        pass
    if arm:  # Arm cores report implementer and part numbers, not a name
        return f"{platform.machine()} (implementer {arm.get('cpu implementer', '?')}, part {arm.get('cpu part', '?')})"
    return platform.machine()


def cpu_baseline(wl, meas_np, small=False):
    import oracle
    secs = oracle_sample(wl, meas_np, 0)
    return {"value": round(1.0 / secs, 5), "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"1 projection fwd+adjoint incl. voxelization of all Gaussians and its adjoint "
                      f"({'small' if small else 'paper-scale'} workload), FP64 C oracle, {secs:.1f} s"}


def run_reference(a):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    wl, meas_np = build_workload(a.small)
    for k in range(a.warmup):
        oracle_sample(wl, meas_np, k % wl.p, a.kind)
    t = time.perf_counter()
    for k in range(a.steps):
        oracle_sample(wl, meas_np, (a.warmup + k) % wl.p, a.kind)
    el = time.perf_counter() - t
    value = a.steps / el
    sample = ("each step: 1 projection fwd+adjoint incl. voxelization of all Gaussians and its adjoint, "
              "FP64 C oracle (the path's plain definition), host cores")
    line = {"metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(el * 1e3 / a.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD if not a.small else "small", "batch_projections": 1},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "kind": "oracle", "cores": oracle.threads(),
                             "cpu": cpu_model(), "sample": sample},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_rasterizer(a):
    """Stage-1 rasterizer alone (for profiling): B views of the paper-scale
    reference set, forward and adjoint (dY = 1), event-timed."""
    import numpy as np
    import torch
    import paper_2503_22139_gb300 as pmf
    import synth
    torch.cuda.set_device(0)
    wl = synth.paper_workload(p=660)
    B = min(a.batch, wl.p)
    d = lambda x, t=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=t, device="cuda")
    vw = d(wl.views[synth.select_batch(wl.p, B, 0)], torch.float64)
    g = pmf.Gaussians(d(wl.ref.mean), d(wl.ref.scale), d(wl.ref.quat), d(wl.ref.value), wl.kappa)
    cap = pmf.gs_rasterize_count(wl.det, vw, g)
    ws = pmf.ops._ws(pmf.ops.gs_rasterize_workspace(wl.det, B, g.n, cap), "cuda")
    Y = pmf.gs_rasterize(wl.det, vw, g, ws=ws)
    dY = torch.ones_like(Y)
    grads = pmf.gs_rasterize_backward(wl.det, vw, g, dY, ws=ws)

    def step():
        pmf.gs_rasterize(wl.det, vw, g, ws=ws, out=Y)
        pmf.gs_rasterize_backward(wl.det, vw, g, dY, grads=grads, ws=ws)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.steps, 1)
    print(json.dumps({"metric": "rasterized views/s (Eq. 9 forward + adjoint, Stage 1)", "value": round(B / ms * 1e3, 3),
                      "unit": "views/s", "ms_per_step": round(ms, 4), "steps": a.steps, "warmup": a.warmup,
                      "config": {"workload": "paper-scale reference set, 100k Gaussians, 512x384 detector",
                                 "views": B, "pairs": cap}}))


def run_uneven(a):
    """The uneven batch alone (for profiling): four volumes of different grids
    (each its reference set voxelized in fp32) with 17 / 40 / 64 / 96 views of
    512x384, projected and back-projected (dY = 1) as one batched launch each
    way, then as one launch pair per volume; event-timed."""
    import torch
    import paper_2503_22139_gb300 as pmf
    from paper_2503_22139_gb300 import ops
    import synth
    torch.cuda.set_device(0)
    items, dys = [], []
    for u in synth.uneven_volumes():
        ug = pmf.Gaussians(*(torch.as_tensor(x, device="cuda") for x in
                             (u.ref.mean, u.ref.scale, u.ref.quat, u.ref.value)), u.kappa)
        items.append((u.grid, u.det, torch.as_tensor(u.views, dtype=torch.float64, device="cuda"),
                      pmf.gs_voxelize(u.grid, ug)[0], True))
        dys.append(torch.ones((u.p, u.det.nv, u.det.nu), device="cuda"))
    ys = [torch.empty((it[2].shape[0], it[1].nv, it[1].nu), device="cuda") for it in items]
    gs_out = [torch.empty(it[0].shape, device="cuda") for it in items]
    bitems = [(it[0], it[1], it[2], dy, True) for it, dy in zip(items, dys)]
    nviews = sum(it[2].shape[0] for it in items)

    def batched_fwd():
        ops.conebeam_project_batched(items, out=ys)

    def batched_adj():
        ops.conebeam_project_backward_batched(bitems, out=gs_out)

    def per_volume_fwd():
        for it, y in zip(items, ys):
            ops.conebeam_project(it[0], it[1], it[2], it[3], shared=True, out=y)

    def per_volume_adj():
        for it, dy, go in zip(items, dys, gs_out):
            ops.conebeam_project_backward(it[0], it[1], it[2], dy, shared=True, out=go)

    ms = {}
    for name, f in (("batched_forward", batched_fwd), ("batched_adjoint", batched_adj),
                    ("per_volume_forward", per_volume_fwd), ("per_volume_adjoint", per_volume_adj)):
        for _ in range(a.warmup):
            f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps):
            f()
        e1.record()
        torch.cuda.synchronize()
        ms[name] = round(e0.elapsed_time(e1) / a.steps, 3)
    res = {k: round(nviews / ((ms[k + "_forward"] + ms[k + "_adjoint"]) / 1e3), 3) for k in ("batched", "per_volume")}
    print(json.dumps({"metric": "projections/s fwd+adjoint, uneven four-volume batch (fp32)", "value": res["batched"],
                      "unit": "projections/s", "per_volume_launches": res["per_volume"], "ms": ms, "steps": a.steps,
                      "warmup": a.warmup, "config": {"workload": "128x128x64 / 160x160x80 / 200x200x100 / 256x256x128 "
                                                                 "@2 mm, 17/40/64/96 views of 512x384", "views": nviews}}))


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.rasterizer:
        run_rasterizer(a)
    elif a.uneven:
        run_uneven(a)
    else:
        run_native(a)


if __name__ == "__main__":
    main()
