"""Seeded synthetic workloads shaped like the PMF-STGR studies.

The paper reconstructs 200x200x100 volumes at 2 mm (Sec. 2.3.3, Table I) from
cone-beam scans with SAD/SDD 1000/1500 mm, 512x384 detectors at 0.776 mm and 660
projections over 360 degrees at 11 frames/s; the reference anatomy is held by up to
100,000 Gaussians and the motion basis by three levels of Gaussians (Sec. 2.3.2).
The XCAT phantom and the patient scans are not available, so every array here is
drawn from a seeded NumPy PCG64 generator with those shapes instead.

Conventions shared by every consumer (they define the inputs, not the method):
  * volumes are [nz][ny][nx] with x fastest, centred on the isocentre;
  * a Gaussian set is mean[G,3] (mm), scale[G,3] (per-axis standard deviation,
    mm), quat[G,4] (w, x, y, z; need not be unit length) and value[G,C];
  * a view is 12 float64 numbers: source[3], detector centre[3], du[3], dv[3]
    (du/dv are one-pixel step vectors, mm); pixel (a, b) sits at
    det + (a + 1/2 - nu/2) du + (b + 1/2 - nv/2) dv;
  * temporal coefficients are [P][L][3] (projection, MBC level, Cartesian axis).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    vx: float
    vy: float
    vz: float

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def extent_mm(self):
        return (self.nx * self.vx, self.ny * self.vy, self.nz * self.vz)

    @property
    def v_iso(self) -> float:
        return float((self.vx * self.vy * self.vz) ** (1.0 / 3.0))


@dataclass(frozen=True)
class Detector:
    nu: int
    nv: int
    step_mm: float  # ray-march step; the path uses it as given

    @property
    def q(self) -> int:
        return self.nu * self.nv


@dataclass
class GaussianSet:
    mean: np.ndarray   # [G,3] float32, mm
    scale: np.ndarray  # [G,3] float32, mm (standard deviations)
    quat: np.ndarray   # [G,4] float32, (w, x, y, z)
    value: np.ndarray  # [G,C] float32

    @property
    def g(self) -> int:
        return int(self.mean.shape[0])

    @property
    def channels(self) -> int:
        return int(self.value.shape[1])


@dataclass
class Workload:
    name: str
    grid: Grid
    det: Detector
    ref: GaussianSet
    mbc: List[GaussianSet]
    views: np.ndarray          # [P,12] float64
    coeff: np.ndarray          # [P,L,3] float32
    kappa: float
    measured: Optional[np.ndarray] = None  # [P,nv,nu] float32
    meta: dict = field(default_factory=dict)
    gt: Optional[GaussianSet] = None       # ground-truth reference set (its projections are the targets)

    @property
    def p(self) -> int:
        return int(self.views.shape[0])

    @property
    def levels(self) -> int:
        return len(self.mbc)


def seeds_for(workload: str) -> dict:
    """Seed plan: workload k (0 = the small case, 1 = the paper-scale case)
    draws from 1000*(k+1) + {0: reference Gaussians, 1: MBC Gaussians,
    2: temporal coefficients, 3: smooth stand-in projections, 4: the
    ground-truth reference Gaussian set}."""
    base = 1000 * ({"small": 0, "paper": 1}[workload] + 1)
    return {"ref": base, "mbc": base + 1, "coeff": base + 2, "measured": base + 3, "gt": base + 4}


def circular_views(p: int, sad: float, sdd: float, nu: int, nv: int,
                   du_mm: float, dv_mm: float, start: float = 0.0,
                   arc: float = 2.0 * np.pi) -> np.ndarray:
    """Circular source trajectory about +z with a flat detector opposite the source.

    theta_p = start + arc * p / P; source = SAD (cos, sin, 0); detector centre =
    -(SDD - SAD) (cos, sin, 0); u axis = (-sin, cos, 0); v axis = +z.  The scan
    protocol (360 degrees, SAD 1000 mm, SDD 1500 mm) is Table I / Sec. 2.3.3.
    """
    th = start + arc * np.arange(p, dtype=np.float64) / float(p)
    c, s = np.cos(th), np.sin(th)
    views = np.zeros((p, 12), dtype=np.float64)
    views[:, 0] = sad * c
    views[:, 1] = sad * s
    views[:, 3] = -(sdd - sad) * c
    views[:, 4] = -(sdd - sad) * s
    views[:, 6] = -s * du_mm
    views[:, 7] = c * du_mm
    views[:, 11] = dv_mm
    return views


def _unit_quats(rng: np.random.Generator, g: int) -> np.ndarray:
    q = rng.standard_normal((g, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def gaussian_set(rng: np.random.Generator, grid: Grid, g: int,
                 scale_lo_vox: float, scale_hi_vox: float,
                 channels: int = 1, value_std: Optional[float] = None) -> GaussianSet:
    """Centres uniform in the volume box, per-axis scales log-uniform in
    [lo, hi] voxels (times the isotropic voxel size), random unit quaternions,
    and values U[0,1] (channels=1, densities) or N(0, value_std) (signed MBC
    vectors)."""
    ext = np.array(grid.extent_mm, dtype=np.float64)
    mean = (rng.random((g, 3)) - 0.5) * ext
    scale = np.exp(rng.uniform(np.log(scale_lo_vox), np.log(scale_hi_vox), (g, 3))) * grid.v_iso
    quat = _unit_quats(rng, g)
    if value_std is None:
        value = rng.random((g, channels))
    else:
        value = rng.normal(0.0, value_std, (g, channels))
    return GaussianSet(mean.astype(np.float32), scale.astype(np.float32), quat,
                       value.astype(np.float32))


def mbc_levels(rng: np.random.Generator, grid: Grid, counts, stds) -> List[GaussianSet]:
    """Three-level coarse-to-fine MBC Gaussians (Sec. 2.3.1-2.3.2).  Level l has
    G_l Gaussians whose 3-vector values are N(0, std_l) mm; their scales are
    exp(U(ln 0.35, ln 0.7)) times the mean spacing (N/G_l)^(1/3) voxels."""
    out = []
    for g, std in zip(counts, stds):
        spacing = (grid.n / float(g)) ** (1.0 / 3.0)
        out.append(gaussian_set(rng, grid, g, 0.35 * spacing, 0.7 * spacing,
                                channels=3, value_std=std))
    return out


def uniform_coefficients(rng: np.random.Generator, p: int, levels: int) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, (p, levels, 3)).astype(np.float32)


def breathing_coefficients(rng: np.random.Generator, p: int, levels: int,
                           fps: float = 11.0, period_s: float = 4.0) -> np.ndarray:
    """Stand-in for the motion encoder's output (Sec. 2.3.1): a breathing-like
    sinusoid sampled at the acquisition frame rate.  Each cycle c has period
    period_s * U(0.8, 1.2) and amplitude U(0.8, 1.2); w[p,l,k] = alpha_lk *
    a_c * sin(phi(t_p) + psi_lk) with alpha ~ U(0.5, 1) and psi ~ U(-0.3, 0.3)."""
    t = np.arange(p, dtype=np.float64) / fps
    total = t[-1] + period_s * 2.0 if p else 0.0
    starts, periods, amps = [0.0], [], []
    while starts[-1] <= total:
        periods.append(period_s * rng.uniform(0.8, 1.2))
        amps.append(rng.uniform(0.8, 1.2))
        starts.append(starts[-1] + periods[-1])
    starts = np.array(starts[:-1])
    periods, amps = np.array(periods), np.array(amps)
    cyc = np.searchsorted(starts, t, side="right") - 1
    phase = 2.0 * np.pi * (cyc + (t - starts[cyc]) / periods[cyc])
    alpha = rng.uniform(0.5, 1.0, (levels, 3))
    psi = rng.uniform(-0.3, 0.3, (levels, 3))
    w = alpha[None] * amps[cyc][:, None, None] * np.sin(phase[:, None, None] + psi[None])
    return w.astype(np.float32)


def measured_projections(rng: np.random.Generator, p: int, nu: int, nv: int,
                         level: float) -> np.ndarray:
    """Smooth, positive stand-ins for measured cone-beam projections: a baseline
    plus six separable 2-D bumps per view, scaled to `level` (mm x density)."""
    a = np.arange(nu, dtype=np.float64)
    b = np.arange(nv, dtype=np.float64)
    out = np.empty((p, nv, nu), dtype=np.float32)
    for i in range(p):
        img = np.full((nv, nu), 0.3)
        for _ in range(6):
            ca, cb = rng.uniform(0, nu), rng.uniform(0, nv)
            wa, wb = rng.uniform(0.05, 0.3) * nu, rng.uniform(0.05, 0.3) * nv
            amp = rng.uniform(0.2, 1.0)
            img += amp * np.outer(np.exp(-0.5 * ((b - cb) / wb) ** 2),
                                  np.exp(-0.5 * ((a - ca) / wa) ** 2))
        out[i] = (level * img / img.max()).astype(np.float32)
    return out


def select_batch(p_total: int, batch: int, step: int, seed: int = 7) -> np.ndarray:
    """Projection indices of training batch `step`: consecutive slices of one
    seeded permutation of the scan, wrapping around."""
    perm = np.random.default_rng(seed).permutation(p_total)
    idx = (step * batch + np.arange(batch)) % p_total
    return perm[idx]


def small_workload(with_measured: bool = True) -> Workload:
    """Small case: 64^3 at 4 mm, 2,000 reference Gaussians (scales 1-4 voxels),
    one MBC level of 200 Gaussians with N(0, 2 mm) vectors, 8 views over 360
    degrees, 128x128 detector at 1.6 mm, SAD/SDD 1000/1500 mm, 0.5-voxel step,
    coefficients U[-1, 1]."""
    sd = seeds_for("small")
    grid = Grid(64, 64, 64, 4.0, 4.0, 4.0)
    det = Detector(128, 128, 2.0)
    ref = gaussian_set(np.random.default_rng(sd["ref"]), grid, 2000, 1.0, 4.0)
    mbc = mbc_levels(np.random.default_rng(sd["mbc"]), grid, [200], [2.0])
    views = circular_views(8, 1000.0, 1500.0, det.nu, det.nv, 1.6, 1.6)
    coeff = uniform_coefficients(np.random.default_rng(sd["coeff"]), 8, 1)
    meas = (measured_projections(np.random.default_rng(sd["measured"]), 8, det.nu, det.nv, 200.0)
            if with_measured else None)
    return Workload("small-64^3-2k-8views", grid, det, ref, mbc, views, coeff, 3.0, meas)


def paper_workload(p: int = 660, with_measured: bool = False, measured_for=None) -> Workload:
    """Paper-scale case: 200x200x100 at 2 mm with 100,000 reference Gaussians
    (scales 0.5-3 voxels); MBC levels of 500 / 2,000 / 8,000 Gaussians with
    5 / 2 / 1 mm vectors; 660 views over 360 degrees, 512x384 detector at
    0.776 mm, SAD/SDD 1000/1500 mm, 1 mm step (0.5 voxel); breathing
    coefficients at 11 frames/s with a ~4 s period."""
    sd = seeds_for("paper")
    grid = Grid(200, 200, 100, 2.0, 2.0, 2.0)
    det = Detector(512, 384, 1.0)
    ref = gaussian_set(np.random.default_rng(sd["ref"]), grid, 100_000, 0.5, 3.0)
    mbc = mbc_levels(np.random.default_rng(sd["mbc"]), grid, [500, 2000, 8000], [5.0, 2.0, 1.0])
    views = circular_views(660, 1000.0, 1500.0, det.nu, det.nv, 0.776, 0.776)[:p]
    coeff = breathing_coefficients(np.random.default_rng(sd["coeff"]), 660, 3)[:p]
    meas = None
    if with_measured:
        rng = np.random.default_rng(sd["measured"])
        meas = measured_projections(rng, p, det.nu, det.nv, 400.0)
    # a second draw of the reference recipe: the training target is its
    # projections through the same forward model (same MBCs and coefficients)
    gt = gaussian_set(np.random.default_rng(sd["gt"]), grid, 100_000, 0.5, 3.0)
    return Workload("paper-200x200x100-100k-660views", grid, det, ref, mbc, views, coeff, 3.0, meas, gt=gt)


def paper_workload_1mm(p: int = 660) -> Workload:
    """The paper-scale scan at 1 mm voxels (Sec. 4: the 65 GB, batch-8 case):
    the same Gaussian sets, views and coefficients as paper_workload (the same
    physical object, scales 1-6 mm), voxelized on 400x400x200 at 1 mm and
    marched at 0.5 mm (0.5 voxel)."""
    wl = paper_workload(p)
    grid = Grid(400, 400, 200, 1.0, 1.0, 1.0)
    det = Detector(wl.det.nu, wl.det.nv, 0.5)
    return Workload("paper-1mm-400x400x200-100k-660views", grid, det, wl.ref, wl.mbc, wl.views, wl.coeff, wl.kappa,
                    None, gt=wl.gt)


def fd_subproblem(seed: int = 3000) -> Workload:
    """Gradient-check sub-problem: 16^3 at 4 mm, 200 reference Gaussians, three
    MBC levels of 4 / 8 / 16 Gaussians, 4 views, 32x32 detector at 3.2 mm,
    2 mm step, no cutoff (kappa = inf)."""
    grid = Grid(16, 16, 16, 4.0, 4.0, 4.0)
    det = Detector(32, 32, 2.0)
    rng = np.random.default_rng(seed)
    ref = gaussian_set(rng, grid, 200, 1.0, 3.0)
    mbc = mbc_levels(rng, grid, [4, 8, 16], [3.0, 2.0, 1.0])
    views = circular_views(4, 1000.0, 1500.0, det.nu, det.nv, 3.2, 3.2, start=0.3)
    coeff = uniform_coefficients(rng, 4, 3)
    meas = measured_projections(rng, 4, det.nu, det.nv, 40.0)
    return Workload("fd-16^3-200-4views", grid, det, ref, mbc, views, coeff, float("inf"), meas)


def uneven_volumes():
    """Uneven batch: four volumes at 2 mm (128^2x64, 160^2x80, 200^2x100,
    256^2x128) holding 30k / 50k / 100k / 150k Gaussians, three MBC levels as
    in the paper-scale case, and 17 / 40 / 64 / 96 views each (512x384)."""
    shapes = [(128, 128, 64), (160, 160, 80), (200, 200, 100), (256, 256, 128)]
    counts = [30_000, 50_000, 100_000, 150_000]
    views_per = [17, 40, 64, 96]
    out = []
    for i, (shp, g, p) in enumerate(zip(shapes, counts, views_per)):
        base = 4000 + 10 * i
        grid = Grid(shp[0], shp[1], shp[2], 2.0, 2.0, 2.0)
        det = Detector(512, 384, 1.0)
        ref = gaussian_set(np.random.default_rng(base), grid, g, 0.5, 3.0)
        mbc = mbc_levels(np.random.default_rng(base + 1), grid, [500, 2000, 8000], [5.0, 2.0, 1.0])
        views = circular_views(p, 1000.0, 1500.0, det.nu, det.nv, 0.776, 0.776)
        coeff = breathing_coefficients(np.random.default_rng(base + 2), p, 3)
        out.append(Workload(f"volume{i}-{shp[0]}x{shp[1]}x{shp[2]}", grid, det, ref, mbc,
                            views, coeff, 3.0))
    return out
