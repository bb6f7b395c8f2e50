// Shared machinery of the cone-beam ray marcher (Eq. 6, source-anchored
// samples src + m step r, m >= 0) and its adjoint, for sm_103a: ray set-up,
// chunk anchors, the lock-step chunk boxes, the batched work list and the
// host-side checks and launch-shape dispatch.  Included by project.cu (the
// forward) and backproject.cu (the adjoint); everything here is internal.
//
// Precision: the source sits ~1 m from the volume, so a ray's direction and
// start are set up in double precision and then carried as float-float (hi + lo)
// pairs in voxel-index space.  Each chunk of samples starts from an anchor
// whose integer part is exact and whose fraction is float, so every sample
// position is good to ~1e-6 voxel while the inner loops are plain fp32.
//
// Work split: one ray per thread; a CTA covers a 16 x (rays/16) pixel tile.
// The tile's rays all leave the same source, so sample m of every ray lies at
// the same distance m*step from it: the CTA marches its rays in lock-step
// chunks, and the voxels one chunk touches form a small box (about 16x16x7 at
// the paper's geometry for 32-sample chunks).
#pragma once

#include <climits>

#include "pmf_common.cuh"

namespace pmf {
namespace {


// Launch shapes (MarchShape): CH samples per chunk (the staged brick's length
// along the rays) and RPB rays per CTA (a 16 x RPB/16 pixel tile, one ray per
// thread).  The C entry points use 32 and 256 for the projector, 48 and 128
// for the adjoint; plans may pick others.
constexpr unsigned kFull = 0xffffffffu;

struct Ray {
    float uh[3], ul[3];  // index-space position of sample m = 0 (the source), float-float
    float dh[3], dl[3];  // index-space step, float-float
    int mlo, mhi;        // samples that can touch the zero-padded volume (mhi < mlo: none)
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Per-view constants of the ray set-up as float-float (hi + lo) pairs.  Three
// threads of the CTA form them in double precision (one axis each); every ray
// of the tile then sets itself up in fp32 arithmetic, which keeps the fp64
// pipe (a small fraction of the fp32 rate on this part) out of the per-ray path.
struct ViewFF {
    float d0h[3], d0l[3];  // det - src, mm
    float duh[3], dul[3];  // detector u pixel vector, mm
    float dvh[3], dvl[3];  // detector v pixel vector, mm
    float ush[3], usl[3];  // the source in voxel-index space (voxel centres at integers)
    float kh[3], kl[3];    // step / voxel size along each axis
};

__device__ __forceinline__ void split_ff(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

// Threads 0..2 fill vf for view vw; the caller synchronises before use.
__device__ __forceinline__ void view_setup(ViewFF& vf, const pmf_view& vw, const GridD& g, double step) {
    const int t = threadIdx.x;
    if (t >= 3) return;
    const int n = t == 0 ? g.nx : (t == 1 ? g.ny : g.nz);
    const double iv = 1.0 / (double)(t == 0 ? g.vx : (t == 1 ? g.vy : g.vz));
    split_ff(vw.det[t] - vw.src[t], vf.d0h[t], vf.d0l[t]);
    split_ff(vw.du[t], vf.duh[t], vf.dul[t]);
    split_ff(vw.dv[t], vf.dvh[t], vf.dvl[t]);
    split_ff(fma(vw.src[t], iv, 0.5 * (double)n - 0.5), vf.ush[t], vf.usl[t]);
    split_ff(step * iv, vf.kh[t], vf.kl[t]);
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

// Ray through the centre of pixel (a, b): direction d = (det - src) + ca du + cb dv
// with ca, cb the pixel's offsets from the detector centre (exact in fp32),
// normalised, scaled to the index-space step, all in float-float arithmetic
// (about 44 bits, against the 48 of the double-precision definition).
__device__ __forceinline__ Ray ray_init(const ViewFF& vf, int nu, int nv, int a, int b, const GridD& g) {
    Ray r;
    const float ca = (float)a + (0.5f - 0.5f * (float)nu), cb = (float)b + (0.5f - 0.5f * (float)nv);
    float dh[3], dl[3];
    float Lh = 0.0f, Le = 0.0f;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        float p1, e1, p2, e2, s1, t1, s2, t2;
        two_prod(ca, vf.duh[t], p1, e1);
        e1 = fmaf(ca, vf.dul[t], e1);
        two_prod(cb, vf.dvh[t], p2, e2);
        e2 = fmaf(cb, vf.dvl[t], e2);
        two_sum(vf.d0h[t], p1, s1, t1);
        two_sum(s1, p2, s2, t2);
        fast_two_sum(s2, ((vf.d0l[t] + e1) + e2) + (t1 + t2), dh[t], dl[t]);
        float q, qe, ls, le;
        two_prod(dh[t], dh[t], q, qe);
        two_sum(Lh, q, ls, le);
        Lh = ls;
        Le += (qe + le) + 2.0f * dh[t] * dl[t];
    }
    float Ll;
    fast_two_sum(Lh, Le, Lh, Ll);
    // 1/sqrt(L): fp32 seed, one Newton step with the residual in float-float
    const float y0 = rsqrtf(Lh);
    float q, qe, m, me;
    two_prod(y0, y0, q, qe);
    two_prod(Lh, q, m, me);
    me = fmaf(Lh, qe, fmaf(Ll, q, me));
    const float yl = 0.5f * y0 * ((1.0f - m) - me);
    const int n[3] = {g.nx, g.ny, g.nz};
    float tlo = 0.0f, thi = 3.0e38f;
    bool miss = false;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        // unit direction, then times step / voxel
        float uh, ul, p, e;
        two_prod(dh[t], y0, p, e);
        e = fmaf(dh[t], yl, fmaf(dl[t], y0, e));
        fast_two_sum(p, e, uh, ul);
        two_prod(vf.kh[t], uh, p, e);
        e = fmaf(vf.kh[t], ul, fmaf(vf.kl[t], uh, e));
        fast_two_sum(p, e, r.dh[t], r.dl[t]);
        r.uh[t] = vf.ush[t];
        r.ul[t] = vf.usl[t];
        const float usf = r.uh[t], duf = r.dh[t];
        // the padded volume is u in (-1, n) on every axis
        if (duf != 0.0f) {
            const float inv = 1.0f / duf;
            const float t1 = (-1.0f - usf) * inv, t2 = ((float)n[t] - usf) * inv;
            tlo = fmaxf(tlo, fminf(t1, t2));
            thi = fminf(thi, fmaxf(t1, t2));
        } else if (!(usf > -1.0f && usf < (float)n[t])) {
            miss = true;
        }
    }
    // one sample of slack each side: samples outside the padded box read zeros
    const float mlo = fmaxf(floorf(tlo) - 1.0f, 0.0f), mhi = ceilf(thi) + 1.0f;
    if (miss || !(mhi >= mlo) || !(mhi < 1.0e8f)) {
        r.mlo = 1;
        r.mhi = 0;
    } else {
        r.mlo = (int)mlo;
        r.mhi = (int)mhi;
    }
    return r;
}

// Integer part and fraction of the position of sample m0 (float-float).
__device__ __forceinline__ void anchor(const Ray& r, int m0, int ib[3], float fb[3]) {
    const float m = (float)m0;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const float p = m * r.dh[t];
        const float pe = fmaf(m, r.dh[t], -p);
        float s, e;
        two_sum(r.uh[t], p, s, e);
        const float lo = ((r.ul[t] + pe) + m * r.dl[t]) + e;
        const float fl = floorf(s);
        ib[t] = (int)fl;
        fb[t] = (s - fl) + lo;
    }
}

// Sample j of a chunk, relative to the anchor.
__device__ __forceinline__ float at(const Ray& r, int t, float jf, const float fb[3]) {
    return fmaf(jf, r.dh[t], fmaf(jf, r.dl[t], fb[t]));
}

template <int RPB>
__device__ __forceinline__ void pixel_of(int tile, int ntu, int& a, int& b) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int tu = tile % ntu, tv = tile / ntu;
    a = tu * 16 + (w & 1) * 8 + (l & 7);
    b = tv * (RPB / 16) + (w >> 1) * 4 + (l >> 3);
}

template <typename T>
__device__ __forceinline__ float gather8(const T* vol, const GridD& g, int ix, int iy, int iz, float fx, float fy,
                                         float fz) {
    if ((unsigned)ix < (unsigned)(g.nx - 1) && (unsigned)iy < (unsigned)(g.ny - 1) &&
        (unsigned)iz < (unsigned)(g.nz - 1)) {
        const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
        const T* p = vol + iz * sz + iy * sy + ix;
        const float c000 = Store<T>::ld(p, 0), c100 = Store<T>::ld(p, 1);
        const float c010 = Store<T>::ld(p, sy), c110 = Store<T>::ld(p, sy + 1);
        const float c001 = Store<T>::ld(p, sz), c101 = Store<T>::ld(p, sz + 1);
        const float c011 = Store<T>::ld(p, sz + sy), c111 = Store<T>::ld(p, sz + sy + 1);
        const float a00 = fmaf(fx, c100 - c000, c000), a10 = fmaf(fx, c110 - c010, c010);
        const float a01 = fmaf(fx, c101 - c001, c001), a11 = fmaf(fx, c111 - c011, c011);
        const float b0 = fmaf(fy, a10 - a00, a00), b1 = fmaf(fy, a11 - a01, a01);
        return fmaf(fz, b1 - b0, b0);
    }
    return trilin_cell(vol, g, ix, iy, iz, fx, fy, fz);
}

// Shared block state for the lock-step march.
struct BoxState {
    int range[2];   // min mlo, max mhi over the CTA's rays
    int box[2][6];  // double-buffered cell bounds of the current chunk: lo xyz, hi xyz
    ViewFF vf;      // the tile's view, for ray_init
};

// Every thread of the CTA: the per-view constants of view vw into bs.vf.
__device__ __forceinline__ void tile_view(BoxState& bs, const pmf_view& vw, const GridD& g, float step) {
    view_setup(bs.vf, vw, g, (double)step);
    __syncthreads();
}

__device__ __forceinline__ void reset_box(int* b) {
    b[0] = b[1] = b[2] = INT_MAX;
    b[3] = b[4] = b[5] = INT_MIN;
}

// CTA-wide [min mlo, max mhi] over rays with samples.
__device__ __forceinline__ void block_range(BoxState& bs, const Ray& r, bool act) {
    if (threadIdx.x == 0) {
        bs.range[0] = INT_MAX;
        bs.range[1] = INT_MIN;
        reset_box(bs.box[0]);
        reset_box(bs.box[1]);
    }
    __syncthreads();
    int lo = act ? r.mlo : INT_MAX, hi = act ? r.mhi : INT_MIN;
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    if ((threadIdx.x & 31) == 0 && lo != INT_MAX) {
        atomicMin(&bs.range[0], lo);
        atomicMax(&bs.range[1], hi);
    }
    __syncthreads();
}

// This thread's sample range in the chunk of CH samples starting at M0, its
// anchor, and its contribution to the chunk's cell box (reduced per warp).
template <int CH>
__device__ __forceinline__ bool chunk_begin(BoxState& bs, int sel, const Ray& r, bool live, int M0, int& j0,
                                            int& j1, int ib[3], float fb[3]) {
    j0 = max(r.mlo, M0) - M0;
    j1 = min(r.mhi, M0 + CH - 1) - M0;
    const bool act = live && j0 <= j1;
    int clo[3] = {INT_MAX, INT_MAX, INT_MAX}, chi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (act) {
        anchor(r, M0, ib, fb);
        // the same expression as the staged inner loops (fmaf(j, dh, fb)):
        // it is monotonic in j, so every sample's cell lies between these two
#pragma unroll
        for (int t = 0; t < 3; t++) {
            const int f0 = ib[t] + (int)floorf(fmaf((float)j0, r.dh[t], fb[t]));
            const int f1 = ib[t] + (int)floorf(fmaf((float)j1, r.dh[t], fb[t]));
            clo[t] = min(f0, f1);
            chi[t] = max(f0, f1);
        }
    }
#pragma unroll
    for (int t = 0; t < 3; t++) {
        clo[t] = __reduce_min_sync(kFull, clo[t]);
        chi[t] = __reduce_max_sync(kFull, chi[t]);
    }
    if ((threadIdx.x & 31) == 0 && clo[0] != INT_MAX) {
#pragma unroll
        for (int t = 0; t < 3; t++) {
            atomicMin(&bs.box[sel][t], clo[t]);
            atomicMax(&bs.box[sel][3 + t], chi[t]);
        }
    }
    if (threadIdx.x == 0) reset_box(bs.box[sel ^ 1]);
    return act;
}

// Box geometry after the reduction: corners of cells [lo, hi] are [lo, hi + 1].
struct Box {
    int lx, ly, lz, bx, by, bz;
    long long vol;
};

__device__ __forceinline__ Box read_box(const BoxState& bs, int sel) {
    Box b;
    b.lx = bs.box[sel][0]; b.ly = bs.box[sel][1]; b.lz = bs.box[sel][2];
    if (b.lx == INT_MAX) {
        b.bx = b.by = b.bz = 0;
        b.vol = 0;
        return b;
    }
    b.bx = bs.box[sel][3] - b.lx + 2;
    b.by = bs.box[sel][4] - b.ly + 2;
    b.bz = bs.box[sel][5] - b.lz + 2;
    b.vol = (long long)b.bx * b.by * b.bz;
    return b;
}

// ------------------------------------------------- batched (uneven) launches
//
// Several volumes -- different grids, detectors and view counts -- in one
// launch: work item w is tile (w - begin_i) % ntiles_i of view
// (w - begin_i) / ntiles_i of item i.  By default each CTA runs one work item
// (kernels without a work-list loop, which compile to the single-volume
// kernels' code: the loop forms ran 0.5-1% slower per tile); a persistent
// launch of fewer CTAs walks the work items round-robin.  A tile's arithmetic
// is the single-volume kernel's, so the results equal per-volume launches bit
// for bit.

constexpr int kMaxItems = 16;

struct ProjItem {
    GridD g;
    int nu, nv, ntu, ntiles, P;
    float step, bound_mult, spv;
    const pmf_view* views;
    const void* vol;
    int64_t vol_stride;
    float* proj;
    const float* dproj;
    unsigned long long* acc;
    unsigned* maxbits;
    float* dvol;
    int64_t cells, nq, begin;
};

struct ProjBatch {
    int n;
    int64_t total;
    ProjItem it[kMaxItems];
};

__device__ __forceinline__ int find_item(const ProjBatch& B, int64_t w) {
    int i = 0;
    while (i + 1 < B.n && w >= B.it[i + 1].begin) i++;
    return i;
}

pmf_status check_proj(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(det != nullptr, "detector is null");
    PMF_REQUIRE(det->nu > 0 && det->nv > 0, "detector size must be positive");
    PMF_REQUIRE(det->step_mm > 0.0f && isfinite(det->step_mm), "step_mm must be positive");
    PMF_REQUIRE(P >= 0 && P < 65536, "P must be in [0, 65535]");
    PMF_REQUIRE(P == 0 || views != nullptr, "views is null");
    const int64_t n = (int64_t)grid->nx * grid->ny * grid->nz;
    PMF_REQUIRE(n < ((int64_t)1 << 31), "volume too large for the projector (N < 2^31)");
    return PMF_OK;
}

// Bound on the trilinear weight one ray's samples within one chunk can give a
// single voxel: along the axis where the ray moves fastest in index space the
// samples are at least h = step / (sqrt(3) v_max) apart, and a unit hat
// function sampled at spacing h sums to at most 1/h + 1; each sample adds at
// most 1 and a chunk holds `chunk` samples.
float chunk_samples_per_voxel(const pmf_grid* grid, float step, int chunk) {
    const double vmax = fmax(fmax((double)grid->vx, (double)grid->vy), (double)grid->vz);
    const double s = sqrt(3.0) * vmax / (double)step + 1.0;
    return (float)fmin(s, (double)chunk);
}

int max_samples_per_voxel(const pmf_grid* grid, float step) {
    // a ray crosses the open 2x2x2-voxel support of one voxel over at most its
    // diagonal, 2 |v|, so it takes at most floor(2|v| / step) + 1 samples there
    const double diag = 2.0 * sqrt((double)grid->vx * grid->vx + (double)grid->vy * grid->vy + (double)grid->vz * grid->vz);
    return (int)floor(diag / (double)step) + 1;
}

bool valid_shape(const MarchShape& sh, bool adjoint = false) { return valid_march_shape(sh, adjoint); }

// (chunk, rays) -> template instantiation
#define PMF_DISPATCH_MARCH(sh, CH, RPB, ...)                                                                  \
    switch ((sh).chunk * 1000 + (sh).rays) {                                                                \
        case 32256: { constexpr int CH = 32, RPB = 256; __VA_ARGS__; break; }                               \
        case 32128: { constexpr int CH = 32, RPB = 128; __VA_ARGS__; break; }                               \
        case 16256: { constexpr int CH = 16, RPB = 256; __VA_ARGS__; break; }                               \
        case 16128: { constexpr int CH = 16, RPB = 128; __VA_ARGS__; break; }                               \
        default: return set_error(PMF_EINVAL, "unsupported march shape: chunk %d, rays %d", (sh).chunk, (sh).rays); \
    }

int tiles_v(int nv, int rays) { return (nv + rays / 16 - 1) / (rays / 16); }

int num_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 152;
    return sms > 0 ? sms : 152;
}

// CTAs of a batched launch over the concatenated work list.  ctas = 0: one CTA
// per work item, so the hardware schedules the uneven tiles as it does for
// per-volume launches (a static share per persistent CTA finishes unevenly:
// the four-volume batch ran 12-16% slower persistent).  ctas > 0 (plans'
// persistent forms): that many CTAs, lowered to the largest prime that divides
// no item's tile count; CTA c walks work items c, c + G, c + 2G, ..., and a G
// sharing a factor with the tiles per view (608 and 768 share 32 at the paper
// detector) would keep every CTA on the same few detector columns.
unsigned persistent_ctas(int64_t total, unsigned ctas, int rays, const int* ntiles, int n) {
    (void)rays;
    if (total <= 0) return 1;
    if (ctas == 0 || total <= (int64_t)ctas) return (unsigned)(total < 0x7fffffffLL ? total : 0x7fffffffLL);
    auto ok = [&](int64_t g) {
        for (int64_t d = 2; d * d <= g; d++)
            if (g % d == 0) return false;
        for (int i = 0; i < n; i++)
            if (ntiles[i] % g == 0) return false;
        return true;
    };
    for (int64_t g = ctas; g >= 2; g--)
        if (ok(g)) return (unsigned)g;
    return ctas;
}

// Order of a batch's items in the work list: longest rays first (the volume's
// diagonal over the step bounds the samples per ray), so the tiles that take
// longest start first and the launch does not end on a tail of them.  Stable;
// results do not depend on the order.
template <typename Item>
void longest_first(int n, const Item* items, int* ord) {
    double len[kMaxItems];
    for (int i = 0; i < n; i++) {
        const pmf_grid& g = items[i].grid;
        const double ex = (double)g.nx * g.vx, ey = (double)g.ny * g.vy, ez = (double)g.nz * g.vz;
        len[i] = sqrt(ex * ex + ey * ey + ez * ez) / (double)items[i].det.step_mm;
        ord[i] = i;
    }
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && len[ord[j]] > len[ord[j - 1]]; j--) {
            const int t = ord[j];
            ord[j] = ord[j - 1];
            ord[j - 1] = t;
        }
}

pmf_status fill_item(const pmf_project_item& in, int64_t begin, int rays, ProjItem& it) {
    pmf_status st = check_proj(&in.grid, &in.det, in.P, in.views);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(in.vol_stride >= 0, "vol_stride must be >= 0");
    it = ProjItem{};
    it.g = make_grid(&in.grid);
    it.nu = in.det.nu; it.nv = in.det.nv;
    it.ntu = (in.det.nu + 15) / 16;
    it.ntiles = it.ntu * tiles_v(in.det.nv, rays);
    PMF_REQUIRE((int64_t)it.ntiles * in.P < ((int64_t)1 << 31), "an item's views x pixel tiles must be below 2^31");
    it.P = in.P;
    it.step = in.det.step_mm;
    it.views = in.views;
    it.vol_stride = in.vol_stride;
    it.nq = (int64_t)in.det.nu * in.det.nv * in.P;
    it.begin = begin;
    return PMF_OK;
}

}  // namespace
}  // namespace pmf
