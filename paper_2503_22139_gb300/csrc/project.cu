// Cone-beam ray marcher (Eq. 6, source-anchored samples src + m step r, m >= 0),
// its exact adjoint, and the L1/L2 projection loss (Eq. 10/12, Eq. 1) for
// sm_103a.
//
// Precision: the source sits ~1 m from the volume, so a ray's direction and
// start are set up in double precision and then carried as float-float (hi + lo)
// pairs in voxel-index space.  Each chunk of 32 samples starts from an anchor
// whose integer part is exact and whose fraction is float, so every sample
// position is good to ~1e-6 voxel while the inner loop is plain fp32.
//
// Work split: one ray per thread; a 256-thread CTA covers a 16x16 pixel tile
// (each warp an 8x4 patch).  The tile's rays all leave the same source, so
// sample m of every ray lies at the same distance m*step from it: the CTA
// marches its rays in lock-step chunks of 32 samples, and the voxels one chunk
// touches form a small box (about 16x16x7 at the paper's geometry).
//  - Forward: the box is staged in shared memory with coalesced loads (zero
//    outside the grid), and the 8-corner trilinear gathers read shared memory.
//  - Adjoint: every sample adds its 8 trilinear corner weights into a
//    shared-memory box in 32-bit fixed point (per-CTA scale); a warp's lanes
//    take pixels 8 apart and start their chunk at staggered samples, so its
//    simultaneous atomics land on different voxels.  The box is then flushed
//    with one 64-bit fixed-point atomic per touched voxel (global scale 2^k
//    from a provable bound).  Integer sums are order independent, so the
//    result is bit-reproducible.
// A chunk whose box does not fit in shared memory falls back to direct
// (bounds-checked) global gathers or atomics.
#include <climits>

#include "pmf_common.cuh"

namespace pmf {
namespace {

// Launch shapes (MarchShape): CH samples per chunk (the staged brick's length
// along the rays) and RPB rays per CTA (a 16 x RPB/16 pixel tile, one ray per
// thread).  The C entry points use 32 and 256; plans may pick others.
constexpr int kBox = 6144;    // shared-memory box capacity (words)
constexpr int kPitch = 33;    // box row pitch: x = lane (box width <= 32), odd against bank conflicts
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

// Ray through the centre of pixel (a, b) of view `vw`.
__device__ __forceinline__ Ray ray_init(const pmf_view& vw, int nu, int nv, int a, int b, const GridD& g,
                                        double step) {
    Ray r;
    const double ca = (double)a + 0.5 - 0.5 * (double)nu, cb = (double)b + 0.5 - 0.5 * (double)nv;
    double d[3];
    double len2 = 0.0;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        d[t] = fma(cb, vw.dv[t], fma(ca, vw.du[t], vw.det[t] - vw.src[t]));
        len2 = fma(d[t], d[t], len2);
    }
    // 1/sqrt(len2): fp32 seed, two Newton steps in double
    double y = (double)rsqrtf((float)len2);
    y = y * (1.5 - 0.5 * len2 * y * y);
    y = y * (1.5 - 0.5 * len2 * y * y);
    const int n[3] = {g.nx, g.ny, g.nz};
    const double iv[3] = {1.0 / (double)g.vx, 1.0 / (double)g.vy, 1.0 / (double)g.vz};
    float tlo = 0.0f, thi = 3.0e38f;
    bool miss = false;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const double us = fma(vw.src[t], iv[t], 0.5 * (double)n[t] - 0.5);
        const double du = step * (d[t] * y) * iv[t];
        r.uh[t] = (float)us;
        r.ul[t] = (float)(us - (double)r.uh[t]);
        r.dh[t] = (float)du;
        r.dl[t] = (float)(du - (double)r.dh[t]);
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
};

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
    bool fits;  // width <= 32 and by * bz rows of kPitch words fit in kBox
};

__device__ __forceinline__ Box read_box(const BoxState& bs, int sel) {
    Box b;
    b.lx = bs.box[sel][0]; b.ly = bs.box[sel][1]; b.lz = bs.box[sel][2];
    if (b.lx == INT_MAX) {
        b.bx = b.by = b.bz = 0;
        b.vol = 0;
        b.fits = false;
        return b;
    }
    b.bx = bs.box[sel][3] - b.lx + 2;
    b.by = bs.box[sel][4] - b.ly + 2;
    b.bz = bs.box[sel][5] - b.lz + 2;
    b.vol = (long long)b.bx * b.by * b.bz;
    b.fits = b.bx <= 32 && (long long)b.by * b.bz * kPitch <= kBox;
    return b;
}

// ----------------------------------------------------------------- forward

// One 16x16 pixel tile of view p: every thread of the CTA calls it.
template <typename T, int CH, int RPB>
__device__ __forceinline__ void project_tile(const GridD& g, int nu, int nv, int ntu, float step,
                                             const pmf_view* __restrict__ views, const T* __restrict__ vol,
                                             int64_t vol_stride, float* __restrict__ proj, int p, int tile,
                                             float* box, BoxState& bs) {
    int a, b;
    pixel_of<RPB>(tile, ntu, a, b);
    const bool in = a < nu && b < nv;
    Ray r;
    if (in) {
        r = ray_init(views[p], nu, nv, a, b, g, (double)step);
    } else {
        r.mlo = 1; r.mhi = 0;
    }
    const bool live = in && r.mlo <= r.mhi;
    const T* V = vol + (int64_t)p * vol_stride;
    block_range(bs, r, live);
    const int Mlo = bs.range[0], Mhi = bs.range[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float acc = 0.0f;
    int sel = 0;
    for (int M0 = Mlo; M0 <= Mhi; M0 += CH, sel ^= 1) {
        int j0, j1, ib[3];
        float fb[3];
        const bool act = chunk_begin<CH>(bs, sel, r, live, M0, j0, j1, ib, fb);
        __syncthreads();
        const Box bx = read_box(bs, sel);
        if (threadIdx.x == 0 && bx.vol > 0 && !bx.fits) diag_count(PMF_DIAG_PROJECT_BOX_FALLBACK);
        if (bx.vol > 0 && bx.fits) {
            // stage the box: lane = x, one warp per (y, z) row, zero outside the grid
            {
                const int x = bx.lx + lane;
                const bool xin = lane < bx.bx && (unsigned)x < (unsigned)g.nx;
                for (int zz = 0; zz < bx.bz; zz++) {
                    const int z = bx.lz + zz;
                    const bool zin = (unsigned)z < (unsigned)g.nz;
                    for (int yy = warp; yy < bx.by; yy += RPB / 32) {
                        const int y = bx.ly + yy;
                        float val = 0.0f;
                        if (xin && zin && (unsigned)y < (unsigned)g.ny)
                            val = Store<T>::ld(V, ((int64_t)z * g.ny + y) * g.nx + x);
                        box[(zz * bx.by + yy) * kPitch + lane] = val;
                    }
                }
            }
            __syncthreads();
            if (act) {
                // positions relative to the anchor cell; the box was bounded
                // with the same expression, so every cell is inside it
                const float syf = (float)kPitch, szf = (float)(kPitch * bx.by);
                const int sy = kPitch, sz = kPitch * bx.by;
                const float* qa = box + (ib[0] - bx.lx) + (ib[1] - bx.ly) * sy + (ib[2] - bx.lz) * sz;
                float jf = (float)j0;
                for (int j = j0; j <= j1; j++, jf += 1.0f) {
                    const float ux = fmaf(jf, r.dh[0], fb[0]), uy = fmaf(jf, r.dh[1], fb[1]),
                                uz = fmaf(jf, r.dh[2], fb[2]);
                    const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
                    const float fx = ux - flx, fy = uy - fly, fz = uz - flz;
                    const float* q = qa + (int)fmaf(flz, szf, fmaf(fly, syf, flx));
                    const float c000 = q[0], c100 = q[1], c010 = q[sy], c110 = q[sy + 1];
                    const float c001 = q[sz], c101 = q[sz + 1], c011 = q[sz + sy], c111 = q[sz + sy + 1];
                    const float a00 = fmaf(fx, c100 - c000, c000), a10 = fmaf(fx, c110 - c010, c010);
                    const float a01 = fmaf(fx, c101 - c001, c001), a11 = fmaf(fx, c111 - c011, c011);
                    const float b0 = fmaf(fy, a10 - a00, a00), b1 = fmaf(fy, a11 - a01, a01);
                    acc += fmaf(fz, b1 - b0, b0);
                }
            }
        } else if (act) {
            for (int j = j0; j <= j1; j++) {
                const float jf = (float)j;
                const float ux = at(r, 0, jf, fb), uy = at(r, 1, jf, fb), uz = at(r, 2, jf, fb);
                const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
                acc += gather8(V, g, ib[0] + (int)flx, ib[1] + (int)fly, ib[2] + (int)flz, ux - flx, uy - fly,
                               uz - flz);
            }
        }
        __syncthreads();
    }
    if (in) proj[((int64_t)p * nv + b) * nu + a] = step * acc;
}

template <typename T, int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_project(GridD g, int nu, int nv, int ntu, float step,
                                                  const pmf_view* __restrict__ views, const T* __restrict__ vol,
                                                  int64_t vol_stride, float* __restrict__ proj) {
    __shared__ float box[kBox];
    __shared__ BoxState bs;
    project_tile<T, CH, RPB>(g, nu, nv, ntu, step, views, vol, vol_stride, proj, blockIdx.y, blockIdx.x, box, bs);
}

__global__ void k_absmax_f(const float* __restrict__ x, int64_t n, unsigned* out) { absmax_bits(x, n, out); }

// ----------------------------------------------------------------- adjoint

// 2x2x2 corner weights of the cell a ray is in, slot c = dx + 2 dy + 4 dz.
struct Window {
    int cx, cy, cz;
    float w[8];
};

__device__ __forceinline__ void win_clear(Window& W) {
#pragma unroll
    for (int c = 0; c < 8; c++) W.w[c] = 0.0f;
}

// Direct global sink (chunks whose box does not fit in shared memory).
struct GlobalSink {
    unsigned long long* acc;
    GridD g;
    float scale;  // step * g * 2^kg
    __device__ __forceinline__ void put(int x, int y, int z, float w) const {
        if (w == 0.0f) return;
        if ((unsigned)x >= (unsigned)g.nx || (unsigned)y >= (unsigned)g.ny || (unsigned)z >= (unsigned)g.nz) return;
        red_add(acc + ((int64_t)z * g.ny + y) * g.nx + x, to_fixed(w, scale));
    }
};

template <class S>
__device__ __forceinline__ void win_flush_all(Window& W, const S& s) {
#pragma unroll
    for (int c = 0; c < 8; c++) s.put(W.cx + (c & 1), W.cy + ((c >> 1) & 1), W.cz + (c >> 2), W.w[c]);
    win_clear(W);
}

// Move the window to cell (x, y, z): corners shared by the old and new cell
// keep their weights, the others are flushed.
template <class S>
__device__ __forceinline__ void win_move(Window& W, int x, int y, int z, const S& s) {
    const int dx = x - W.cx, dy = y - W.cy, dz = z - W.cz;
    if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) {
        win_flush_all(W, s);
        W.cx = x; W.cy = y; W.cz = z;
        return;
    }
    if (dx == 1) {
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
            s.put(W.cx, W.cy + ((c >> 1) & 1), W.cz + (c >> 2), W.w[c]);
            W.w[c] = W.w[c + 1];
            W.w[c + 1] = 0.0f;
        }
        W.cx += 1;
    } else if (dx == -1) {
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
            s.put(W.cx + 1, W.cy + ((c >> 1) & 1), W.cz + (c >> 2), W.w[c + 1]);
            W.w[c + 1] = W.w[c];
            W.w[c] = 0.0f;
        }
        W.cx -= 1;
    }
    if (dy == 1) {
#pragma unroll
        for (int c = 0; c < 8; c++) {
            if (c & 2) continue;
            s.put(W.cx + (c & 1), W.cy, W.cz + (c >> 2), W.w[c]);
            W.w[c] = W.w[c + 2];
            W.w[c + 2] = 0.0f;
        }
        W.cy += 1;
    } else if (dy == -1) {
#pragma unroll
        for (int c = 0; c < 8; c++) {
            if (c & 2) continue;
            s.put(W.cx + (c & 1), W.cy + 1, W.cz + (c >> 2), W.w[c + 2]);
            W.w[c + 2] = W.w[c];
            W.w[c] = 0.0f;
        }
        W.cy -= 1;
    }
    if (dz == 1) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            s.put(W.cx + (c & 1), W.cy + ((c >> 1) & 1), W.cz, W.w[c]);
            W.w[c] = W.w[c + 4];
            W.w[c + 4] = 0.0f;
        }
        W.cz += 1;
    } else if (dz == -1) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            s.put(W.cx + (c & 1), W.cy + ((c >> 1) & 1), W.cz + 1, W.w[c + 4]);
            W.w[c + 4] = W.w[c];
            W.w[c] = 0.0f;
        }
        W.cz -= 1;
    }
}

__device__ __forceinline__ void win_add(Window& W, float fx, float fy, float fz) {
    const float ex = 1.0f - fx, ey = 1.0f - fy, ez = 1.0f - fz;
    const float a0 = ey * ez, a1 = fy * ez, a2 = ey * fz, a3 = fy * fz;
    W.w[0] = fmaf(ex, a0, W.w[0]); W.w[1] = fmaf(fx, a0, W.w[1]);
    W.w[2] = fmaf(ex, a1, W.w[2]); W.w[3] = fmaf(fx, a1, W.w[3]);
    W.w[4] = fmaf(ex, a2, W.w[4]); W.w[5] = fmaf(fx, a2, W.w[5]);
    W.w[6] = fmaf(ex, a3, W.w[6]); W.w[7] = fmaf(fx, a3, W.w[7]);
}

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: floats in [2^23, 2^24) are integers
constexpr int kMagicBits = 0x4b400000;

// 2^k so that a bound b < 2^(bits) after scaling.
__device__ __forceinline__ int exp_for(float bound, int bits) {
    if (!(bound > 0.0f) || !isfinite(bound)) return 0;
    int e;
    frexpf(bound, &e);
    const int k = bits - e;
    return k > 126 ? 126 : (k < -126 ? -126 : k);
}

// Adjoint lane layout: lane l = g + 8 q of warp w takes pixel
// (2 g + (w & 1), (w >> 1) + 4 q) of the 16x16 tile and starts its chunk at
// sample 3 g + 2 q.  Shared-memory atomics are served per half-warp, and
// within each half this spreads the 16 simultaneous corner addresses over the
// banks (about 3.6 conflict rounds per warp-wide atomic at the paper
// geometry, against 4.3 for adjacent pixels staggered 4 samples apart).
template <int RPB>
__device__ __forceinline__ void pixel_of_spread(int tile, int ntu, int& a, int& b) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, g = l & 7, q = l >> 3;
    const int tu = tile % ntu, tv = tile / ntu;
    a = tu * 16 + 2 * g + (w & 1);
    b = tv * (RPB / 16) + (w >> 1) + (RPB / 64) * q;
}

__device__ __forceinline__ int adjoint_phase() {
    const int l = threadIdx.x & 31;
    return 3 * (l & 7) + 2 * (l >> 3);
}

// One pixel tile of view p of the adjoint; box must be all zero on entry and is
// all zero again on return.
template <int CH, int RPB>
__device__ __forceinline__ void backproject_tile(const GridD& g, int nu, int nv, int ntu, float step,
                                                 const pmf_view* __restrict__ views,
                                                 const float* __restrict__ dproj, int64_t vol_stride,
                                                 unsigned long long* __restrict__ acc, const unsigned* maxbits,
                                                 float bound_mult, float samples_per_voxel, int p, int tile,
                                                 int* box, BoxState& bs, unsigned& sgmax, float* gsum) {
    int a, b;
    pixel_of_spread<RPB>(tile, ntu, a, b);
    const bool in = a < nu && b < nv;
    const float gy = in ? __ldg(dproj + ((int64_t)p * nv + b) * nu + a) : 0.0f;
    Ray r;
    if (in && gy != 0.0f) {
        r = ray_init(views[p], nu, nv, a, b, g, (double)step);
    } else {
        r.mlo = 1; r.mhi = 0;
    }
    const bool live = r.mlo <= r.mhi;
    // scales: global 2^kg (all views, provable bound) and CTA 2^kb <= 2^kg.
    // Within one chunk a voxel receives at most step * S * sum_r |g_r| from the
    // CTA's rays, where S bounds the trilinear weight one ray's samples put in
    // one voxel (a hat function sampled at spacing h sums to at most 1/h + 1).
    if (threadIdx.x == 0) sgmax = 0u;
    __syncthreads();
    {
        float a = live ? fabsf(gy) : 0.0f;
        unsigned m = __reduce_max_sync(kFull, __float_as_uint(a));
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
        if ((threadIdx.x & 31) == 0) {
            gsum[threadIdx.x >> 5] = a;
            if (m) atomicMax(&sgmax, m);
        }
    }
    __syncthreads();
    float gtot = 0.0f;
    for (int i = 0; i < RPB / 32; i++) gtot += gsum[i];  // fixed order, same in every thread
    const int kg = fixed_exponent(__uint_as_float(*maxbits) * bound_mult);
    const float bcta = gtot * step * samples_per_voxel;
    const float bray = __uint_as_float(sgmax) * step * samples_per_voxel;
    // box sums < 2^29 and every single addend < 2^21 (round_small needs < 2^22)
    const int kb = min(min(exp_for(bcta, 29), exp_for(bray, 21)), kg);
    const int shift = kg - kb;
    const float gsb = step * gy * ldexpf(1.0f, kb), gsg = step * gy * ldexpf(1.0f, kg);
    unsigned long long* A = acc + (int64_t)p * vol_stride;
    const GlobalSink gsink{A, g, gsg};

    block_range(bs, r, live);
    const int Mlo = bs.range[0], Mhi = bs.range[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int sel = 0;
    for (int M0 = Mlo; M0 <= Mhi; M0 += CH, sel ^= 1) {
        int j0, j1, ib[3];
        float fb[3];
        const bool act = chunk_begin<CH>(bs, sel, r, live, M0, j0, j1, ib, fb);
        __syncthreads();
        const Box bx = read_box(bs, sel);
        if (threadIdx.x == 0 && bx.vol > 0 && !bx.fits) diag_count(PMF_DIAG_BACKPROJECT_BOX_FALLBACK);
        if (bx.vol > 0 && bx.fits) {
            if (act) {
                const int sy = kPitch, sz = kPitch * bx.by;
                const float syf = (float)sy, szf = (float)sz;
                // positions relative to the anchor cell, bounded like the box
                int* qa = box + (ib[0] - bx.lx) + (ib[1] - bx.ly) * sy + (ib[2] - bx.lz) * sz;
                // every sample adds its 8 scaled corner weights to the box; the
                // weights are formed with the bias kMagic, so each rounds to an
                // integer-valued float and converts with one integer subtract.
                // Lanes start at staggered samples (adjoint_phase), so a
                // half-warp's simultaneous atomics land on different voxels
                // and mostly different banks.
                const int phase = adjoint_phase();
                for (int k = 0; k < CH; k++) {
                    const int j = (k + phase) & (CH - 1);
                    if (j < j0 || j > j1) continue;
                    const float jf = (float)j;
                    const float ux = fmaf(jf, r.dh[0], fb[0]), uy = fmaf(jf, r.dh[1], fb[1]),
                                uz = fmaf(jf, r.dh[2], fb[2]);
                    const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
                    const int idx = (int)fmaf(flz, szf, fmaf(fly, syf, flx));
                    const float fx = ux - flx, fy = uy - fly, fz = uz - flz;
                    const float ex = 1.0f - fx, ey = 1.0f - fy, ez = (1.0f - fz) * gsb, fzs = fz * gsb;
                    const float a0 = ey * ez, a1 = fy * ez, a2 = ey * fzs, a3 = fy * fzs;
                    int* q = qa + idx;
                    int* q2 = q + sz;
                    atomicAdd(q, __float_as_int(fmaf(ex, a0, kMagic)) - kMagicBits);
                    atomicAdd(q + 1, __float_as_int(fmaf(fx, a0, kMagic)) - kMagicBits);
                    atomicAdd(q + kPitch, __float_as_int(fmaf(ex, a1, kMagic)) - kMagicBits);
                    atomicAdd(q + kPitch + 1, __float_as_int(fmaf(fx, a1, kMagic)) - kMagicBits);
                    atomicAdd(q2, __float_as_int(fmaf(ex, a2, kMagic)) - kMagicBits);
                    atomicAdd(q2 + 1, __float_as_int(fmaf(fx, a2, kMagic)) - kMagicBits);
                    atomicAdd(q2 + kPitch, __float_as_int(fmaf(ex, a3, kMagic)) - kMagicBits);
                    atomicAdd(q2 + kPitch + 1, __float_as_int(fmaf(fx, a3, kMagic)) - kMagicBits);
                }
            }
            __syncthreads();
            // flush the box: lane = x, one warp per (y, z) row; one 64-bit atomic
            // per touched in-grid voxel, and re-zero it
            {
                const int x = bx.lx + lane;
                const bool xin = lane < bx.bx && (unsigned)x < (unsigned)g.nx;
                for (int zz = 0; zz < bx.bz; zz++) {
                    const int z = bx.lz + zz;
                    for (int yy = warp; yy < bx.by; yy += RPB / 32) {
                        const int i = (zz * bx.by + yy) * kPitch + lane;
                        if (lane >= bx.bx) continue;
                        const int v = box[i];
                        if (v == 0) continue;
                        box[i] = 0;
                        const int y = bx.ly + yy;
                        if (xin && (unsigned)y < (unsigned)g.ny && (unsigned)z < (unsigned)g.nz)
                            atomicAdd(A + ((int64_t)z * g.ny + y) * g.nx + x,
                                      (unsigned long long)((long long)v * (1ll << shift)));
                    }
                }
            }
        } else if (act) {
            Window W;
            W.cx = INT_MIN;
            win_clear(W);
            for (int j = j0; j <= j1; j++) {
                const float jf = (float)j;
                const float ux = at(r, 0, jf, fb), uy = at(r, 1, jf, fb), uz = at(r, 2, jf, fb);
                const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
                const int cx = ib[0] + (int)flx, cy = ib[1] + (int)fly, cz = ib[2] + (int)flz;
                if (W.cx == INT_MIN) {
                    W.cx = cx; W.cy = cy; W.cz = cz;
                } else if (cx != W.cx || cy != W.cy || cz != W.cz) {
                    win_move(W, cx, cy, cz, gsink);
                }
                win_add(W, ux - flx, uy - fly, uz - flz);
            }
            if (W.cx != INT_MIN) win_flush_all(W, gsink);
        }
        __syncthreads();
    }
}

template <int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_backproject(GridD g, int nu, int nv, int ntu, float step,
                                                      const pmf_view* __restrict__ views,
                                                      const float* __restrict__ dproj, int64_t vol_stride,
                                                      unsigned long long* __restrict__ acc, const unsigned* maxbits,
                                                      float bound_mult, float samples_per_voxel) {
    __shared__ int box[kBox];
    __shared__ BoxState bs;
    __shared__ unsigned sgmax;
    __shared__ float gsum[RPB / 32];
    for (int i = threadIdx.x; i < kBox; i += RPB) box[i] = 0;
    backproject_tile<CH, RPB>(g, nu, nv, ntu, step, views, dproj, vol_stride, acc, maxbits, bound_mult, samples_per_voxel,
                     blockIdx.y, blockIdx.x, box, bs, sgmax, gsum);
}

__global__ void k_fixed_to_float_f(const unsigned long long* __restrict__ acc, int64_t n, const unsigned* maxbits,
                                   float bound_mult, float* out, int accumulate) {
    const float bound = __uint_as_float(*maxbits) * bound_mult;
    const int kexp = fixed_exponent(bound);
    const float inv = ldexpf(1.0f, -kexp);
    const bool bad = !isfinite(bound);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) diag_count(PMF_DIAG_NONFINITE);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float r = bad ? __int_as_float(0x7fc00000) : from_fixed(acc[t], inv);
        out[t] = accumulate ? out[t] + r : r;
    }
}

// ------------------------------------------------- batched (uneven) launches
//
// Several volumes -- different grids, detectors and view counts -- in one
// persistent launch: work item w is tile (w - begin_i) % ntiles_i of view
// (w - begin_i) / ntiles_i of item i, and each CTA walks the work items
// round-robin.  A tile's arithmetic is the single-volume kernel's, so the
// results equal per-volume launches bit for bit.

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

template <typename T, int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_project_batched(const __grid_constant__ ProjBatch B) {
    __shared__ float box[kBox];
    __shared__ BoxState bs;
    for (int64_t w = blockIdx.x; w < B.total; w += gridDim.x) {
        const ProjItem& it = B.it[find_item(B, w)];
        const int64_t local = w - it.begin;
        project_tile<T, CH, RPB>(it.g, it.nu, it.nv, it.ntu, it.step, it.views, (const T*)it.vol, it.vol_stride, it.proj,
                        (int)(local / it.ntiles), (int)(local % it.ntiles), box, bs);
        __syncthreads();
    }
}

template <int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_backproject_batched(const __grid_constant__ ProjBatch B) {
    __shared__ int box[kBox];
    __shared__ BoxState bs;
    __shared__ unsigned sgmax;
    __shared__ float gsum[RPB / 32];
    for (int i = threadIdx.x; i < kBox; i += RPB) box[i] = 0;
    for (int64_t w = blockIdx.x; w < B.total; w += gridDim.x) {
        const ProjItem& it = B.it[find_item(B, w)];
        const int64_t local = w - it.begin;
        backproject_tile<CH, RPB>(it.g, it.nu, it.nv, it.ntu, it.step, it.views, it.dproj, it.vol_stride, it.acc, it.maxbits,
                         it.bound_mult, it.spv, (int)(local / it.ntiles), (int)(local % it.ntiles), box, bs, sgmax,
                         gsum);
        __syncthreads();
    }
}

// blockIdx.y = item
__global__ void k_absmax_batched(const __grid_constant__ ProjBatch B) {
    const ProjItem& it = B.it[blockIdx.y];
    absmax_bits(it.dproj, it.nq, it.maxbits);
}

__global__ void k_fixed_to_float_batched(const __grid_constant__ ProjBatch B, int accumulate) {
    const ProjItem& it = B.it[blockIdx.y];
    const float bound = __uint_as_float(*it.maxbits) * it.bound_mult;
    const int kexp = fixed_exponent(bound);
    const float inv = ldexpf(1.0f, -kexp);
    const bool bad = !isfinite(bound);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) diag_count(PMF_DIAG_NONFINITE);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < it.cells; t += (int64_t)gridDim.x * blockDim.x) {
        const float r = bad ? __int_as_float(0x7fc00000) : from_fixed(it.acc[t], inv);
        it.dvol[t] = accumulate ? it.dvol[t] + r : r;
    }
}

// ------------------------------------------------------------------ loss

constexpr int kLossThreads = 256;

__global__ void __launch_bounds__(kLossThreads) k_loss(int kind, int64_t n, const float* __restrict__ pred,
                                                       const float* __restrict__ meas, float* d_pred, float* part) {
    __shared__ float red[kLossThreads / 32];
    const float invn = 1.0f / (float)n;
    float s = 0.0f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float r = __ldg(pred + t) - __ldg(meas + t);
        if (kind == 1) {
            s += fabsf(r);
            if (d_pred) d_pred[t] = (r > 0.0f ? invn : (r < 0.0f ? -invn : 0.0f));
        } else {
            s = fmaf(r, r, s);
            if (d_pred) d_pred[t] = 2.0f * r * invn;
        }
    }
    const float tot = block_sum<kLossThreads>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_loss_final(const float* part, int nb, int64_t n, float* loss) {
    double s = 0.0;  // one thread; fixed order
    for (int b = 0; b < nb; b++) s += (double)part[b];
    *loss = (float)(s / (double)n);
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

bool valid_shape(const MarchShape& sh) {
    return (sh.chunk == 16 || sh.chunk == 32) && (sh.rays == 128 || sh.rays == 256) && sh.form >= 0 && sh.form <= 16;
}

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

// Persistent CTAs: `ctas` if given, else as many as are resident at 256
// threads x 4 per SM (<= 64 registers), i.e. 1024 threads per SM.
unsigned persistent_ctas(int64_t total, unsigned ctas, int rays) {
    const int64_t cap = ctas ? (int64_t)ctas : (int64_t)num_sms() * (1024 / rays);
    return (unsigned)(total < cap ? (total > 0 ? total : 1) : cap);
}

pmf_status project_grid(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views,
                        pmf_dtype dtype, const void* vol, int64_t vol_stride, float* proj, const MarchShape& sh,
                        cudaStream_t s) {
    pmf_status st = check_proj(grid, det, P, views);
    if (st != PMF_OK) return st;
    if ((st = validate_dtype(dtype)) != PMF_OK) return st;
    if (P == 0) return PMF_OK;
    PMF_REQUIRE(vol && proj, "null pointer");
    PMF_REQUIRE(vol_stride >= 0, "vol_stride must be >= 0");
    GridD g = make_grid(grid);
    const int ntu = (det->nu + 15) / 16, ntv = tiles_v(det->nv, sh.rays);
    dim3 gr((unsigned)(ntu * ntv), (unsigned)P);
    PMF_DISPATCH_MARCH(sh, CH, RPB, PMF_DISPATCH_DTYPE(dtype, T, k_project<T, CH, RPB><<<gr, RPB, 0, s>>>(g, det->nu, det->nv, ntu, det->step_mm, views, (const T*)vol, vol_stride, proj)));
    return check_launch("conebeam_project");
}

pmf_status backproject_grid(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views,
                            const float* d_proj, float* d_vol, int64_t vol_stride, int accumulate, void* ws,
                            size_t ws_bytes, const MarchShape& sh, cudaStream_t s) {
    pmf_status st = check_proj(grid, det, P, views);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(vol_stride >= 0, "vol_stride must be >= 0");
    PMF_REQUIRE(d_vol != nullptr && (P == 0 || d_proj != nullptr), "null pointer");
    size_t need;
    conebeam_project_backward_workspace(grid, P, vol_stride, &need);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    GridD g = make_grid(grid);
    unsigned* maxbits = (unsigned*)ws;
    unsigned long long* acc = (unsigned long long*)((char*)ws + align_up(256));
    cudaMemsetAsync(ws, 0, need, s);
    const int64_t Q = (int64_t)det->nu * det->nv;
    const double rays = (double)Q * (vol_stride ? 1.0 : (double)P);
    const float bound_mult = (float)((double)det->step_mm * rays * (double)max_samples_per_voxel(grid, det->step_mm));
    const int64_t cells = vol_stride ? (int64_t)(P > 0 ? P - 1 : 0) * vol_stride + g.n : g.n;
    if (P > 0) {
        const int64_t nq = Q * P;
        int64_t nb = (nq + 255) / 256;
        k_absmax_f<<<(unsigned)(nb < 1024 ? nb : 1024), 256, 0, s>>>(d_proj, nq, maxbits);
        const int ntu = (det->nu + 15) / 16, ntv = tiles_v(det->nv, sh.rays);
        dim3 gr((unsigned)(ntu * ntv), (unsigned)P);
        const float spv = chunk_samples_per_voxel(grid, det->step_mm, sh.chunk);
        PMF_DISPATCH_MARCH(sh, CH, RPB, k_backproject<CH, RPB><<<gr, RPB, 0, s>>>(g, det->nu, det->nv, ntu, det->step_mm, views, d_proj, vol_stride, acc, maxbits, bound_mult, spv));
    }
    int64_t nb = (cells + 255) / 256;
    k_fixed_to_float_f<<<(unsigned)(nb < 4 * kStreamBlocks ? nb : 4 * kStreamBlocks), 256, 0, s>>>(
        acc, cells, maxbits, bound_mult, d_vol, accumulate);
    return check_launch("conebeam_project_backward");
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
    it.P = in.P;
    it.step = in.det.step_mm;
    it.views = in.views;
    it.vol_stride = in.vol_stride;
    it.nq = (int64_t)in.det.nu * in.det.nv * in.P;
    it.begin = begin;
    return PMF_OK;
}

pmf_status project_batched_impl(int32_t n, const pmf_project_item* items, pmf_dtype dtype, const MarchShape& sh,
                                unsigned ctas, cudaStream_t s) {
    PMF_REQUIRE(n >= 0 && n <= kMaxItems, "n must be in [0, %d]", kMaxItems);
    PMF_REQUIRE(n == 0 || items != nullptr, "items is null");
    pmf_status st = validate_dtype(dtype);
    if (st != PMF_OK) return st;
    ProjBatch B{};
    B.n = n;
    int64_t total = 0;
    for (int i = 0; i < n; i++) {
        if ((st = fill_item(items[i], total, sh.rays, B.it[i])) != PMF_OK) return st;
        PMF_REQUIRE(items[i].P == 0 || (items[i].vol && items[i].proj), "item %d: null pointer", i);
        B.it[i].vol = items[i].vol;
        B.it[i].proj = items[i].proj;
        total += (int64_t)B.it[i].ntiles * items[i].P;
    }
    B.total = total;
    if (total == 0) return PMF_OK;
    const unsigned nc = persistent_ctas(total, ctas, sh.rays);
    PMF_DISPATCH_MARCH(sh, CH, RPB, PMF_DISPATCH_DTYPE(dtype, T, k_project_batched<T, CH, RPB><<<nc, RPB, 0, s>>>(B)));
    return check_launch("conebeam_project_batched");
}

size_t bp_item_bytes(const pmf_backproject_item& it) {
    const int64_t n = (int64_t)it.grid.nx * it.grid.ny * it.grid.nz;
    const int64_t cells = it.vol_stride ? (int64_t)(it.P > 0 ? it.P - 1 : 0) * it.vol_stride + n : n;
    return align_up(256) + align_up(sizeof(unsigned long long) * (size_t)cells);
}

pmf_status backproject_batched_impl(int32_t n, const pmf_backproject_item* items, int accumulate, void* ws,
                                    size_t ws_bytes, const MarchShape& sh, unsigned ctas, cudaStream_t s) {
    size_t need = 0;
    pmf_status st = conebeam_project_backward_batched_workspace(n, items, &need);
    if (st != PMF_OK) return st;
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    ProjBatch B{};
    B.n = n;
    int64_t total = 0, maxq = 0, maxcells = 0;
    char* cur = (char*)ws;
    for (int i = 0; i < n; i++) {
        const pmf_backproject_item& in = items[i];
        pmf_project_item tmp{in.grid, in.det, in.P, in.views, nullptr, in.vol_stride, nullptr};
        if ((st = fill_item(tmp, total, sh.rays, B.it[i])) != PMF_OK) return st;
        PMF_REQUIRE(in.d_vol != nullptr && (in.P == 0 || in.d_proj != nullptr), "item %d: null pointer", i);
        ProjItem& it = B.it[i];
        const int64_t Q = (int64_t)in.det.nu * in.det.nv;
        const double rays = (double)Q * (in.vol_stride ? 1.0 : (double)in.P);
        it.bound_mult = (float)((double)in.det.step_mm * rays * (double)max_samples_per_voxel(&in.grid, in.det.step_mm));
        it.spv = chunk_samples_per_voxel(&in.grid, in.det.step_mm, sh.chunk);
        it.dproj = in.d_proj;
        it.dvol = in.d_vol;
        it.maxbits = (unsigned*)cur;
        it.acc = (unsigned long long*)(cur + align_up(256));
        it.cells = in.vol_stride ? (int64_t)(in.P > 0 ? in.P - 1 : 0) * in.vol_stride + it.g.n : it.g.n;
        cur += bp_item_bytes(in);
        total += (int64_t)it.ntiles * in.P;
        maxq = it.nq > maxq ? it.nq : maxq;
        maxcells = it.cells > maxcells ? it.cells : maxcells;
    }
    B.total = total;
    if (n == 0) return PMF_OK;
    cudaMemsetAsync(ws, 0, need, s);
    if (maxq > 0) {
        const int64_t nb = (maxq + 255) / 256;
        k_absmax_batched<<<dim3((unsigned)(nb < 1024 ? nb : 1024), (unsigned)n), 256, 0, s>>>(B);
    }
    if (total > 0) {
        const unsigned nc = persistent_ctas(total, ctas, sh.rays);
        PMF_DISPATCH_MARCH(sh, CH, RPB, k_backproject_batched<CH, RPB><<<nc, RPB, 0, s>>>(B));
    }
    const int64_t nc = (maxcells + 255) / 256;
    k_fixed_to_float_batched<<<dim3((unsigned)(nc < 4 * kStreamBlocks ? nc : 4 * kStreamBlocks), (unsigned)n), 256, 0, s>>>(
        B, accumulate);
    return check_launch("conebeam_project_backward_batched");
}

}  // namespace

PMF_DIAG_ACCESSOR(diag_project)

// Launch shapes for plans: form 0 is one CTA per (view, tile), form k > 0 a
// persistent launch of k CTAs per SM; chunk and rays pick the kernel variant.
// Every form and shape runs the same per-sample arithmetic; the chunk length
// moves the float-float anchors (results differ in the last bits) and the
// rays per CTA the adjoint's per-CTA fixed-point scale (likewise).
pmf_status project_launch(const pmf_project_item& it, pmf_dtype dtype, const MarchShape& sh, cudaStream_t s) {
    if (!valid_shape(sh)) return set_error(PMF_EINVAL, "invalid march shape");
    if (sh.form == 0)
        return project_grid(&it.grid, &it.det, it.P, it.views, dtype, it.vol, it.vol_stride, it.proj, sh, s);
    return project_batched_impl(1, &it, dtype, sh, (unsigned)(sh.form * num_sms()), s);
}

pmf_status backproject_launch(const pmf_backproject_item& it, int accumulate, void* ws, size_t ws_bytes,
                              const MarchShape& sh, cudaStream_t s) {
    if (!valid_shape(sh)) return set_error(PMF_EINVAL, "invalid march shape");
    if (sh.form == 0)
        return backproject_grid(&it.grid, &it.det, it.P, it.views, it.d_proj, it.d_vol, it.vol_stride, accumulate,
                                ws, ws_bytes, sh, s);
    return backproject_batched_impl(1, &it, accumulate, ws, ws_bytes, sh, (unsigned)(sh.form * num_sms()), s);
}

}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status conebeam_project(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views,
                            pmf_dtype dtype, const void* vol, int64_t vol_stride, float* proj, pmf_stream stream) {
    return project_grid(grid, det, P, views, dtype, vol, vol_stride, proj, MarchShape{}, (cudaStream_t)stream);
}

pmf_status conebeam_project_backward_workspace(const pmf_grid* grid, int32_t P, int64_t vol_stride, size_t* bytes) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(bytes != nullptr && P >= 0 && vol_stride >= 0, "bad arguments");
    const int64_t n = (int64_t)grid->nx * grid->ny * grid->nz;
    const int64_t cells = vol_stride ? (int64_t)(P > 0 ? P - 1 : 0) * vol_stride + n : n;
    *bytes = align_up(256) + align_up(sizeof(unsigned long long) * (size_t)cells);
    return PMF_OK;
}

pmf_status conebeam_project_backward(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views,
                                     const float* d_proj, float* d_vol, int64_t vol_stride, int accumulate, void* ws,
                                     size_t ws_bytes, pmf_stream stream) {
    return backproject_grid(grid, det, P, views, d_proj, d_vol, vol_stride, accumulate, ws, ws_bytes, MarchShape{},
                            (cudaStream_t)stream);
}

pmf_status conebeam_project_batched(int32_t n, const pmf_project_item* items, pmf_dtype dtype, pmf_stream stream) {
    return project_batched_impl(n, items, dtype, MarchShape{}, 0, (cudaStream_t)stream);
}

pmf_status conebeam_project_backward_batched_workspace(int32_t n, const pmf_backproject_item* items, size_t* bytes) {
    PMF_REQUIRE(bytes != nullptr && n >= 0 && n <= kMaxItems && (n == 0 || items != nullptr), "bad arguments");
    size_t tot = 0;
    for (int i = 0; i < n; i++) {
        pmf_status st = validate_grid(&items[i].grid);
        if (st != PMF_OK) return st;
        tot += bp_item_bytes(items[i]);
    }
    *bytes = tot;
    return PMF_OK;
}

pmf_status conebeam_project_backward_batched(int32_t n, const pmf_backproject_item* items, int accumulate, void* ws,
                                             size_t ws_bytes, pmf_stream stream) {
    return backproject_batched_impl(n, items, accumulate, ws, ws_bytes, MarchShape{}, 0, (cudaStream_t)stream);
}

pmf_status projection_loss_workspace(int64_t count, size_t* bytes) {
    PMF_REQUIRE(bytes != nullptr && count >= 0, "bad arguments");
    *bytes = align_up(sizeof(float) * kStreamBlocks);
    return PMF_OK;
}

pmf_status projection_loss(int32_t kind, int32_t P, int64_t Q, const float* pred, const float* meas, float* loss,
                           float* d_pred, void* ws, size_t ws_bytes, pmf_stream stream) {
    PMF_REQUIRE(kind == 1 || kind == 2, "kind must be 1 (L1) or 2 (L2)");
    PMF_REQUIRE(P >= 1 && Q >= 1, "P and Q must be positive");
    PMF_REQUIRE(pred && meas && loss, "null pointer");
    size_t need;
    projection_loss_workspace((int64_t)P * Q, &need);
    pmf_status st = validate_ws(ws, ws_bytes, need);
    if (st != PMF_OK) return st;
    const int64_t n = (int64_t)P * Q;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t nb = (n + kLossThreads - 1) / kLossThreads;
    const int blocks = (int)(nb < kStreamBlocks ? nb : kStreamBlocks);
    k_loss<<<blocks, kLossThreads, 0, s>>>(kind, n, pred, meas, d_pred, (float*)ws);
    k_loss_final<<<1, 1, 0, s>>>((const float*)ws, blocks, n, loss);
    return check_launch("projection_loss");
}

}  // extern "C"
