// Exact adjoint of the cone-beam ray marcher (Eq. 6) for sm_103a.  Every
// sample adds its 8 trilinear corner weights into a shared-memory box in
// 32-bit fixed point (per-CTA scale); a warp's lanes take spread pixels and
// start their chunk at staggered samples, so its simultaneous atomics land on
// different voxels.  The box's bank layout follows the tile's rays: rows 33
// words apart (65 for boxes wider than 32 voxels), x mirrored when the rays' x
// and y steps differ in sign, planes a stride of 16 (mod 32) words apart,
// which keeps the cells of nearby samples in different banks.  The box is then flushed with one 64-bit
// fixed-point atomic per touched voxel (global scale 2^k from a provable
// bound).  Integer sums are order independent, so the result is
// bit-reproducible and independent of the layout.  A chunk whose box does not
// fit in shared memory falls back to direct global atomics.
#include "march.cuh"

namespace pmf {
namespace {

// The adjoint's shared box: 192 words per sample of the chunk (9,216 words for
// the default 48-sample chunk), in dynamic shared memory.
template <int CH>
__host__ __device__ constexpr int box_words() { return 192 * CH; }

// (chunk, rays) -> template instantiation of the adjoint, whose chunks may
// also be 48 and 64 samples long
#define PMF_DISPATCH_ADJOINT(sh, CH, RPB, ...)                                                                \
    switch ((sh).chunk * 1000 + (sh).rays) {                                                                \
        case 48128: { constexpr int CH = 48, RPB = 128; __VA_ARGS__; break; }                               \
        case 48256: { constexpr int CH = 48, RPB = 256; __VA_ARGS__; break; }                               \
        case 64128: { constexpr int CH = 64, RPB = 128; __VA_ARGS__; break; }                               \
        case 64256: { constexpr int CH = 64, RPB = 256; __VA_ARGS__; break; }                               \
        case 32128: { constexpr int CH = 32, RPB = 128; __VA_ARGS__; break; }                               \
        case 32256: { constexpr int CH = 32, RPB = 256; __VA_ARGS__; break; }                               \
        case 16128: { constexpr int CH = 16, RPB = 128; __VA_ARGS__; break; }                               \
        case 16256: { constexpr int CH = 16, RPB = 256; __VA_ARGS__; break; }                               \
        default: return set_error(PMF_EINVAL, "unsupported adjoint shape: chunk %d, rays %d", (sh).chunk, (sh).rays); \
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
// sample 3 g + 2 q (of its own samples in the chunk).  A warp-wide shared
// atomic whose 32 addresses lie in distinct banks takes one wavefront
// (measured); each further address in the busiest bank adds one.  This layout
// spreads the 32 simultaneous corner addresses over the banks (measured at the
// paper geometry: 2.85 wavefronts per warp-wide atomic with the ray-following
// box layout below, 3.8 with a fixed one).
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

// Whether a tile's box stores x mirrored.  With the row pitch 33 a voxel's
// bank is (x + y) mod 32, so cells of nearby samples collide where x and y
// step in opposite directions (x + y stays put); mirroring x in the box,
// (bx - 1 - x + y) mod 32, moves those apart again (it collides only where x
// and y step the same way).  Decided from the ray through the tile's centre:
// mirrored when its x and y steps differ in sign.  Only the bank layout
// depends on it, never a result.
template <int RPB>
__device__ __forceinline__ bool tile_mirror(const pmf_view& vw, int nu, int nv, int ntu, int tile) {
    const float ca = (float)((tile % ntu) * 16 + 8) - 0.5f * (float)nu;
    const float cb = (float)((tile / ntu) * (RPB / 16) + RPB / 32) - 0.5f * (float)nv;
    const float dx = (float)(vw.det[0] - vw.src[0]) + ca * (float)vw.du[0] + cb * (float)vw.dv[0];
    const float dy = (float)(vw.det[1] - vw.src[1]) + ca * (float)vw.du[1] + cb * (float)vw.dv[1];
    return dx * dy < 0.0f;
}

// Plane stride of the box: the smallest stride >= rows * pitch that is 16
// (mod 32), so cells one plane apart fall half a bank row apart.
__device__ __forceinline__ int plane_stride(int rows, int pitch) {
    const int s = rows * pitch;
    return s + ((16 - (s & 31)) & 31);
}

// The samples j0..j1 of one ray of the chunk into a box with rows PITCH words
// apart (a template argument, so the corner offsets are immediates) and NBOX
// words in all.
template <int PITCH, int NBOX>
__device__ __forceinline__ void scatter_samples(const Ray& r, const Box& bx, int sz, bool mirror, float sxf, float gsb,
                                                int j0, int j1, const int ib[3], const float fb[3], int* box) {
    constexpr int sy = PITCH;
    const float syf = (float)sy, szf = (float)sz;
    // positions relative to the anchor cell, bounded like the box.
    // Box column of voxel x: x - lx, or bx - 1 - (x - lx) mirrored;
    // a sample's base address is its cell's lower-x corner, or its
    // upper-x corner when mirrored, so the corners always sit at
    // +0, +1, +sy, +sy + 1 (the two x weights trade places)
    int* qa = box + (mirror ? bx.bx - 2 - (ib[0] - bx.lx) : ib[0] - bx.lx) + (ib[1] - bx.ly) * sy +
              (ib[2] - bx.lz) * sz;
    // every sample adds its 8 scaled corner weights to the box; the
    // weights are formed with the bias kMagic, so each rounds to an
    // integer-valued float and converts with one integer subtract.
    // Lanes start at staggered samples (adjoint_phase), so a
    // warp's simultaneous atomics land on different voxels and
    // mostly different banks.
    // each lane visits exactly its own samples j0..j1, starting at its
    // stagger (taken modulo its count) and wrapping, so a chunk the
    // ray only enters or leaves costs no idle iterations
    const int len = j1 - j0 + 1;
    int jj = adjoint_phase() % len;
    for (int k = 0; k < len; k++) {
        const int j = j0 + jj;
        jj = jj + 1 == len ? 0 : jj + 1;
        const float jf = (float)j;
        const float ux = fmaf(jf, r.dh[0], fb[0]), uy = fmaf(jf, r.dh[1], fb[1]),
                    uz = fmaf(jf, r.dh[2], fb[2]);
        const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
        const int idx = (int)fmaf(flx, sxf, fmaf(fly, syf, flz * szf));
        const float fx = ux - flx, fy = uy - fly, fz = uz - flz;
        const float ex = 1.0f - fx, ey = 1.0f - fy, ez = (1.0f - fz) * gsb, fzs = fz * gsb;
        const float a0 = ey * ez, a1 = fy * ez, a2 = ey * fzs, a3 = fy * fzs;
        const float w0 = mirror ? fx : ex, w1 = mirror ? ex : fx;  // the corners at +0 and +1
        int* q = qa + idx;
        int* q2 = q + sz;
        if (!PMF_DCHECK(q >= box && q2 + PITCH + 1 < box + NBOX)) continue;
        atomicAdd(q, __float_as_int(fmaf(w0, a0, kMagic)) - kMagicBits);
        atomicAdd(q + 1, __float_as_int(fmaf(w1, a0, kMagic)) - kMagicBits);
        atomicAdd(q + PITCH, __float_as_int(fmaf(w0, a1, kMagic)) - kMagicBits);
        atomicAdd(q + PITCH + 1, __float_as_int(fmaf(w1, a1, kMagic)) - kMagicBits);
        atomicAdd(q2, __float_as_int(fmaf(w0, a2, kMagic)) - kMagicBits);
        atomicAdd(q2 + 1, __float_as_int(fmaf(w1, a2, kMagic)) - kMagicBits);
        atomicAdd(q2 + PITCH, __float_as_int(fmaf(w0, a3, kMagic)) - kMagicBits);
        atomicAdd(q2 + PITCH + 1, __float_as_int(fmaf(w1, a3, kMagic)) - kMagicBits);
    }
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
    tile_view(bs, views[p], g, step);
    Ray r;
    if (in && gy != 0.0f) {
        r = ray_init(bs.vf, nu, nv, a, b, g);
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
    const bool mirror = tile_mirror<RPB>(views[p], nu, nv, ntu, tile);
    const float sxf = mirror ? -1.0f : 1.0f;
    int sel = 0;
    for (int M0 = Mlo; M0 <= Mhi; M0 += CH, sel ^= 1) {
        int j0, j1, ib[3];
        float fb[3];
        const bool act = chunk_begin<CH>(bs, sel, r, live, M0, j0, j1, ib, fb);
        __syncthreads();
        const Box bx = read_box(bs, sel);
        const int pitch = bx.bx <= 32 ? 33 : 65;
        const int sz = plane_stride(bx.by, pitch);
        const bool fits = bx.vol > 0 && bx.bx <= 64 && (long long)bx.bz * sz <= box_words<CH>();
        if (threadIdx.x == 0 && bx.vol > 0 && !fits) diag_count(PMF_DIAG_BACKPROJECT_BOX_FALLBACK);
        if (fits) {
            if (act) {
                if (pitch == 33) scatter_samples<33, box_words<CH>()>(r, bx, sz, mirror, sxf, gsb, j0, j1, ib, fb, box);
                else scatter_samples<65, box_words<CH>()>(r, bx, sz, mirror, sxf, gsb, j0, j1, ib, fb, box);
            }
            __syncthreads();
            // flush the box: lane = x, one warp per (y, z) row; one 64-bit atomic
            // per touched in-grid voxel, and re-zero it
            for (int col = lane; col < bx.bx; col += 32) {
                const int x = bx.lx + (mirror ? bx.bx - 1 - col : col);  // box column col
                const bool xin = (unsigned)x < (unsigned)g.nx;
                for (int zz = 0; zz < bx.bz; zz++) {
                    const int z = bx.lz + zz;
                    for (int yy = warp; yy < bx.by; yy += RPB / 32) {
                        const int i = zz * sz + yy * pitch + col;
                        if (!PMF_DCHECK(i < box_words<CH>())) continue;
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
__global__ void __launch_bounds__(RPB, 768 / RPB) k_backproject(GridD g, int nu, int nv, int ntu, float step,
                                                      const pmf_view* __restrict__ views,
                                                      const float* __restrict__ dproj, int64_t vol_stride,
                                                      unsigned long long* __restrict__ acc, const unsigned* maxbits,
                                                      float bound_mult, float samples_per_voxel) {
    extern __shared__ int box[];  // box_words<CH>()
    __shared__ BoxState bs;
    __shared__ unsigned sgmax;
    __shared__ float gsum[RPB / 32];
    for (int i = threadIdx.x; i < box_words<CH>(); i += RPB) box[i] = 0;
    backproject_tile<CH, RPB>(g, nu, nv, ntu, step, views, dproj, vol_stride, acc, maxbits, bound_mult, samples_per_voxel,
                     blockIdx.y, blockIdx.x, box, bs, sgmax, gsum);
}

// The fixed-point accumulator to fp32 (added to out when accumulating).  MAX:
// also the maximum of |out| over the written values, as abs_bits, into
// *out_max (zeroed by the caller): the bound a consumer of out would
// otherwise take in a pass of its own.  Blocks are whole warps.
template <bool MAX>
__global__ void k_fixed_to_float_f(const unsigned long long* __restrict__ acc, int64_t n, const unsigned* maxbits,
                                   float bound_mult, float* out, int accumulate, unsigned* out_max) {
    const float bound = __uint_as_float(*maxbits) * bound_mult;
    const int kexp = fixed_exponent(bound);
    const float inv = ldexpf(1.0f, -kexp);
    const bool bad = !isfinite(bound);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) diag_count(PMF_DIAG_NONFINITE);
    unsigned m = 0u;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float r = bad ? __int_as_float(0x7fc00000) : from_fixed(acc[t], inv);
        const float v = accumulate ? out[t] + r : r;
        out[t] = v;
        if (MAX) m = max(m, abs_bits(v));
    }
    if (MAX) block_max_bits(m, out_max);
}

// Four values per thread and iteration: two 16-byte accumulator loads and one
// 16-byte store (out 16-byte aligned); the n % 4 tail element by element.
template <bool MAX>
__global__ void k_fixed_to_float_f4(const unsigned long long* __restrict__ acc, int64_t n, const unsigned* maxbits,
                                    float bound_mult, float* out, int accumulate, unsigned* out_max) {
    const float bound = __uint_as_float(*maxbits) * bound_mult;
    const int kexp = fixed_exponent(bound);
    const float inv = ldexpf(1.0f, -kexp);
    const bool bad = !isfinite(bound);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) diag_count(PMF_DIAG_NONFINITE);
    const float qnan = __int_as_float(0x7fc00000);
    unsigned m = 0u;
    const int64_t n4 = n >> 2, g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    const ulonglong2* a2 = (const ulonglong2*)acc;
    float4* o4 = (float4*)out;
    for (int64_t t = g0; t < n4; t += gs) {
        const ulonglong2 p = a2[2 * t], q = a2[2 * t + 1];
        float4 r;
        r.x = bad ? qnan : from_fixed(p.x, inv);
        r.y = bad ? qnan : from_fixed(p.y, inv);
        r.z = bad ? qnan : from_fixed(q.x, inv);
        r.w = bad ? qnan : from_fixed(q.y, inv);
        if (accumulate) {
            const float4 o = o4[t];
            r.x = o.x + r.x; r.y = o.y + r.y; r.z = o.z + r.z; r.w = o.w + r.w;
        }
        o4[t] = r;
        if (MAX) m = max(m, max(max(abs_bits(r.x), abs_bits(r.y)), max(abs_bits(r.z), abs_bits(r.w))));
    }
    for (int64_t t = 4 * n4 + g0; t < n; t += gs) {
        const float r = bad ? qnan : from_fixed(acc[t], inv);
        const float v = accumulate ? out[t] + r : r;
        out[t] = v;
        if (MAX) m = max(m, abs_bits(v));
    }
    if (MAX) block_max_bits(m, out_max);
}

template <int CH, int RPB>
__global__ void __launch_bounds__(RPB, 768 / RPB) k_backproject_batched(const __grid_constant__ ProjBatch B) {
    extern __shared__ int box[];  // box_words<CH>()
    __shared__ BoxState bs;
    __shared__ unsigned sgmax;
    __shared__ float gsum[RPB / 32];
    for (int i = threadIdx.x; i < box_words<CH>(); i += RPB) box[i] = 0;
    for (int64_t w = blockIdx.x; w < B.total; w += gridDim.x) {
        const ProjItem it = B.it[find_item(B, w)];  // a copy: the tile code reads registers, not the parameter block
        const int local = (int)(w - it.begin);  // < 2^31: checked when the item is filled
        backproject_tile<CH, RPB>(it.g, it.nu, it.nv, it.ntu, it.step, it.views, it.dproj, it.vol_stride, it.acc, it.maxbits,
                         it.bound_mult, it.spv, local / it.ntiles, local % it.ntiles, box, bs, sgmax,
                         gsum);
        __syncthreads();
    }
}

// One work item per CTA (the default launch): the same tile, without the
// work-list loop.
template <int CH, int RPB>
__global__ void __launch_bounds__(RPB, 768 / RPB) k_backproject_batched1(const __grid_constant__ ProjBatch B) {
    extern __shared__ int box[];  // box_words<CH>()
    __shared__ BoxState bs;
    __shared__ unsigned sgmax;
    __shared__ float gsum[RPB / 32];
    for (int i = threadIdx.x; i < box_words<CH>(); i += RPB) box[i] = 0;
    const int64_t w = blockIdx.x;
    const ProjItem it = B.it[find_item(B, w)];
    const int local = (int)(w - it.begin);
    backproject_tile<CH, RPB>(it.g, it.nu, it.nv, it.ntu, it.step, it.views, it.dproj, it.vol_stride, it.acc, it.maxbits,
                     it.bound_mult, it.spv, local / it.ntiles, local % it.ntiles, box, bs, sgmax, gsum);
}

// blockIdx.y = item
__global__ void k_absmax_batched(const __grid_constant__ ProjBatch B) {
    const ProjItem& it = B.it[blockIdx.y];
    absmax_bits(it.dproj, it.nq, it.maxbits);
}

// As k_fixed_to_float_f for every item (blockIdx.y = item); out_max takes the
// maximum over all items.
template <bool MAX>
__global__ void k_fixed_to_float_batched(const __grid_constant__ ProjBatch B, int accumulate, unsigned* out_max) {
    const ProjItem& it = B.it[blockIdx.y];
    const float bound = __uint_as_float(*it.maxbits) * it.bound_mult;
    const int kexp = fixed_exponent(bound);
    const float inv = ldexpf(1.0f, -kexp);
    const bool bad = !isfinite(bound);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) diag_count(PMF_DIAG_NONFINITE);
    unsigned m = 0u;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < it.cells; t += (int64_t)gridDim.x * blockDim.x) {
        const float r = bad ? __int_as_float(0x7fc00000) : from_fixed(it.acc[t], inv);
        const float v = accumulate ? it.dvol[t] + r : r;
        it.dvol[t] = v;
        if (MAX) m = max(m, abs_bits(v));
    }
    if (MAX) block_max_bits(m, out_max);
}

pmf_status backproject_grid(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views,
                            const float* d_proj, float* d_vol, int64_t vol_stride, int accumulate, void* ws,
                            size_t ws_bytes, const MarchShape& sh, cudaStream_t s, unsigned* out_max = nullptr) {
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
        PMF_DISPATCH_ADJOINT(sh, CH, RPB, {
            constexpr int smem = (int)sizeof(int) * box_words<CH>();
            cudaFuncSetAttribute(k_backproject<CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_backproject<CH, RPB><<<gr, RPB, smem, s>>>(g, det->nu, det->nv, ntu, det->step_mm, views, d_proj, vol_stride, acc,
                                                      maxbits, bound_mult, spv);
        });
    }
    int64_t nb = (cells + 255) / 256;
    if (out_max) cudaMemsetAsync(out_max, 0, sizeof(unsigned), s);
    const unsigned ncv = (unsigned)(nb < 4 * kStreamBlocks ? nb : 4 * kStreamBlocks);
    if (((uintptr_t)d_vol & 15) == 0) {
        if (out_max) k_fixed_to_float_f4<true><<<ncv, 256, 0, s>>>(acc, cells, maxbits, bound_mult, d_vol, accumulate, out_max);
        else k_fixed_to_float_f4<false><<<ncv, 256, 0, s>>>(acc, cells, maxbits, bound_mult, d_vol, accumulate, out_max);
    } else {
        if (out_max) k_fixed_to_float_f<true><<<ncv, 256, 0, s>>>(acc, cells, maxbits, bound_mult, d_vol, accumulate, out_max);
        else k_fixed_to_float_f<false><<<ncv, 256, 0, s>>>(acc, cells, maxbits, bound_mult, d_vol, accumulate, out_max);
    }
    return check_launch("conebeam_project_backward");
}

size_t bp_item_bytes(const pmf_backproject_item& it) {
    const int64_t n = (int64_t)it.grid.nx * it.grid.ny * it.grid.nz;
    const int64_t cells = it.vol_stride ? (int64_t)(it.P > 0 ? it.P - 1 : 0) * it.vol_stride + n : n;
    return align_up(256) + align_up(sizeof(unsigned long long) * (size_t)cells);
}

pmf_status backproject_batched_impl(int32_t n, const pmf_backproject_item* items, int accumulate, void* ws,
                                    size_t ws_bytes, const MarchShape& sh, unsigned ctas, cudaStream_t s,
                                    unsigned* out_max = nullptr) {
    size_t need = 0;
    pmf_status st = conebeam_project_backward_batched_workspace(n, items, &need);
    if (st != PMF_OK) return st;
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    ProjBatch B{};
    B.n = n;
    int64_t total = 0, maxq = 0, maxcells = 0;
    char* cur = (char*)ws;
    int ord[kMaxItems];
    longest_first(n, items, ord);  // work-list position k holds item ord[k]
    for (int k = 0; k < n; k++) {
        const pmf_backproject_item& in = items[ord[k]];
        pmf_project_item tmp{in.grid, in.det, in.P, in.views, nullptr, in.vol_stride, nullptr};
        if ((st = fill_item(tmp, total, sh.rays, B.it[k])) != PMF_OK) return st;
        PMF_REQUIRE(in.d_vol != nullptr && (in.P == 0 || in.d_proj != nullptr), "item %d: null pointer", ord[k]);
        ProjItem& it = B.it[k];
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
    if (out_max) cudaMemsetAsync(out_max, 0, sizeof(unsigned), s);
    if (n == 0) return PMF_OK;
    cudaMemsetAsync(ws, 0, need, s);
    if (maxq > 0) {
        const int64_t nb = (maxq + 255) / 256;
        k_absmax_batched<<<dim3((unsigned)(nb < 1024 ? nb : 1024), (unsigned)n), 256, 0, s>>>(B);
    }
    if (total > 0) {
        int ntl[kMaxItems];
        for (int i = 0; i < n; i++) ntl[i] = B.it[i].ntiles;
        const unsigned nc = persistent_ctas(total, ctas, sh.rays, ntl, n);
        PMF_DISPATCH_ADJOINT(sh, CH, RPB, {
            constexpr int smem = (int)sizeof(int) * box_words<CH>();
            if ((int64_t)nc == total) {
                cudaFuncSetAttribute(k_backproject_batched1<CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                k_backproject_batched1<CH, RPB><<<nc, RPB, smem, s>>>(B);
            } else {
                cudaFuncSetAttribute(k_backproject_batched<CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                k_backproject_batched<CH, RPB><<<nc, RPB, smem, s>>>(B);
            }
        });
    }
    const int64_t nc = (maxcells + 255) / 256;
    const dim3 gc((unsigned)(nc < 4 * kStreamBlocks ? nc : 4 * kStreamBlocks), (unsigned)n);
    if (out_max) k_fixed_to_float_batched<true><<<gc, 256, 0, s>>>(B, accumulate, out_max);
    else k_fixed_to_float_batched<false><<<gc, 256, 0, s>>>(B, accumulate, out_max);
    return check_launch("conebeam_project_backward_batched");
}

}  // namespace

PMF_DIAG_ACCESSOR(diag_backproject)

pmf_status backproject_launch(const pmf_backproject_item& it, int accumulate, void* ws, size_t ws_bytes,
                              const MarchShape& sh, cudaStream_t s, unsigned* out_max) {
    if (!valid_shape(sh, true)) return set_error(PMF_EINVAL, "invalid march shape");
    if (sh.form == 0)
        return backproject_grid(&it.grid, &it.det, it.P, it.views, it.d_proj, it.d_vol, it.vol_stride, accumulate,
                                ws, ws_bytes, sh, s, out_max);
    return backproject_batched_impl(1, &it, accumulate, ws, ws_bytes, sh, (unsigned)(sh.form * num_sms()), s, out_max);
}

}  // namespace pmf

using namespace pmf;

extern "C" {

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
    return backproject_grid(grid, det, P, views, d_proj, d_vol, vol_stride, accumulate, ws, ws_bytes,
                            default_backproject_shape(),
                            (cudaStream_t)stream);
}

pmf_status conebeam_project_backward_absmax(const pmf_grid* grid, const pmf_detector* det, int32_t P,
                                            const pmf_view* views, const float* d_proj, float* d_vol,
                                            int64_t vol_stride, int accumulate, void* ws, size_t ws_bytes,
                                            unsigned* d_vol_absmax_bits, pmf_stream stream) {
    PMF_REQUIRE(d_vol_absmax_bits != nullptr, "d_vol_absmax_bits is null");
    return backproject_grid(grid, det, P, views, d_proj, d_vol, vol_stride, accumulate, ws, ws_bytes,
                            default_backproject_shape(), (cudaStream_t)stream, d_vol_absmax_bits);
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
    return backproject_batched_impl(n, items, accumulate, ws, ws_bytes, default_backproject_shape(), 0,
                                    (cudaStream_t)stream);
}
}  // extern "C"
