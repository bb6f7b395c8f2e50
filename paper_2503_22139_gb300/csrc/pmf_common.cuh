// Shared device helpers for the PMF-STGR sm_103a kernels: storage-type loads
// and stores, grid geometry, zero-padded trilinear interpolation, 64-bit fixed
// point for reproducible scatters, and host-side status plumbing.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pmf.h"

namespace pmf {

// ------------------------------------------------------------ host status

pmf_status set_error(pmf_status st, const char* fmt, ...);
pmf_status check_launch(const char* what);

#define PMF_REQUIRE(cond, ...)                                 \
    do {                                                       \
        if (!(cond)) return ::pmf::set_error(PMF_EINVAL, __VA_ARGS__); \
    } while (0)

pmf_status validate_grid(const pmf_grid* g);
pmf_status validate_dtype(pmf_dtype dt);
pmf_status validate_ws(const void* ws, size_t ws_bytes, size_t need);

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Fixed launch width for grid-stride kernels whose reductions must not depend
// on the device: 4 x 152 SMs.
constexpr int kStreamBlocks = 608;

// ---------------------------------------------------- device diagnostics
//
// Counters of the slow paths and of non-finite scatter inputs (pmf_diag).
// Every translation unit that includes this header has its own array;
// pmf_device_counters adds them up through the accessors below.
static __device__ unsigned long long g_diag[PMF_DIAG_COUNT];

__device__ __forceinline__ void diag_count(int which) { atomicAdd(&g_diag[which], 1ull); }

// Bounds checks of the debug build (compiled with -DPMF_DEBUG): PMF_DCHECK(ok)
// is `ok`, and a false check counts PMF_DIAG_BOUNDS, so the caller skips the
// access instead of faulting; in the normal build it is the constant true and
// compiles away.  Used at the shared-memory box and list indices.
#ifdef PMF_DEBUG
__device__ __forceinline__ bool debug_check(bool ok) {
    if (!ok) diag_count(PMF_DIAG_BOUNDS);
    return ok;
}
#define PMF_DCHECK(cond) (::pmf::debug_check(cond))
#else
#define PMF_DCHECK(cond) true
#endif

#define PMF_DIAG_ACCESSOR(fn)                                                                     \
    pmf_status fn(unsigned long long* out, int reset) {                                           \
        unsigned long long v[PMF_DIAG_COUNT];                                                     \
        cudaError_t e = cudaMemcpyFromSymbol(v, g_diag, sizeof(v));                               \
        if (e == cudaSuccess && reset) {                                                          \
            const unsigned long long z[PMF_DIAG_COUNT] = {};                                      \
            e = cudaMemcpyToSymbol(g_diag, z, sizeof(z));                                         \
        }                                                                                         \
        if (e != cudaSuccess) return ::pmf::set_error(PMF_ECUDA, #fn ": %s", cudaGetErrorString(e)); \
        for (int i = 0; i < PMF_DIAG_COUNT; i++) out[i] += v[i];                                  \
        return PMF_OK;                                                                            \
    }

pmf_status diag_voxelize(unsigned long long* out, int reset);
pmf_status diag_project(unsigned long long* out, int reset);
pmf_status diag_warp(unsigned long long* out, int reset);
pmf_status diag_backproject(unsigned long long* out, int reset);
pmf_status diag_splat(unsigned long long* out, int reset);

// Launch shape of the ray marchers used by plans: form 0 is one CTA per
// (view, pixel tile), k > 0 a persistent launch of k CTAs per SM; chunk (16,
// 32 or 48, and for the adjoint also 64) is the number of samples per staged
// brick along the rays and rays (128 or 256) the rays per CTA.  Forms give identical results; chunk and rays
// move the last bits (anchors, per-CTA fixed-point scale).
struct MarchShape {
    int form = 0;
    int chunk = 32;
    int rays = 256;
    int tma = 1;  // forward only: 1 stages fp32 boxes with bulk tensor copies when the layout allows, 0 never
};
// The adjoint's default: 128 rays per CTA (a 16x8 pixel tile), whose rays have
// closer sample ranges, so fewer lanes idle at the chunks where rays enter or
// leave the volume, and 48-sample chunks, which halve the per-chunk work (box
// set-up, barriers and the flush) against 32 while six CTAs of 128 still fit
// an SM (measured at the paper-scale geometry: 7.87 -> 7.02 ms per 32 views;
// 40 samples 7.59, 56 samples 7.23, 64 samples 7.70 at four CTAs per SM).
// A launch shape the marchers take: the projector's chunks are 16, 32 or 48
// samples, the adjoint's may also be 64.
inline bool valid_march_shape(const MarchShape& sh, bool adjoint) {
    const bool chunk = sh.chunk == 16 || sh.chunk == 32 || sh.chunk == 48 || (adjoint && sh.chunk == 64);
    return chunk && (sh.rays == 128 || sh.rays == 256) && sh.form >= 0 && sh.form <= 16;
}
// The projector's default: 256 rays per CTA and 48-sample chunks, staged by
// bulk copies into a 52 KB box (measured at the paper-scale geometry: 4.05 ->
// 3.69 ms per 32 views, the 32-sample chunks' 32 KB box also overflowing at
// some view angles; 40 samples 3.78, 56 samples 3.74).
inline MarchShape default_project_shape() {
    MarchShape m;
    m.chunk = 48;
    return m;
}
inline MarchShape default_backproject_shape() {
    MarchShape m;
    m.chunk = 48;
    m.rays = 128;
    return m;
}
pmf_status project_launch(const pmf_project_item& it, pmf_dtype dtype, const MarchShape& sh, cudaStream_t s);
// out_max (optional, device): receives max |d_vol| as abs_bits (see
// conebeam_project_backward_absmax).
pmf_status backproject_launch(const pmf_backproject_item& it, int accumulate, void* ws, size_t ws_bytes,
                              const MarchShape& sh, cudaStream_t s, unsigned* out_max = nullptr);

// ------------------------------------------------------- storage dtypes

template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p, int64_t i) { return __ldg(p + i); }
    static __device__ __forceinline__ void st(float* p, int64_t i, float v) { p[i] = v; }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, int64_t i) {
        return __bfloat162float(__ldg(p + i));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, int64_t i, float v) { p[i] = __float2bfloat16_rn(v); }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p, int64_t i) { return __half2float(__ldg(p + i)); }
    static __device__ __forceinline__ void st(__half* p, int64_t i, float v) { p[i] = __float2half_rn(v); }
};

#define PMF_DISPATCH_DTYPE(dt, T, ...)                          \
    switch (dt) {                                               \
        case PMF_F32: { using T = float; __VA_ARGS__; break; }  \
        case PMF_BF16: { using T = __nv_bfloat16; __VA_ARGS__; break; } \
        case PMF_F16: { using T = __half; __VA_ARGS__; break; } \
        default: return ::pmf::set_error(PMF_EINVAL, "unknown dtype %d", (int)dt); \
    }

// ------------------------------------------------------------- geometry

struct GridD {
    int nx, ny, nz;
    float vx, vy, vz;       // voxel size, mm
    float ivx, ivy, ivz;    // 1 / voxel size
    int64_t n;
};

inline GridD make_grid(const pmf_grid* g) {
    GridD d;
    d.nx = g->nx; d.ny = g->ny; d.nz = g->nz;
    d.vx = g->vx; d.vy = g->vy; d.vz = g->vz;
    d.ivx = 1.0f / g->vx; d.ivy = 1.0f / g->vy; d.ivz = 1.0f / g->vz;
    d.n = (int64_t)g->nx * g->ny * g->nz;
    return d;
}

// ---------------------------------------------------- trilinear helpers

// Value of vol at integer (i,j,k), zero outside the grid.
template <typename T>
__device__ __forceinline__ float vox_or_zero(const T* vol, const GridD& g, int i, int j, int k) {
    bool in = (unsigned)i < (unsigned)g.nx && (unsigned)j < (unsigned)g.ny && (unsigned)k < (unsigned)g.nz;
    return in ? Store<T>::ld(vol, ((int64_t)k * g.ny + j) * g.nx + i) : 0.0f;
}

// The 8 corners of cell (i0,j0,k0), c[dx + 2 dy + 4 dz], zero outside the
// grid.  Cells with all corners inside (nearly all) take one bounds test and
// one base address; the values are the same either way.
template <typename T>
__device__ __forceinline__ void corners8(const T* vol, const GridD& g, int i0, int j0, int k0, float c[8]) {
    if ((unsigned)i0 < (unsigned)(g.nx - 1) && (unsigned)j0 < (unsigned)(g.ny - 1) &&
        (unsigned)k0 < (unsigned)(g.nz - 1)) {
        const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
        const T* p = vol + ((int64_t)k0 * g.ny + j0) * g.nx + i0;
        c[0] = Store<T>::ld(p, 0); c[1] = Store<T>::ld(p, 1);
        c[2] = Store<T>::ld(p, sy); c[3] = Store<T>::ld(p, sy + 1);
        c[4] = Store<T>::ld(p, sz); c[5] = Store<T>::ld(p, sz + 1);
        c[6] = Store<T>::ld(p, sz + sy); c[7] = Store<T>::ld(p, sz + sy + 1);
    } else {
#pragma unroll
        for (int q = 0; q < 8; q++) c[q] = vox_or_zero(vol, g, i0 + (q & 1), j0 + ((q >> 1) & 1), k0 + (q >> 2));
    }
}

// Trilinear blend of 8 corners c[dx + 2 dy + 4 dz] with fractions f.
__device__ __forceinline__ float trilin8(const float c[8], float fx, float fy, float fz) {
    const float c000 = c[0], c100 = c[1], c010 = c[2], c110 = c[3], c001 = c[4], c101 = c[5], c011 = c[6],
                c111 = c[7];
    float a00 = fmaf(fx, c100 - c000, c000), a10 = fmaf(fx, c110 - c010, c010);
    float a01 = fmaf(fx, c101 - c001, c001), a11 = fmaf(fx, c111 - c011, c011);
    float b0 = fmaf(fy, a10 - a00, a00), b1 = fmaf(fy, a11 - a01, a01);
    return fmaf(fz, b1 - b0, b0);
}

// Zero-padded trilinear interpolation at cell (i0,j0,k0) with fractions f.
template <typename T>
__device__ __forceinline__ float trilin_cell(const T* vol, const GridD& g, int i0, int j0, int k0, float fx,
                                             float fy, float fz) {
    float c[8];
    corners8(vol, g, i0, j0, k0, c);
    return trilin8(c, fx, fy, fz);
}

// Split a small offset t (in voxels) into floor and fraction exactly.
__device__ __forceinline__ void split_offset(float t, int& fl, float& f) {
    float ft = floorf(t);
    fl = (int)ft;
    f = t - ft;
}

// ------------------------------------------------- packed fp32 pairs
// sm_100+ executes add/sub/mul/fma on two fp32 values held in a 64-bit register
// pair as one instruction.  Each half is the ordinary IEEE round-to-nearest
// fp32 operation, so a packed form gives the scalar form's bits.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo2(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi2(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ------------------------------------------------------- fixed point
//
// Reproducible scatter: every contribution is rounded to an integer multiple of
// 2^-e and added with 64-bit integer atomics, which are order independent.
// e is chosen per call so that `bound` (a provable bound on the magnitude of
// any accumulated sum) stays below 2^62.

__device__ __forceinline__ int fixed_exponent(float bound) {
    if (!(bound > 0.0f) || !isfinite(bound)) return 0;
    int e;
    frexpf(bound, &e);  // bound < 2^e
    int k = 62 - e;
    return k > 126 ? 126 : (k < -126 ? -126 : k);
}

__device__ __forceinline__ unsigned long long to_fixed(float x, float scale) {
    return (unsigned long long)__float2ll_rn(x * scale);
}

__device__ __forceinline__ float from_fixed(unsigned long long a, float inv_scale) {
    return __ll2float_rn((long long)a) * inv_scale;
}

__device__ __forceinline__ void red_add(unsigned long long* p, unsigned long long v) {
    if (v) atomicAdd(p, v);
}

// Non-negative float max via the order-preserving bit pattern.
// |x| as ordered bits: for non-negative floats the unsigned order of the bit
// patterns is the numeric order, and +inf and every NaN sort above all finite
// values, so a maximum over these bits keeps a NaN or infinity visible (fmaxf
// would drop a NaN).
__device__ __forceinline__ unsigned abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

// Grid-stride maximum of |x[0..n)| into *out as abs_bits (every thread of the
// launch calls it; blocks are whole warps).
__device__ __forceinline__ void absmax_bits(const float* __restrict__ x, int64_t n, unsigned* out) {
    unsigned m = 0u;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        m = max(m, abs_bits(__ldg(x + t)));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// Block-wide maximum of the threads' m (abs bits) into *out: one atomic per
// block, skipped when *out already holds at least the block's value (*out
// only grows, so a stale read only costs an atomic).  Same-address atomics
// from every warp of a large grid serialise in L2.  Every thread of the block
// calls it; blocks are whole warps.
__device__ __forceinline__ void block_max_bits(unsigned m, unsigned* out) {
    __shared__ unsigned wmax[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (int)(blockDim.x + 31) >> 5;
    m = __reduce_max_sync(0xffffffffu, m);
    if (l == 0) wmax[w] = m;
    __syncthreads();
    if (w == 0) {
        m = __reduce_max_sync(0xffffffffu, l < nw ? wmax[l] : 0u);
        if (l == 0 && m > *(volatile unsigned*)out) atomicMax(out, m);
    }
}

// --------------------------------------------------- block reductions

template <int NT>
__device__ __forceinline__ float block_sum(float v, float* smem) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem[w] = v;
    __syncthreads();
    float r = 0.0f;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; i++) r += smem[i];
    }
    return r;  // valid in thread 0
}

}  // namespace pmf
