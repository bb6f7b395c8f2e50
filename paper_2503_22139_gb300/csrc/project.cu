// Cone-beam ray marcher (Eq. 6, source-anchored samples src + m step r, m >= 0),
// its exact adjoint, and the L1/L2 projection loss (Eq. 10/12, Eq. 1) for
// sm_103a.
//
// Precision: the source sits ~1 m from the volume, so a ray's direction and
// start are set up in double precision, then carried as float-float (hi + lo)
// pairs in voxel-index space.  Samples are taken in runs of 32 from an anchor
// whose integer part is exact and whose fraction is float, so every sample
// position is accurate to ~1e-6 voxel while the inner loop is plain fp32.
//
// Threads: one ray per thread; a 256-thread CTA covers a 16x16 pixel tile and
// each warp an 8x4 patch, so the 32 rays of a warp sample neighbouring voxels
// at each step and their gathers share cache lines.
//
// Adjoint: the same march scatters step * dL/dY * (trilinear weights) into a
// 64-bit fixed-point accumulator (scale 2^k chosen per call from a provable
// bound), merging consecutive samples that fall in the same cell before each
// atomic.  Integer atomics are order independent, so the result is
// bit-reproducible.
#include <climits>

#include "pmf_common.cuh"

namespace pmf {
namespace {

constexpr int kRay = 256;  // threads per CTA (16 x 16 pixels)
constexpr int kRun = 32;   // samples per float anchor

struct RayMarch {
    int nsamp;       // number of samples (0: the ray misses the padded volume)
    float hi[3];     // index-space position of the first sample, float-float
    float lo[3];
    float dhi[3];    // index-space step, float-float
    float dlo[3];
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Pixel (a, b) of `view`: direction, sample range and float-float start.
__device__ __forceinline__ RayMarch ray_setup(const pmf_view& vw, int nu, int nv, int a, int b, const GridD& g,
                                              double step) {
    RayMarch r;
    const double ca = (double)a + 0.5 - 0.5 * (double)nu, cb = (double)b + 0.5 - 0.5 * (double)nv;
    double d[3];
    double len2 = 0.0;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        d[t] = fma(cb, vw.dv[t], fma(ca, vw.du[t], vw.det[t] - vw.src[t]));
        len2 = fma(d[t], d[t], len2);
    }
    // 1/sqrt(len2): fp32 seed, two Newton steps in double (~1e-16 relative)
    double y = (double)rsqrtf((float)len2);
    y = y * (1.5 - 0.5 * len2 * y * y);
    y = y * (1.5 - 0.5 * len2 * y * y);
    const int n[3] = {g.nx, g.ny, g.nz};
    const double iv[3] = {1.0 / (double)g.vx, 1.0 / (double)g.vy, 1.0 / (double)g.vz};
    double us[3], du[3];
    float tlo = 0.0f, thi = 3.0e38f;
    bool miss = false;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        us[t] = fma(vw.src[t], iv[t], 0.5 * (double)n[t] - 0.5);
        du[t] = step * (d[t] * y) * iv[t];
        const float usf = (float)us[t], duf = (float)du[t];
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
        r.nsamp = 0;
    } else {
        r.nsamp = (int)(mhi - mlo) + 1;
    }
    const double m0 = (double)mlo;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const double u0 = fma(m0, du[t], us[t]);
        r.hi[t] = (float)u0;
        r.lo[t] = (float)(u0 - (double)r.hi[t]);
        r.dhi[t] = (float)du[t];
        r.dlo[t] = (float)(du[t] - (double)r.dhi[t]);
    }
    return r;
}

// Advance the float-float start by kRun steps (exact up to the lo word).
__device__ __forceinline__ void advance(RayMarch& r) {
#pragma unroll
    for (int t = 0; t < 3; t++) {
        float s, e;
        two_sum(r.hi[t], (float)kRun * r.dhi[t], s, e);
        float lo = r.lo[t] + (float)kRun * r.dlo[t] + e;
        float s2 = s + lo;
        r.lo[t] = lo - (s2 - s);
        r.hi[t] = s2;
    }
}

__device__ __forceinline__ void pixel_of(int tile, int ntu, int& a, int& b) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int tu = tile % ntu, tv = tile / ntu;
    a = tu * 16 + (w & 1) * 8 + (l & 7);
    b = tv * 16 + (w >> 1) * 4 + (l >> 3);
}

template <typename T>
__device__ __forceinline__ float gather8(const T* vol, const GridD& g, int ix, int iy, int iz, float fx, float fy,
                                         float fz) {
    // interior cells skip the per-corner bounds checks
    if ((unsigned)ix < (unsigned)(g.nx - 1) && (unsigned)iy < (unsigned)(g.ny - 1) &&
        (unsigned)iz < (unsigned)(g.nz - 1)) {
        const int64_t sx = 1, sy = g.nx, sz = (int64_t)g.nx * g.ny;
        const T* p = vol + iz * sz + iy * sy + ix;
        const float c000 = Store<T>::ld(p, 0), c100 = Store<T>::ld(p, sx);
        const float c010 = Store<T>::ld(p, sy), c110 = Store<T>::ld(p, sy + sx);
        const float c001 = Store<T>::ld(p, sz), c101 = Store<T>::ld(p, sz + sx);
        const float c011 = Store<T>::ld(p, sz + sy), c111 = Store<T>::ld(p, sz + sy + sx);
        const float a00 = fmaf(fx, c100 - c000, c000), a10 = fmaf(fx, c110 - c010, c010);
        const float a01 = fmaf(fx, c101 - c001, c001), a11 = fmaf(fx, c111 - c011, c011);
        const float b0 = fmaf(fy, a10 - a00, a00), b1 = fmaf(fy, a11 - a01, a01);
        return fmaf(fz, b1 - b0, b0);
    }
    return trilin_cell(vol, g, ix, iy, iz, fx, fy, fz);
}

template <typename T>
__global__ void __launch_bounds__(kRay) k_project(GridD g, int nu, int nv, int ntu, float step,
                                                  const pmf_view* __restrict__ views, const T* __restrict__ vol,
                                                  int64_t vol_stride, float* __restrict__ proj) {
    const int p = blockIdx.y;
    int a, b;
    pixel_of(blockIdx.x, ntu, a, b);
    if (a >= nu || b >= nv) return;
    const pmf_view vw = views[p];
    RayMarch r = ray_setup(vw, nu, nv, a, b, g, (double)step);
    const T* V = vol + (int64_t)p * vol_stride;
    float acc = 0.0f;
    for (int jb = 0; jb < r.nsamp; jb += kRun) {
        int ib[3];
        float fb[3];
#pragma unroll
        for (int t = 0; t < 3; t++) {
            const float fl = floorf(r.hi[t]);
            ib[t] = (int)fl;
            fb[t] = (r.hi[t] - fl) + r.lo[t];
        }
        const int jn = min(kRun, r.nsamp - jb);
        for (int j = 0; j < jn; j++) {
            const float jf = (float)j;
            const float ux = fmaf(jf, r.dhi[0], fmaf(jf, r.dlo[0], fb[0]));
            const float uy = fmaf(jf, r.dhi[1], fmaf(jf, r.dlo[1], fb[1]));
            const float uz = fmaf(jf, r.dhi[2], fmaf(jf, r.dlo[2], fb[2]));
            const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
            acc += gather8(V, g, ib[0] + (int)flx, ib[1] + (int)fly, ib[2] + (int)flz, ux - flx, uy - fly, uz - flz);
        }
        advance(r);
    }
    proj[((int64_t)p * nv + b) * nu + a] = step * acc;
}

__global__ void k_absmax_f(const float* __restrict__ x, int64_t n, unsigned* out) {
    float m = 0.f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(__ldg(x + t)));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// Scatter the 8 corner weights of one cell times g.
__device__ __forceinline__ void flush_cell(unsigned long long* acc, const GridD& g, int ix, int iy, int iz,
                                           const float* w, float gs) {
#pragma unroll
    for (int c = 0; c < 8; c++) {
        if (w[c] == 0.0f) continue;
        const int i = ix + (c & 1), j = iy + ((c >> 1) & 1), k = iz + (c >> 2);
        if ((unsigned)i >= (unsigned)g.nx || (unsigned)j >= (unsigned)g.ny || (unsigned)k >= (unsigned)g.nz) continue;
        red_add(acc + ((int64_t)k * g.ny + j) * g.nx + i, to_fixed(w[c] * gs, 1.0f));
    }
}

__global__ void __launch_bounds__(kRay) k_backproject(GridD g, int nu, int nv, int ntu, float step,
                                                      const pmf_view* __restrict__ views,
                                                      const float* __restrict__ dproj, int64_t vol_stride,
                                                      unsigned long long* __restrict__ acc, const unsigned* maxbits,
                                                      float bound_mult) {
    const int p = blockIdx.y;
    int a, b;
    pixel_of(blockIdx.x, ntu, a, b);
    if (a >= nu || b >= nv) return;
    const float gy = __ldg(dproj + ((int64_t)p * nv + b) * nu + a);
    if (gy == 0.0f) return;
    const int kexp = fixed_exponent(__uint_as_float(*maxbits) * bound_mult);
    const float gs = step * gy * ldexpf(1.0f, kexp);  // scaled contribution per unit weight
    const pmf_view vw = views[p];
    RayMarch r = ray_setup(vw, nu, nv, a, b, g, (double)step);
    unsigned long long* A = acc + (int64_t)p * vol_stride;
    int cx = INT_MIN, cy = 0, cz = 0;
    float w[8];
#pragma unroll
    for (int c = 0; c < 8; c++) w[c] = 0.0f;
    for (int jb = 0; jb < r.nsamp; jb += kRun) {
        int ib[3];
        float fb[3];
#pragma unroll
        for (int t = 0; t < 3; t++) {
            const float fl = floorf(r.hi[t]);
            ib[t] = (int)fl;
            fb[t] = (r.hi[t] - fl) + r.lo[t];
        }
        const int jn = min(kRun, r.nsamp - jb);
        for (int j = 0; j < jn; j++) {
            const float jf = (float)j;
            const float ux = fmaf(jf, r.dhi[0], fmaf(jf, r.dlo[0], fb[0]));
            const float uy = fmaf(jf, r.dhi[1], fmaf(jf, r.dlo[1], fb[1]));
            const float uz = fmaf(jf, r.dhi[2], fmaf(jf, r.dlo[2], fb[2]));
            const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
            const int ix = ib[0] + (int)flx, iy = ib[1] + (int)fly, iz = ib[2] + (int)flz;
            const float fx = ux - flx, fy = uy - fly, fz = uz - flz;
            if (ix != cx || iy != cy || iz != cz) {
                if (cx != INT_MIN) flush_cell(A, g, cx, cy, cz, w, gs);
                cx = ix; cy = iy; cz = iz;
#pragma unroll
                for (int c = 0; c < 8; c++) w[c] = 0.0f;
            }
            const float ex = 1.0f - fx, ey = 1.0f - fy, ez = 1.0f - fz;
            w[0] += ex * ey * ez; w[1] += fx * ey * ez; w[2] += ex * fy * ez; w[3] += fx * fy * ez;
            w[4] += ex * ey * fz; w[5] += fx * ey * fz; w[6] += ex * fy * fz; w[7] += fx * fy * fz;
        }
        advance(r);
    }
    if (cx != INT_MIN) flush_cell(A, g, cx, cy, cz, w, gs);
}

__global__ void k_fixed_to_float_f(const unsigned long long* __restrict__ acc, int64_t n, const unsigned* maxbits,
                                   float bound_mult, float* out, int accumulate) {
    const float bound = __uint_as_float(*maxbits) * bound_mult;
    const int kexp = fixed_exponent(bound);
    const float inv = ldexpf(1.0f, -kexp);
    const bool bad = !isfinite(bound);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float r = bad ? __int_as_float(0x7fc00000) : from_fixed(acc[t], inv);
        out[t] = accumulate ? out[t] + r : r;
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

int max_samples_per_voxel(const pmf_grid* grid, float step) {
    // a ray crosses the open 2x2x2-voxel support of one voxel over at most its
    // diagonal, 2 |v|, so it takes at most floor(2|v| / step) + 1 samples there
    const double diag = 2.0 * sqrt((double)grid->vx * grid->vx + (double)grid->vy * grid->vy + (double)grid->vz * grid->vz);
    return (int)floor(diag / (double)step) + 1;
}

}  // namespace
}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status conebeam_project(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views,
                            pmf_dtype dtype, const void* vol, int64_t vol_stride, float* proj, pmf_stream stream) {
    pmf_status st = check_proj(grid, det, P, views);
    if (st != PMF_OK) return st;
    if ((st = validate_dtype(dtype)) != PMF_OK) return st;
    if (P == 0) return PMF_OK;
    PMF_REQUIRE(vol && proj, "null pointer");
    PMF_REQUIRE(vol_stride >= 0, "vol_stride must be >= 0");
    GridD g = make_grid(grid);
    const int ntu = (det->nu + 15) / 16, ntv = (det->nv + 15) / 16;
    dim3 gr((unsigned)(ntu * ntv), (unsigned)P);
    cudaStream_t s = (cudaStream_t)stream;
    PMF_DISPATCH_DTYPE(dtype, T, k_project<T><<<gr, kRay, 0, s>>>(g, det->nu, det->nv, ntu, det->step_mm, views, (const T*)vol, vol_stride, proj));
    return check_launch("conebeam_project");
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
    pmf_status st = check_proj(grid, det, P, views);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(vol_stride >= 0, "vol_stride must be >= 0");
    PMF_REQUIRE(d_vol != nullptr && (P == 0 || d_proj != nullptr), "null pointer");
    size_t need;
    conebeam_project_backward_workspace(grid, P, vol_stride, &need);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
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
        const int ntu = (det->nu + 15) / 16, ntv = (det->nv + 15) / 16;
        dim3 gr((unsigned)(ntu * ntv), (unsigned)P);
        k_backproject<<<gr, kRay, 0, s>>>(g, det->nu, det->nv, ntu, det->step_mm, views, d_proj, vol_stride, acc,
                                          maxbits, bound_mult);
    }
    int64_t nb = (cells + 255) / 256;
    k_fixed_to_float_f<<<(unsigned)(nb < 4 * kStreamBlocks ? nb : 4 * kStreamBlocks), 256, 0, s>>>(
        acc, cells, maxbits, bound_mult, d_vol, accumulate);
    return check_launch("conebeam_project_backward");
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
