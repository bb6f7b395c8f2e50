// DVF combine (Eq. 3), pull warp (Eq. 2), their fusion, and the adjoints, for
// sm_103a.  All streaming kernels are grid-stride loops over voxels with a fixed
// grid (so reductions do not depend on the device); coefficient tables are read
// through the read-only cache as warp-uniform broadcasts.
//
// Reproducibility: the warp transpose scatters into d_ref with 64-bit
// fixed-point atomics (scale chosen from max |d_out| * P * N < 2^62); the
// coefficient gradients are block partials reduced in a fixed order.
#include "pmf_common.cuh"

namespace pmf {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxL = 8;

// Corner weights of a trilinear cell and their derivatives with respect to
// the fractional position.
struct Cell {
    int i0, j0, k0;
    float fx, fy, fz;
};

__device__ __forceinline__ Cell make_cell(int i, int j, int k, float tx, float ty, float tz) {
    Cell c;
    int ox, oy, oz;
    split_offset(tx, ox, c.fx);
    split_offset(ty, oy, c.fy);
    split_offset(tz, oz, c.fz);
    c.i0 = i + ox; c.j0 = j + oy; c.k0 = k + oz;
    return c;
}

// Trilinear value and gradient (with respect to the continuous index) from
// the 8 corners of a cell.
__device__ __forceinline__ float trilin8_grad(const float cv[8], const Cell& c, float& gx, float& gy, float& gz) {
    const float v000 = cv[0], v100 = cv[1], v010 = cv[2], v110 = cv[3], v001 = cv[4], v101 = cv[5], v011 = cv[6],
                v111 = cv[7];
    float a00 = fmaf(c.fx, v100 - v000, v000), a10 = fmaf(c.fx, v110 - v010, v010);
    float a01 = fmaf(c.fx, v101 - v001, v001), a11 = fmaf(c.fx, v111 - v011, v011);
    float b0 = fmaf(c.fy, a10 - a00, a00), b1 = fmaf(c.fy, a11 - a01, a01);
    gz = b1 - b0;
    gy = fmaf(c.fz, (a11 - a01) - (a10 - a00), a10 - a00);
    float ex0 = fmaf(c.fy, (v110 - v010) - (v100 - v000), v100 - v000);
    float ex1 = fmaf(c.fy, (v111 - v011) - (v101 - v001), v101 - v001);
    gx = fmaf(c.fz, ex1 - ex0, ex0);
    return fmaf(c.fz, b1 - b0, b0);
}

// The same at a cell of vol, zero padding outside the grid.
template <typename T>
__device__ __forceinline__ float trilin_grad(const T* vol, const GridD& g, const Cell& c, float& gx, float& gy,
                                             float& gz) {
    float cv[8];
    corners8(vol, g, c.i0, c.j0, c.k0, cv);
    return trilin8_grad(cv, c, gx, gy, gz);
}

__device__ __forceinline__ void scatter_cell(unsigned long long* acc, const GridD& g, const Cell& c, float val,
                                             float scale) {
    const float wx[2] = {1.f - c.fx, c.fx}, wy[2] = {1.f - c.fy, c.fy}, wz[2] = {1.f - c.fz, c.fz};
#pragma unroll
    for (int dz = 0; dz < 2; dz++) {
        const int k = c.k0 + dz;
        if ((unsigned)k >= (unsigned)g.nz) continue;
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const int j = c.j0 + dy;
            if ((unsigned)j >= (unsigned)g.ny) continue;
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const int i = c.i0 + dx;
                if ((unsigned)i >= (unsigned)g.nx) continue;
                const float w = wx[dx] * wy[dy] * wz[dz];
                red_add(acc + ((int64_t)k * g.ny + j) * g.nx + i, to_fixed(val * w, scale));
            }
        }
    }
}

__device__ __forceinline__ void voxel_ijk(int64_t v, const GridD& g, int& i, int& j, int& k) {
    i = (int)(v % g.nx);
    int64_t r = v / g.nx;
    j = (int)(r % g.ny);
    k = (int)(r / g.ny);
}

// ----------------------------------------------------------- combine

template <typename T>
__global__ void __launch_bounds__(kThreads) k_combine(GridD g, int L, int P, const T* __restrict__ E,
                                                      const float* __restrict__ w, T* __restrict__ D) {
    const int64_t N = g.n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        float e[kMaxL][3];
        for (int l = 0; l < L; l++)
#pragma unroll
            for (int k = 0; k < 3; k++) e[l][k] = Store<T>::ld(E, ((int64_t)l * 3 + k) * N + v);
        for (int p = 0; p < P; p++) {
#pragma unroll
            for (int k = 0; k < 3; k++) {
                float acc = 0.f;
                for (int l = 0; l < L; l++) acc = fmaf(__ldg(w + (p * L + l) * 3 + k), e[l][k], acc);
                Store<T>::st(D, ((int64_t)p * 3 + k) * N + v, acc);
            }
        }
    }
}

// d_mbc[l][k][v] = sum_p d_dvf[p][k][v] coeff[p][l][k]
__global__ void __launch_bounds__(kThreads) k_combine_bwd_mbc(GridD g, int L, int P, const float* __restrict__ w,
                                                              const float* __restrict__ dD, float* dE, int accumulate) {
    const int64_t N = g.n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        for (int l = 0; l < L; l++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                float acc = 0.f;
                for (int p = 0; p < P; p++) acc = fmaf(__ldg(dD + ((int64_t)p * 3 + k) * N + v), __ldg(w + (p * L + l) * 3 + k), acc);
                const int64_t o = ((int64_t)l * 3 + k) * N + v;
                dE[o] = accumulate ? dE[o] + acc : acc;
            }
    }
}

// Block partials of d_coeff[p][l][k] = sum_v d_dvf[p][k][v] mbc[l][k][v]:
// gridDim.y = P*3 (one (p,k) per y), gridDim.x = fixed voxel split.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_combine_bwd_coeff(GridD g, int L, int P, const T* __restrict__ E,
                                                                const float* __restrict__ dD, float* part) {
    __shared__ float red[kThreads / 32][kMaxL];
    const int64_t N = g.n;
    const int pk = blockIdx.y, p = pk / 3, k = pk % 3;
    float acc[kMaxL];
    for (int l = 0; l < kMaxL; l++) acc[l] = 0.f;
    const float* d = dD + ((int64_t)p * 3 + k) * N;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const float dv = __ldg(d + v);
        for (int l = 0; l < L; l++) acc[l] = fmaf(dv, Store<T>::ld(E, ((int64_t)l * 3 + k) * N + v), acc[l]);
    }
    for (int l = 0; l < L; l++) {
        float r = acc[l];
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][l] = r;
    }
    __syncthreads();
    if (threadIdx.x < L) {
        float r = 0.f;
        for (int wi = 0; wi < kThreads / 32; wi++) r += red[wi][threadIdx.x];
        // part[(p*L + l)*3 + k][block]
        part[(((int64_t)p * L + threadIdx.x) * 3 + k) * gridDim.x + blockIdx.x] = r;
    }
}

// Sum `nb` block partials per output in index order (double accumulator).
__global__ void k_reduce_partials(const float* part, int64_t nout, int nb, float* out, int accumulate) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    double r = 0.0;
    for (int b = 0; b < nb; b++) r += (double)part[o * nb + b];
    out[o] = accumulate ? out[o] + (float)r : (float)r;
}

// --------------------------------------------------------------- warp

template <typename T>
__global__ void __launch_bounds__(kThreads) k_warp(GridD g, int P, const T* __restrict__ ref, const T* __restrict__ D,
                                                   T* __restrict__ W) {
    const int64_t N = g.n, total = N * P;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / N, v = t - p * N;
        int i, j, k;
        voxel_ijk(v, g, i, j, k);
        const T* Dp = D + p * 3 * N;
        const Cell c = make_cell(i, j, k, Store<T>::ld(Dp, v) * g.ivx, Store<T>::ld(Dp, N + v) * g.ivy,
                                 Store<T>::ld(Dp, 2 * N + v) * g.ivz);
        Store<T>::st(W, t, trilin_cell(ref, g, c.i0, c.j0, c.k0, c.fx, c.fy, c.fz));
    }
}

__global__ void k_absmax(const float* __restrict__ x, int64_t n, unsigned* out) { absmax_bits(x, n, out); }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_warp_bwd(GridD g, int P, const T* __restrict__ ref,
                                                       const T* __restrict__ D, const float* __restrict__ dW,
                                                       float* d_dvf, unsigned long long* acc, const unsigned* maxbits,
                                                       int accumulate) {
    const int64_t N = g.n, total = N * P;
    const int kexp = fixed_exponent(__uint_as_float(*maxbits) * (float)total);
    const float scale = ldexpf(1.0f, kexp);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / N, v = t - p * N;
        int i, j, k;
        voxel_ijk(v, g, i, j, k);
        const T* Dp = D + p * 3 * N;
        const Cell c = make_cell(i, j, k, Store<T>::ld(Dp, v) * g.ivx, Store<T>::ld(Dp, N + v) * g.ivy,
                                 Store<T>::ld(Dp, 2 * N + v) * g.ivz);
        const float gw = __ldg(dW + t);
        if (d_dvf) {
            float gx, gy, gz;
            trilin_grad(ref, g, c, gx, gy, gz);
            float* o = d_dvf + p * 3 * N + v;
            const float r0 = gw * gx * g.ivx, r1 = gw * gy * g.ivy, r2 = gw * gz * g.ivz;
            o[0] = accumulate ? o[0] + r0 : r0;
            o[N] = accumulate ? o[N] + r1 : r1;
            o[2 * N] = accumulate ? o[2 * N] + r2 : r2;
        }
        if (gw != 0.f) scatter_cell(acc, g, c, gw, scale);
    }
}

// d_ref (=/+=) fixed-point accumulator * 2^-k, k from the same bound.
__global__ void k_fixed_to_float(const unsigned long long* __restrict__ acc, int64_t n, const unsigned* maxbits,
                                 float bound_mult, float* out, int accumulate) {
    const float bound = __uint_as_float(*maxbits) * bound_mult;
    const int kexp = fixed_exponent(bound);
    const float inv = ldexpf(1.0f, -kexp);
    const bool bad = !isfinite(bound);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) diag_count(PMF_DIAG_NONFINITE);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float r = bad ? __int_as_float(0x7fc00000) : from_fixed(acc[t], inv);
        out[t] = accumulate ? out[t] + r : r;
    }
}

// ----------------------------------------------------- fused combine + warp

template <typename T, typename TO>
__global__ void __launch_bounds__(kThreads) k_warp_combine(GridD g, int L, int P, const T* __restrict__ ref,
                                                           const T* __restrict__ E, const float* __restrict__ w,
                                                           TO* __restrict__ W) {
    const int64_t N = g.n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        voxel_ijk(v, g, i, j, k);
        float e[kMaxL][3];
        for (int l = 0; l < L; l++)
#pragma unroll
            for (int a = 0; a < 3; a++) e[l][a] = Store<T>::ld(E, ((int64_t)l * 3 + a) * N + v);
        for (int p = 0; p < P; p++) {
            float d[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                float acc = 0.f;
                for (int l = 0; l < L; l++) acc = fmaf(__ldg(w + (p * L + l) * 3 + a), e[l][a], acc);
                d[a] = acc;
            }
            const Cell c = make_cell(i, j, k, d[0] * g.ivx, d[1] * g.ivy, d[2] * g.ivz);
            Store<TO>::st(W, (int64_t)p * N + v, trilin_cell(ref, g, c.i0, c.j0, c.k0, c.fx, c.fy, c.fz));
        }
    }
}

// Fused adjoint with the DVF recomputed.  Per voxel, loops over p in order:
// d_mbc accumulates in registers (fixed order), d_ref scatters in fixed point,
// d_coeff contributions are reduced per warp and kept per warp in shared
// memory, then per block, then across blocks in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_warp_combine_bwd(GridD g, int L, int P, const T* __restrict__ ref,
                                                               const T* __restrict__ E, const float* __restrict__ w,
                                                               const float* __restrict__ dW, float* d_mbc,
                                                               unsigned long long* acc, const unsigned* maxbits,
                                                               float* part, int accumulate) {
    extern __shared__ float swarp[];  // [kThreads/32][P*L*3]
    const int PL3 = P * L * 3;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < (kThreads / 32) * PL3; t += kThreads) swarp[t] = 0.f;
    __syncthreads();
    const int64_t N = g.n;
    const int kexp = fixed_exponent(__uint_as_float(*maxbits) * (float)(N * P));
    const float scale = ldexpf(1.0f, kexp);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations so the
    // shuffles below stay converged
    const int64_t vbeg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iters = (N + stride - 1) / stride;
    for (int64_t it = 0; it < iters; it++) {
        const int64_t v = vbeg + it * stride;
        const bool live = v < N;
        int i = 0, j = 0, k = 0;
        float e[kMaxL][3], gE[kMaxL][3];
        for (int l = 0; l < L; l++)
#pragma unroll
            for (int a = 0; a < 3; a++) { e[l][a] = live ? Store<T>::ld(E, ((int64_t)l * 3 + a) * N + v) : 0.f; gE[l][a] = 0.f; }
        if (live) voxel_ijk(v, g, i, j, k);
        for (int p = 0; p < P; p++) {
            float gd[3] = {0.f, 0.f, 0.f};
            if (live) {
                float d[3];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    float s = 0.f;
                    for (int l = 0; l < L; l++) s = fmaf(__ldg(w + (p * L + l) * 3 + a), e[l][a], s);
                    d[a] = s;
                }
                const Cell c = make_cell(i, j, k, d[0] * g.ivx, d[1] * g.ivy, d[2] * g.ivz);
                const float gw = __ldg(dW + (int64_t)p * N + v);
                if (gw != 0.f) {
                    float gx, gy, gz;
                    trilin_grad(ref, g, c, gx, gy, gz);
                    gd[0] = gw * gx * g.ivx; gd[1] = gw * gy * g.ivy; gd[2] = gw * gz * g.ivz;
                    scatter_cell(acc, g, c, gw, scale);
                }
            }
            for (int l = 0; l < L; l++) {
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    gE[l][a] = fmaf(gd[a], __ldg(w + (p * L + l) * 3 + a), gE[l][a]);
                    float r = gd[a] * e[l][a];
                    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
                    if (lane == 0) swarp[wid * PL3 + (p * L + l) * 3 + a] += r;
                }
            }
        }
        if (live) {
            for (int l = 0; l < L; l++)
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    float* o = d_mbc + ((int64_t)l * 3 + a) * N + v;
                    *o = accumulate ? *o + gE[l][a] : gE[l][a];
                }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < PL3; t += kThreads) {
        float r = 0.f;
        for (int wi = 0; wi < kThreads / 32; wi++) r += swarp[wi * PL3 + t];
        part[(int64_t)t * gridDim.x + blockIdx.x] = r;
    }
}

// ---------------------------------------------- tiled fused combine + warp
//
// A CTA owns a TX x TY x TZ voxel tile (two voxels per thread: z and
// z + TZ / 2), keeps the coefficient table in shared memory and each voxel's
// MBC vectors in registers for all P projections.  The adjoint scatters V's
// gradient into a shared-memory box covering the tile plus a 4-voxel halo in
// 32-bit fixed point (per-CTA scale, provable bound), flushed once per CTA
// with 64-bit fixed-point atomics at the call's global scale; targets outside
// the halo go straight to global memory.
//
// Both take tiles eight voxels wide (a warp covers 8 x 4 voxels of one
// plane): a 200-voxel row is 25 tiles, where 32-wide tiles left a
// quarter-full last column whose warps paid full cost for 8 voxels.  The
// forward takes an 8x8x4 tile (128 threads), which keeps the staged halo
// small; the adjoint an 8x16x4 tile (256 threads), whose per-CTA work (zeroing
// and flushing the fixed-point box, the coefficient-gradient partials) per
// voxel matches the 32x4x4 tile's -- on an 8x8x4 tile that work, paid by twice
// as many CTAs, outweighed the ragged column.

constexpr int kHalo = 4;
constexpr int kMaxPLTile = 512;  // P * L limit of the tiled path

template <int TX_, int TY_, int TZ_, int PX_, int IX_ = PX_>
struct TileGeom {
    static constexpr int TX = TX_, TY = TY_, TZ = TZ_;
    static constexpr int THREADS = TX * TY * TZ / 2, WARPS = THREADS / 32;
    static constexpr int BX = TX + 2 * kHalo, BY = TY + 2 * kHalo, BZ = TZ + 2 * kHalo;
    static constexpr int PX = PX_;               // row pitch (pairs) of the staged ref box
    static constexpr int BOXN = PX * BY * BZ;    // pairs of the staged ref box
    static constexpr int IX = IX_;               // row pitch (words) of the adjoint's fixed-point box
    static constexpr int IBOXN = IX * BY * BZ;
    static_assert(TZ % 2 == 0 && THREADS % 32 == 0 && PX >= BX && IX >= BX, "tile shape");
};
// Forward: 16-pair rows (32 words), odd rows rotated by 8 pairs (pair_col).
using GeomFwd = TileGeom<8, 8, 4, 16>;
// Adjoint: an 8x16x4 tile of 256 threads, the same CTA size as a 32x4x4 tile
// (its per-CTA work per voxel unchanged) without a ragged x column on a
// 200-voxel row; ragged y tiles leave whole warps outside the grid, which skip
// the per-voxel work.  Its pair box as the forward's; fixed-point rows 24
// words apart put a warp's four rows of atomics on disjoint banks.
using GeomBwd = TileGeom<8, 16, 4, 16, 24>;

struct TileIdx {
    int x0, y0, z0;
    int x, y, z[2];
    int lx, ly, lz;  // box coordinates of the first voxel
};

template <class G>
__device__ __forceinline__ TileIdx tile_idx(const GridD& g) {
    const int ntx = (g.nx + G::TX - 1) / G::TX, nty = (g.ny + G::TY - 1) / G::TY;
    const int b = blockIdx.x, tid = threadIdx.x;
    TileIdx t;
    t.x0 = (b % ntx) * G::TX;
    t.y0 = ((b / ntx) % nty) * G::TY;
    t.z0 = (b / (ntx * nty)) * G::TZ;
    t.lx = tid % G::TX + kHalo;
    t.ly = (tid / G::TX) % G::TY + kHalo;
    t.lz = tid / (G::TX * G::TY) + kHalo;
    t.x = t.x0 + t.lx - kHalo;
    t.y = t.y0 + t.ly - kHalo;
    t.z[0] = t.z0 + t.lz - kHalo;
    t.z[1] = t.z[0] + G::TZ / 2;
    return t;
}

template <class G>
int num_tiles(const GridD& g) {
    return ((g.nx + G::TX - 1) / G::TX) * ((g.ny + G::TY - 1) / G::TY) * ((g.nz + G::TZ - 1) / G::TZ);
}

// a * b rounded once to the nearest integer, for |a b| < 2^22: the product is
// added to 1.5 * 2^23, where the float spacing is 1, by one fused multiply-add.
__device__ __forceinline__ int round_prod_small(float a, float b) {
    return __float_as_int(fmaf(a, b, 12582912.0f)) - 0x4b400000;
}

// Column of box x in a row of the pair box: rotated by 8 pairs in odd rows
// (the row parity is the y parity, BY being even).  8-byte shared loads are
// served per half-warp, and a half-warp reads two adjacent rows of 8 pairs:
// the rotation puts them on complementary halves of the 32 banks.
template <class G>
__device__ __forceinline__ int pair_col(int x, int row) {
    static_assert(G::BX == 16 && G::PX == 16 && G::BY % 2 == 0, "rotation of 16-pair rows");
    return x ^ ((row & 1) << 3);
}

// The tile's box of ref (the tile plus a kHalo-voxel halo) staged in shared
// memory as (x, x+1) pairs: the pair of box voxel (x, row) = (ref there, ref
// one voxel further along x), zero outside the grid, at column pair_col of
// rows G::PX pairs apart.  Displaced samples whose cell lies inside the box
// read their 8 corners as four aligned 8-byte loads instead of going through
// L1/L2.  Each half-warp stages one 16-voxel box row, the right neighbour
// coming from the next lane by a shuffle; the last pair of a row (never a
// lower cell corner) holds a zero.
template <class G, typename T>
__device__ __forceinline__ void stage_halo_pairs(const T* __restrict__ ref, const GridD& g, int bx0, int by0,
                                                 int bz0, float2* sv2) {
    constexpr int BX = G::BX, ROWS = G::BY * G::BZ;
    static_assert(BX == 16 && ROWS % (2 * G::WARPS) == 0, "half-warp rows, the same row count per warp");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xl = lane & 15, x = bx0 + xl;
    const bool inx = (unsigned)x < (unsigned)g.nx;
    for (int row = 2 * warp + (lane >> 4); row < ROWS; row += 2 * G::WARPS) {
        const int y = by0 + row % G::BY, z = bz0 + row / G::BY;
        const bool in = inx && (unsigned)y < (unsigned)g.ny && (unsigned)z < (unsigned)g.nz;
        const float va = in ? Store<T>::ld(ref, ((int64_t)z * g.ny + y) * g.nx + x) : 0.0f;
        const float va1 = __shfl_down_sync(0xffffffffu, va, 1);
        sv2[row * G::PX + pair_col<G>(xl, row)] = make_float2(va, xl == BX - 1 ? 0.0f : va1);
    }
}

// The 8 corners of the cell whose lower corner is box cell (rx, ry, rz), from
// the pair box (the caller has checked that the cell lies inside the box).
template <class G>
__device__ __forceinline__ void corners8_pairs(const float2* sv2, int rx, int ry, int rz, float cv[8]) {
    constexpr int SY = G::PX, SZ = G::PX * G::BY;
    const int r0 = rz * G::BY + ry;  // rows of the cell's y and y + 1 corners (and +BY for z + 1)
    const int i0 = r0 * SY + pair_col<G>(rx, r0), i1 = (r0 + 1) * SY + pair_col<G>(rx, r0 + 1);
    if (!PMF_DCHECK(i0 >= 0 && i1 >= 0 && i0 + SZ < G::BOXN && i1 + SZ < G::BOXN)) {
#pragma unroll
        for (int c = 0; c < 8; c++) cv[c] = 0.0f;
        return;
    }
    const float2 c00 = sv2[i0], c10 = sv2[i1], c01 = sv2[i0 + SZ], c11 = sv2[i1 + SZ];
    cv[0] = c00.x; cv[1] = c00.y; cv[2] = c10.x; cv[3] = c10.y;
    cv[4] = c01.x; cv[5] = c01.y; cv[6] = c11.x; cv[7] = c11.y;
}

template <class G>
__device__ __forceinline__ bool in_box(int rx, int ry, int rz) {
    return (unsigned)rx < (unsigned)(G::BX - 1) && (unsigned)ry < (unsigned)(G::BY - 1) &&
           (unsigned)rz < (unsigned)(G::BZ - 1);
}

// Box coordinate r = l + floor(t) of the lower cell corner and the fraction
// f = t - floor(t) of a displacement t (voxels) for a voxel at box coordinate
// l, from one round-down add of 1.5 * 2^23 (where the float spacing is 1):
// exact for |t| < 2^22.  Larger |t|, inf and NaN give an r far outside the box,
// so a caller that takes r only after testing it against the box never uses
// an inexact result (it recomputes the cell with split_offset instead).
__device__ __forceinline__ int box_floor(float t, int l, float& f) {
    const float tt = __fadd_rd(t, 12582912.0f);
    f = t - (tt - 12582912.0f);
    return (int)((unsigned)__float_as_int(tt) - (0x4b400000u - (unsigned)l));
}

// Coefficient table of a batch as one float4 (x, y, z, 0) per (view, level):
// a view's L levels are L broadcast 16-byte shared loads.
__device__ __forceinline__ void stage_coeff4(const float* __restrict__ w, int PL, float4* sw4) {
    for (int i = threadIdx.x; i < PL; i += blockDim.x) sw4[i] = make_float4(w[3 * i], w[3 * i + 1], w[3 * i + 2], 0.0f);
}

template <typename T, typename TO, int L>
__global__ void __launch_bounds__(GeomFwd::THREADS, 6) k_wc_fwd_tile(GridD g, int P, const T* __restrict__ ref,
                                                     const T* __restrict__ E, const float* __restrict__ w,
                                                     TO* __restrict__ W) {
    using G = GeomFwd;
    extern __shared__ float4 smem_f4[];
    float4* sw4 = smem_f4;                          // [P][L] coefficients
    float2* sv2 = (float2*)(smem_f4 + P * L);       // [BZ][BY][PX] ref pairs
    stage_coeff4(w, P * L, sw4);
    const TileIdx t = tile_idx<G>(g);
    stage_halo_pairs<G>(ref, g, t.x0 - kHalo, t.y0 - kHalo, t.z0 - kHalo, sv2);
    __syncthreads();
    if (t.x >= g.nx || t.y >= g.ny) return;
    const int64_t N = g.n;
    // box coordinates of the thread's voxels (z and z + TZ / 2)
    const int lx = t.lx, ly = t.ly, lz = t.lz;
    const f32x2 M2 = pack2(12582912.0f, 12582912.0f);
    bool in[2];
    f32x2 exy[2][L];
    float ez[2][L];
    TO* out[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        in[h] = t.z[h] < g.nz;
        const int64_t v = in[h] ? ((int64_t)t.z[h] * g.ny + t.y) * g.nx + t.x : 0;
        out[h] = W + v;
#pragma unroll
        for (int l = 0; l < L; l++) {  // MBC vectors in voxels: the displacement is then sum_l c e
            const float ex = in[h] ? Store<T>::ld(E, ((int64_t)l * 3 + 0) * N + v) : 0.0f;
            const float ey = in[h] ? Store<T>::ld(E, ((int64_t)l * 3 + 1) * N + v) : 0.0f;
            const float e_z = in[h] ? Store<T>::ld(E, ((int64_t)l * 3 + 2) * N + v) : 0.0f;
            exy[h][l] = pack2(ex * g.ivx, ey * g.ivy);
            ez[h][l] = e_z * g.ivz;
        }
    }
    for (int p = 0; p < P; p++) {
        f32x2 cxy[L];
        float cz[L];
#pragma unroll
        for (int l = 0; l < L; l++) {
            const float4 c = sw4[p * L + l];
            cxy[l] = pack2(c.x, c.y);
            cz[l] = c.z;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            // a voxel beyond the grid's last z plane (e = 0, no store) runs the
            // same code, so the loop has no branch on it
            // the x and y displacements as one packed pair: their blend, and the
            // round-down add and the fractions of box_floor, take one
            // instruction for both (each half the scalar operation's bits)
            f32x2 dxy = pack2(0.0f, 0.0f);
            float dz = 0.0f;
#pragma unroll
            for (int l = 0; l < L; l++) {
                dxy = fma2(cxy[l], exy[h][l], dxy);
                dz = fmaf(cz[l], ez[h][l], dz);
            }
            const float tx = lo2(dxy), ty = hi2(dxy), tz = dz;
            float fx, fy, fz, cv[8];
            f32x2 tt;
            asm("add.rm.f32x2 %0, %1, %2;" : "=l"(tt) : "l"(dxy), "l"(M2));
            const f32x2 fxy = sub2(dxy, sub2(tt, M2));
            fx = lo2(fxy);
            fy = hi2(fxy);
            const int rx = (int)((unsigned)__float_as_int(lo2(tt)) - (0x4b400000u - (unsigned)lx));
            const int ry = (int)((unsigned)__float_as_int(hi2(tt)) - (0x4b400000u - (unsigned)ly));
            const int rz = box_floor(tz, lz + h * (G::TZ / 2), fz);
            if (in_box<G>(rx, ry, rz)) {
                corners8_pairs<G>(sv2, rx, ry, rz, cv);
            } else {
                int ox, oy, oz;
                split_offset(tx, ox, fx);
                split_offset(ty, oy, fy);
                split_offset(tz, oz, fz);
                corners8(ref, g, t.x + ox, t.y + oy, t.z[h] + oz, cv);
            }
            const float wv = trilin8(cv, fx, fy, fz);
            if (in[h]) Store<TO>::st(out[h], 0, wv);
            out[h] += N;
        }
    }
}

// Sums each of K per-lane values over the warp by halving exchange: at each
// level a lane keeps one half of its values (the lower half when its lane bit
// for that level is clear) and sends the other half to its partner, so K
// values take about K + log2(32 / K) shuffles instead of 5 K.  Lanes end with
// the sum of the value slot that split_slot<K> names for them.
template <int N, int O>
struct SplitReduce {
    static __device__ __forceinline__ void run(float* x, int lane) {
        constexpr int H = (N + 1) / 2;
        const bool up = (lane & O) != 0;
#pragma unroll
        for (int k = 0; k < H; k++) {
            const float hi = H + k < N ? x[H + k] : 0.0f;
            const float r = __shfl_xor_sync(0xffffffffu, up ? x[k] : hi, O);
            x[k] = (up ? hi : x[k]) + r;
        }
        SplitReduce<H, O / 2>::run(x, lane);
    }
};
template <int O>
struct SplitReduce<1, O> {
    static __device__ __forceinline__ void run(float* x, int) {
#pragma unroll
        for (int o = O; o >= 1; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
    }
};

// Which of the K slots lane ends with after SplitReduce<K, 16> (-1: a padding
// slot, or a lane whose partner in the final plain butterfly writes instead).
template <int K>
__device__ __forceinline__ int split_slot(int lane) {
    static_assert(K >= 1 && K <= 32, "one to 32 values per lane");
    int n = K, real = K, slot = 0, last = 32;
    for (int o = 16; o >= 1 && n > 1; o >>= 1) {
        const int h = (n + 1) / 2;
        if (lane & o) {
            slot += h;
            real -= h;
        } else {
            real = real < h ? real : h;
        }
        n = h;
        last = o;
    }
    return real >= 1 && (lane & (last - 1)) == 0 ? slot : -1;
}

__device__ __forceinline__ int exp_bits(float bound, int bits) {
    if (!(bound > 0.0f) || !isfinite(bound)) return 0;
    int e;
    frexpf(bound, &e);
    const int k = bits - e;
    return k > 126 ? 126 : (k < -126 ? -126 : k);
}

template <typename T, int L>
__global__ void __launch_bounds__(GeomBwd::THREADS, 2) k_wc_bwd_tile(GridD g, int P, const T* __restrict__ ref,
                                                        const T* __restrict__ E, const float* __restrict__ w,
                                                        const float* __restrict__ dW, float* d_mbc,
                                                        unsigned long long* acc, const unsigned* maxbits, float* part,
                                                        int accumulate) {
    using G = GeomBwd;
    constexpr int K = 3 * L;  // coefficient-gradient values of one view
    constexpr int SY = G::IX, SZ = G::IX * G::BY;  // fixed-point box strides
    extern __shared__ float4 smem_b4[];
    const int PL = P * L, PK = P * K;
    float4* sw4 = smem_b4;                         // [P][L] coefficients
    float2* sv2 = (float2*)(sw4 + PL);             // [BZ][BY][PX] ref pairs
    int* box = (int*)(sv2 + G::BOXN);              // [BZ][BY][IX] fixed-point dV
    float* swarp = (float*)(box + G::IBOXN);       // [warps][P][L][3]
    __shared__ float red_sum[G::WARPS];
    __shared__ unsigned red_max;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    stage_coeff4(w, PL, sw4);
    for (int i = threadIdx.x; i < G::IBOXN; i += G::THREADS) box[i] = 0;
    for (int i = threadIdx.x; i < G::WARPS * PK; i += G::THREADS) swarp[i] = 0.f;
    if (threadIdx.x == 0) red_max = 0u;
    const TileIdx t = tile_idx<G>(g);
    stage_halo_pairs<G>(ref, g, t.x0 - kHalo, t.y0 - kHalo, t.z0 - kHalo, sv2);
    const int64_t N = g.n;
    bool in[2];
    int64_t v[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        in[h] = t.x < g.nx && t.y < g.ny && t.z[h] < g.nz;
        v[h] = in[h] ? ((int64_t)t.z[h] * g.ny + t.y) * g.nx + t.x : 0;
    }
    // per-CTA fixed-point scale: one target voxel receives at most
    // sum |dW| over the tile's (voxel, view) pairs, each addend at most max |dW|
    float s = 0.f, m = 0.f;
    for (int p = 0; p < P; p++)
#pragma unroll
        for (int h = 0; h < 2; h++)
            if (in[h]) {
                const float a = fabsf(__ldg(dW + (int64_t)p * N + v[h]));
                s += a;
                m = fmaxf(m, a);
            }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    __syncthreads();
    if (lane == 0) {
        red_sum[warp] = s;
        if (mb) atomicMax(&red_max, mb);
    }
    __syncthreads();
    float stot = 0.f;
    for (int i = 0; i < G::WARPS; i++) stot += red_sum[i];
    const int kg = fixed_exponent(__uint_as_float(*maxbits) * (float)(N * P));
    const int kb = min(min(exp_bits(stot, 29), exp_bits(__uint_as_float(red_max), 21)), kg);
    const float sb = ldexpf(1.0f, kb), sg = ldexpf(1.0f, kg);
    const int shift = kg - kb;
    const int bx0 = t.x0 - kHalo, by0 = t.y0 - kHalo, bz0 = t.z0 - kHalo;
    const int lx = t.lx, ly = t.ly, lz = t.lz;
    const int slot = split_slot<K>(lane);

    bool halo_exit = false;
    // MBC vectors in voxels (as in the forward), x and y as packed pairs; the
    // per-view DVF gradient then stays in voxel units and the 1 / voxel
    // factors are applied once at the end
    f32x2 exy[2][L], gExy[2][L];
    float ez[2][L], gEz[2][L];
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int l = 0; l < L; l++) {
            const float ex = in[h] ? Store<T>::ld(E, ((int64_t)l * 3 + 0) * N + v[h]) : 0.f;
            const float ey = in[h] ? Store<T>::ld(E, ((int64_t)l * 3 + 1) * N + v[h]) : 0.f;
            const float e_z = in[h] ? Store<T>::ld(E, ((int64_t)l * 3 + 2) * N + v[h]) : 0.f;
            exy[h][l] = pack2(ex * g.ivx, ey * g.ivy);
            ez[h][l] = e_z * g.ivz;
            gExy[h][l] = pack2(0.f, 0.f);
            gEz[h][l] = 0.f;
        }
    const f32x2 M2 = pack2(12582912.0f, 12582912.0f);
    // dW of the next view is loaded one view ahead
    float gw_next[2];
#pragma unroll
    for (int h = 0; h < 2; h++) gw_next[h] = in[h] && P > 0 ? __ldg(dW + v[h]) : 0.f;
    for (int p = 0; p < P; p++) {
        float gwv[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            gwv[h] = gw_next[h];
            gw_next[h] = in[h] && p + 1 < P ? __ldg(dW + (int64_t)(p + 1) * N + v[h]) : 0.f;
        }
        f32x2 cxy[L], cwxy[L];
        float cz[L], cwz[L];
#pragma unroll
        for (int l = 0; l < L; l++) {
            const float4 c = sw4[p * L + l];
            cxy[l] = pack2(c.x, c.y);
            cz[l] = c.z;
            cwxy[l] = pack2(0.f, 0.f);
            cwz[l] = 0.f;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const float gw = gwv[h];
            if (gw == 0.f) continue;  // also every voxel outside the grid
            f32x2 dxy = pack2(0.f, 0.f);
            float dz = 0.0f;
#pragma unroll
            for (int l = 0; l < L; l++) {
                dxy = fma2(cxy[l], exy[h][l], dxy);
                dz = fmaf(cz[l], ez[h][l], dz);
            }
            const float tx = lo2(dxy), ty = hi2(dxy), tz = dz;
            Cell cl;
            f32x2 tt;
            asm("add.rm.f32x2 %0, %1, %2;" : "=l"(tt) : "l"(dxy), "l"(M2));
            const f32x2 fxy = sub2(dxy, sub2(tt, M2));
            cl.fx = lo2(fxy);
            cl.fy = hi2(fxy);
            const int rx = (int)((unsigned)__float_as_int(lo2(tt)) - (0x4b400000u - (unsigned)lx));
            const int ry = (int)((unsigned)__float_as_int(hi2(tt)) - (0x4b400000u - (unsigned)ly));
            const int rz = box_floor(tz, lz + h * (G::TZ / 2), cl.fz);
            const bool inside = in_box<G>(rx, ry, rz);
            float gx, gy, gz, cv[8];
            if (inside) {
                corners8_pairs<G>(sv2, rx, ry, rz, cv);
            } else {
                int ox, oy, oz;
                split_offset(tx, ox, cl.fx);
                split_offset(ty, oy, cl.fy);
                split_offset(tz, oz, cl.fz);
                cl.i0 = t.x + ox; cl.j0 = t.y + oy; cl.k0 = t.z[h] + oz;
                corners8(ref, g, cl.i0, cl.j0, cl.k0, cv);
            }
            trilin8_grad(cv, cl, gx, gy, gz);
            // dL/d(displacement in voxels), x and y packed
            const f32x2 gdxy = mul2(pack2(gw, gw), pack2(gx, gy));
            const float gdz = gw * gz;
#pragma unroll
            for (int l = 0; l < L; l++) {
                gExy[h][l] = fma2(gdxy, cxy[l], gExy[h][l]);
                gEz[h][l] = fmaf(gdz, cz[l], gEz[h][l]);
                cwxy[l] = fma2(gdxy, exy[h][l], cwxy[l]);
                cwz[l] = fmaf(gdz, ez[h][l], cwz[l]);
            }
            // V's adjoint: the 8 trilinear corners, each weight times gw rounded
            // once to the CTA's fixed point
            if (inside && PMF_DCHECK(rz * SZ + ry * SY + rx >= 0 && rz * SZ + ry * SY + rx + SZ + SY + 1 < G::IBOXN)) {
                int* q = box + rz * SZ + ry * SY + rx;
                const float gz0 = gw * sb * (1.f - cl.fz), gz1 = gw * sb * cl.fz;
                const float wyz[2][2] = {{gz0 * (1.f - cl.fy), gz0 * cl.fy}, {gz1 * (1.f - cl.fy), gz1 * cl.fy}};
                const float wx0 = 1.f - cl.fx, wx1 = cl.fx;
#pragma unroll
                for (int dz = 0; dz < 2; dz++)
#pragma unroll
                    for (int dy = 0; dy < 2; dy++) {
                        int* r = q + dz * SZ + dy * SY;
                        atomicAdd(r, round_prod_small(wyz[dz][dy], wx0));
                        atomicAdd(r + 1, round_prod_small(wyz[dz][dy], wx1));
                    }
            } else {
                scatter_cell(acc, g, cl, gw, sg);
                halo_exit = true;
            }
        }
        // coefficient gradient partials: halving warp reduction, then the
        // warp's own slot
        float cw[K];
#pragma unroll
        for (int l = 0; l < L; l++) {
            cw[3 * l] = lo2(cwxy[l]);
            cw[3 * l + 1] = hi2(cwxy[l]);
            cw[3 * l + 2] = cwz[l];
        }
        SplitReduce<K, 16>::run(cw, lane);
        if (slot >= 0) swarp[warp * PK + p * K + slot] += cw[0];
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
        if (!in[h]) continue;
#pragma unroll
        for (int l = 0; l < L; l++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                float* o = d_mbc + ((int64_t)l * 3 + a) * N + v[h];
                const float gv = a == 0 ? lo2(gExy[h][l]) : (a == 1 ? hi2(gExy[h][l]) : gEz[h][l]);
                const float ge = gv * (a == 0 ? g.ivx : (a == 1 ? g.ivy : g.ivz));
                *o = accumulate ? *o + ge : ge;
            }
    }
    if (__syncthreads_or(halo_exit) && threadIdx.x == 0) diag_count(PMF_DIAG_WARP_HALO_EXIT);
    for (int i = threadIdx.x; i < PK; i += G::THREADS) {
        float r = 0.f;
        for (int wi = 0; wi < G::WARPS; wi++) r += swarp[wi * PK + i];
        part[(int64_t)i * gridDim.x + blockIdx.x] = r;
    }
    for (int i = threadIdx.x; i < G::IBOXN; i += G::THREADS) {
        const int val = box[i];
        if (val == 0) continue;  // also the padding columns of a pitch wider than the box
        const int x = bx0 + i % SY, y = by0 + (i / SY) % G::BY, z = bz0 + i / SZ;
        if ((unsigned)x < (unsigned)g.nx && (unsigned)y < (unsigned)g.ny && (unsigned)z < (unsigned)g.nz)
            atomicAdd(acc + ((int64_t)z * g.ny + y) * g.nx + x, (unsigned long long)((long long)val * (1ll << shift)));
    }
}

// One CTA per output: strided fixed-order partial sums, then a fixed tree,
// in double (the tile partials of a coefficient gradient cancel heavily).
__global__ void __launch_bounds__(256) k_reduce_partials_wide(const float* part, int nb, float* out, int accumulate) {
    __shared__ double red[8];
    const int64_t o = blockIdx.x;
    double r = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) r += (double)part[o * nb + b];
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; i++) t += red[i];
        out[o] = accumulate ? out[o] + (float)t : (float)t;
    }
}

template <typename T, int LL>
void launch_wc_bwd(unsigned nt, size_t smem, cudaStream_t s, const GridD& g, int P, const void* ref, const void* mbc,
                   const float* coeff, const float* d_out, float* d_mbc, unsigned long long* acc,
                   const unsigned* maxbits, float* part, int accumulate) {
    cudaFuncSetAttribute(k_wc_bwd_tile<T, LL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_wc_bwd_tile<T, LL><<<nt, GeomBwd::THREADS, smem, s>>>(g, P, (const T*)ref, (const T*)mbc, coeff, d_out, d_mbc, acc, maxbits,
                                                part, accumulate);
}

unsigned stream_blocks(int64_t work) {
    int64_t b = (work + kThreads - 1) / kThreads;
    return (unsigned)(b < kStreamBlocks ? (b > 0 ? b : 1) : kStreamBlocks);
}

pmf_status check_common(const pmf_grid* grid, int32_t P, pmf_dtype dtype) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    if ((st = validate_dtype(dtype)) != PMF_OK) return st;
    PMF_REQUIRE(P >= 0, "P must be >= 0");
    return PMF_OK;
}

}  // namespace

PMF_DIAG_ACCESSOR(diag_warp)

}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status mbc_combine(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* mbc,
                       const float* coeff, void* dvf, pmf_stream stream) {
    pmf_status st = check_common(grid, P, dtype);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(L >= 1 && L <= kMaxL, "L must be in [1, %d]", kMaxL);
    if (P == 0) return PMF_OK;
    PMF_REQUIRE(mbc && coeff && dvf, "null pointer");
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
    PMF_DISPATCH_DTYPE(dtype, T, k_combine<T><<<stream_blocks(g.n), kThreads, 0, s>>>(g, L, P, (const T*)mbc, coeff, (T*)dvf));
    return check_launch("mbc_combine");
}

pmf_status mbc_combine_backward_workspace(const pmf_grid* grid, int32_t L, int32_t P, size_t* bytes) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(bytes != nullptr, "bytes is null");
    PMF_REQUIRE(L >= 1 && L <= kMaxL && P >= 0, "bad L/P");
    *bytes = align_up(sizeof(float) * (size_t)P * L * 3 * kStreamBlocks);
    return PMF_OK;
}

pmf_status mbc_combine_backward(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* mbc,
                                const float* coeff, const float* d_dvf, float* d_mbc, float* d_coeff, int accumulate,
                                void* ws, size_t ws_bytes, pmf_stream stream) {
    pmf_status st = check_common(grid, P, dtype);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(L >= 1 && L <= kMaxL, "L must be in [1, %d]", kMaxL);
    size_t need;
    mbc_combine_backward_workspace(grid, L, P, &need);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
    PMF_REQUIRE(mbc && d_mbc && (P == 0 || (coeff && d_dvf && d_coeff)), "null pointer");
    if (P == 0) {
        if (!accumulate) cudaMemsetAsync(d_mbc, 0, sizeof(float) * (size_t)(L * 3 * g.n), s);
        return check_launch("mbc_combine_backward");
    }
    k_combine_bwd_mbc<<<stream_blocks(g.n), kThreads, 0, s>>>(g, L, P, coeff, d_dvf, d_mbc, accumulate);
    dim3 gr(kStreamBlocks, (unsigned)(P * 3));
    float* part = (float*)ws;
    PMF_DISPATCH_DTYPE(dtype, T, k_combine_bwd_coeff<T><<<gr, kThreads, 0, s>>>(g, L, P, (const T*)mbc, d_dvf, part));
    int64_t nout = (int64_t)P * L * 3;
    k_reduce_partials<<<(unsigned)((nout + 255) / 256), 256, 0, s>>>(part, nout, kStreamBlocks, d_coeff, accumulate);
    return check_launch("mbc_combine_backward");
}

pmf_status warp_volume(const pmf_grid* grid, int32_t P, pmf_dtype dtype, const void* ref, const void* dvf, void* out,
                       pmf_stream stream) {
    pmf_status st = check_common(grid, P, dtype);
    if (st != PMF_OK) return st;
    if (P == 0) return PMF_OK;
    PMF_REQUIRE(ref && dvf && out, "null pointer");
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
    PMF_DISPATCH_DTYPE(dtype, T, k_warp<T><<<stream_blocks(g.n * P), kThreads, 0, s>>>(g, P, (const T*)ref, (const T*)dvf, (T*)out));
    return check_launch("warp_volume");
}

pmf_status warp_volume_backward_workspace(const pmf_grid* grid, int32_t P, size_t* bytes) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(bytes != nullptr && P >= 0, "bad arguments");
    GridD g = make_grid(grid);
    *bytes = align_up(256) + align_up(sizeof(unsigned long long) * (size_t)g.n);
    return PMF_OK;
}

pmf_status warp_volume_backward(const pmf_grid* grid, int32_t P, pmf_dtype dtype, const void* ref, const void* dvf,
                                const float* d_out, float* d_ref, float* d_dvf, int accumulate, void* ws,
                                size_t ws_bytes, pmf_stream stream) {
    pmf_status st = check_common(grid, P, dtype);
    if (st != PMF_OK) return st;
    size_t need;
    warp_volume_backward_workspace(grid, P, &need);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    PMF_REQUIRE(ref && d_ref && (P == 0 || (dvf && d_out)), "null pointer");
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* maxbits = (unsigned*)ws;
    unsigned long long* acc = (unsigned long long*)((char*)ws + align_up(256));
    cudaMemsetAsync(ws, 0, need, s);
    if (P > 0) {
        k_absmax<<<stream_blocks(g.n * P), kThreads, 0, s>>>(d_out, g.n * P, maxbits);
        PMF_DISPATCH_DTYPE(dtype, T, k_warp_bwd<T><<<stream_blocks(g.n * P), kThreads, 0, s>>>(g, P, (const T*)ref, (const T*)dvf, d_out, d_dvf, acc, maxbits, accumulate));
    }
    k_fixed_to_float<<<stream_blocks(g.n), kThreads, 0, s>>>(acc, g.n, maxbits, (float)(g.n * (int64_t)P), d_ref, accumulate);
    return check_launch("warp_volume_backward");
}

}  // extern "C"

namespace pmf {
namespace {

template <typename T, typename TO, int LL>
void launch_wc_fwd(unsigned nt, size_t smem, cudaStream_t s, const GridD& g, int P, const void* ref, const void* mbc,
                   const float* coeff, void* out) {
    cudaFuncSetAttribute(k_wc_fwd_tile<T, TO, LL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_wc_fwd_tile<T, TO, LL><<<nt, GeomFwd::THREADS, smem, s>>>(g, P, (const T*)ref, (const T*)mbc, coeff, (TO*)out);
}

template <typename T, typename TO>
pmf_status launch_warp_combine(const GridD& g, int32_t L, int32_t P, const void* ref, const void* mbc,
                               const float* coeff, void* out, cudaStream_t s) {
    if (L <= 4 && (int64_t)P * L <= kMaxPLTile && g.n < ((int64_t)1 << 31)) {
        const size_t smem = sizeof(float4) * (size_t)(P * L) + sizeof(float2) * (size_t)GeomFwd::BOXN;
        const unsigned nt = (unsigned)num_tiles<GeomFwd>(g);
        switch (L) {
            case 1: launch_wc_fwd<T, TO, 1>(nt, smem, s, g, P, ref, mbc, coeff, out); break;
            case 2: launch_wc_fwd<T, TO, 2>(nt, smem, s, g, P, ref, mbc, coeff, out); break;
            case 3: launch_wc_fwd<T, TO, 3>(nt, smem, s, g, P, ref, mbc, coeff, out); break;
            default: launch_wc_fwd<T, TO, 4>(nt, smem, s, g, P, ref, mbc, coeff, out); break;
        }
        return check_launch("warp_combine");
    }
    k_warp_combine<T, TO><<<stream_blocks(g.n), kThreads, 0, s>>>(g, L, P, (const T*)ref, (const T*)mbc, coeff, (TO*)out);
    return check_launch("warp_combine");
}

pmf_status warp_combine_impl(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref,
                             const void* mbc, const float* coeff, pmf_dtype out_dtype, void* out, pmf_stream stream) {
    pmf_status st = check_common(grid, P, dtype);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(L >= 1 && L <= kMaxL, "L must be in [1, %d]", kMaxL);
    PMF_REQUIRE(out_dtype == dtype || out_dtype == PMF_F32, "out_dtype must be dtype or PMF_F32");
    if (P == 0) return PMF_OK;
    PMF_REQUIRE(ref && mbc && coeff && out, "null pointer");
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
    if (out_dtype == PMF_F32) {
        PMF_DISPATCH_DTYPE(dtype, T, return (launch_warp_combine<T, float>(g, L, P, ref, mbc, coeff, out, s)));
    }
    PMF_DISPATCH_DTYPE(dtype, T, return (launch_warp_combine<T, T>(g, L, P, ref, mbc, coeff, out, s)));
    return PMF_OK;
}

}  // namespace
}  // namespace pmf

extern "C" {

pmf_status warp_combine(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref, const void* mbc,
                        const float* coeff, void* out, pmf_stream stream) {
    return warp_combine_impl(grid, L, P, dtype, ref, mbc, coeff, dtype, out, stream);
}

pmf_status warp_combine_mixed(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref,
                              const void* mbc, const float* coeff, pmf_dtype out_dtype, void* out, pmf_stream stream) {
    return warp_combine_impl(grid, L, P, dtype, ref, mbc, coeff, out_dtype, out, stream);
}

pmf_status warp_combine_backward_workspace(const pmf_grid* grid, int32_t L, int32_t P, size_t* bytes) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(bytes != nullptr && P >= 0 && L >= 1 && L <= kMaxL, "bad arguments");
    GridD g = make_grid(grid);
    const size_t nb = (size_t)(num_tiles<GeomBwd>(g) > kStreamBlocks ? num_tiles<GeomBwd>(g) : kStreamBlocks);
    *bytes = align_up(256) + align_up(sizeof(unsigned long long) * (size_t)g.n) +
             align_up(sizeof(float) * (size_t)P * L * 3 * nb);
    return PMF_OK;
}

}  // extern "C"

namespace pmf {
namespace {

// The fused adjoint; out_bits (device, optional) holds max |d_out| as abs_bits,
// computed by the producer of d_out, in place of this call's own pass over it.
pmf_status wc_backward_impl(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref,
                            const void* mbc, const float* coeff, const float* d_out, const unsigned* out_bits,
                            float* d_ref, float* d_mbc, float* d_coeff, int accumulate, void* ws, size_t ws_bytes,
                            pmf_stream stream) {
    pmf_status st = check_common(grid, P, dtype);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(L >= 1 && L <= kMaxL, "L must be in [1, %d]", kMaxL);
    size_t need;
    warp_combine_backward_workspace(grid, L, P, &need);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    PMF_REQUIRE(ref && mbc && d_ref && d_mbc && (P == 0 || (coeff && d_out && d_coeff)), "null pointer");
    const size_t smem = sizeof(float) * (kThreads / 32) * (size_t)P * L * 3;
    if (smem > 200 * 1024) return set_error(PMF_EUNSUPPORTED, "P*L too large for the fused adjoint (P*L <= %d)", (int)(200 * 1024 / (4 * 8 * 3)));
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* ws_bits = (unsigned*)ws;
    const unsigned* maxbits = out_bits && P > 0 ? out_bits : ws_bits;
    unsigned long long* acc = (unsigned long long*)((char*)ws + align_up(256));
    float* part = (float*)((char*)acc + align_up(sizeof(unsigned long long) * (size_t)g.n));
    cudaMemsetAsync(ws, 0, align_up(256) + align_up(sizeof(unsigned long long) * (size_t)g.n), s);
    if (P == 0) {
        if (!accumulate) cudaMemsetAsync(d_mbc, 0, sizeof(float) * (size_t)(L * 3 * g.n), s);
    } else {
        if (!out_bits) k_absmax<<<stream_blocks(g.n * P), kThreads, 0, s>>>(d_out, g.n * P, ws_bits);
        if (L <= 4 && (int64_t)P * L <= kMaxPLTile && g.n < ((int64_t)1 << 31)) {
            const int PL3 = P * L * 3;
            const size_t smem2 = sizeof(float4) * (size_t)(P * L) + sizeof(float2) * (size_t)GeomBwd::BOXN +
                                 sizeof(int) * (size_t)GeomBwd::IBOXN + sizeof(float) * (size_t)(GeomBwd::WARPS * PL3);
            const unsigned nt = (unsigned)num_tiles<GeomBwd>(g);
            PMF_DISPATCH_DTYPE(dtype, T, {
                switch (L) {
                    case 1: launch_wc_bwd<T, 1>(nt, smem2, s, g, P, ref, mbc, coeff, d_out, d_mbc, acc, maxbits, part, accumulate); break;
                    case 2: launch_wc_bwd<T, 2>(nt, smem2, s, g, P, ref, mbc, coeff, d_out, d_mbc, acc, maxbits, part, accumulate); break;
                    case 3: launch_wc_bwd<T, 3>(nt, smem2, s, g, P, ref, mbc, coeff, d_out, d_mbc, acc, maxbits, part, accumulate); break;
                    default: launch_wc_bwd<T, 4>(nt, smem2, s, g, P, ref, mbc, coeff, d_out, d_mbc, acc, maxbits, part, accumulate); break;
                }
            });
            k_reduce_partials_wide<<<(unsigned)(P * L * 3), 256, 0, s>>>(part, (int)nt, d_coeff, accumulate);
            k_fixed_to_float<<<stream_blocks(g.n), kThreads, 0, s>>>(acc, g.n, maxbits, (float)(g.n * (int64_t)P), d_ref, accumulate);
            return check_launch("warp_combine_backward");
        }
        const unsigned nb = stream_blocks(g.n);
        PMF_DISPATCH_DTYPE(dtype, T, {
            if (smem > 48 * 1024) cudaFuncSetAttribute(k_warp_combine_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_warp_combine_bwd<T><<<nb, kThreads, smem, s>>>(g, L, P, (const T*)ref, (const T*)mbc, coeff, d_out, d_mbc, acc, maxbits, part, accumulate);
        });
        int64_t nout = (int64_t)P * L * 3;
        k_reduce_partials<<<(unsigned)((nout + 255) / 256), 256, 0, s>>>(part, nout, (int)nb, d_coeff, accumulate);
    }
    k_fixed_to_float<<<stream_blocks(g.n), kThreads, 0, s>>>(acc, g.n, maxbits, (float)(g.n * (int64_t)P), d_ref, accumulate);
    return check_launch("warp_combine_backward");
}

}  // namespace
}  // namespace pmf

extern "C" {

pmf_status warp_combine_backward(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref,
                                 const void* mbc, const float* coeff, const float* d_out, float* d_ref, float* d_mbc,
                                 float* d_coeff, int accumulate, void* ws, size_t ws_bytes, pmf_stream stream) {
    return wc_backward_impl(grid, L, P, dtype, ref, mbc, coeff, d_out, nullptr, d_ref, d_mbc, d_coeff, accumulate, ws,
                            ws_bytes, stream);
}

pmf_status warp_combine_backward_bounded(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref,
                                         const void* mbc, const float* coeff, const float* d_out,
                                         const unsigned* d_out_absmax_bits, float* d_ref, float* d_mbc,
                                         float* d_coeff, int accumulate, void* ws, size_t ws_bytes,
                                         pmf_stream stream) {
    PMF_REQUIRE(d_out_absmax_bits != nullptr, "d_out_absmax_bits is null");
    return wc_backward_impl(grid, L, P, dtype, ref, mbc, coeff, d_out, d_out_absmax_bits, d_ref, d_mbc, d_coeff,
                            accumulate, ws, ws_bytes, stream);
}

}  // extern "C"

// ------------------------------------------- no-allocation adjoint variant
//
// mbc_combine_backward_noalloc: the same computation as mbc_combine_backward
// for callers that cannot allocate device memory on the call path (for
// example code whose device memory is all handed out up front by its own
// pool, or code that must not risk the implicit device-wide synchronization
// that allocating and freeing can cause).  Its scratch -- the per-block
// partial sums of d_coeff -- lives in one fixed array in the library's device
// image instead of a caller-supplied workspace.

#include <mutex>

namespace pmf {
namespace {

constexpr int kNoAllocMaxPL = 128;  // P * L limit: 128 * 3 * 608 floats, about 0.9 MB per device
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_part[kNoAllocMaxPL * 3 * kStreamBlocks];

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};
void* g_noalloc_ctx[kNoAllocMaxDevices] = {};

// The calling thread's current context (cuCtxGetCurrent through the runtime's
// driver entry point, so the library needs no link-time driver dependency);
// nullptr if it cannot be queried.
void* current_context() {
    typedef int (*CtxGetCurrent)(void**);
    static CtxGetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return (CtxGetCurrent)f;
    }();
    void* ctx = nullptr;
    if (fn == nullptr || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of g_noalloc_part on the current device, looked up on the
// first call on each device (the host-side symbol is only a stand-in, never a
// device address) and again whenever the device's context has changed since
// (after cudaDeviceReset the old address is stale).
pmf_status noalloc_scratch(float** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(PMF_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(PMF_EUNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    void* ctx = current_context();
    if (g_noalloc_ptr[dev] == nullptr || ctx == nullptr || ctx != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_part);
        if (e != cudaSuccess || p == nullptr)
            return set_error(PMF_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (float*)p;
        g_noalloc_ctx[dev] = ctx;  // cudaGetSymbolAddress made the primary context current if none was
        if (ctx == nullptr) g_noalloc_ctx[dev] = current_context();
    }
    *out = g_noalloc_ptr[dev];
    return PMF_OK;
}

}  // namespace
}  // namespace pmf

extern "C" pmf_status mbc_combine_backward_noalloc(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype,
                                                   const void* mbc, const float* coeff, const float* d_dvf,
                                                   float* d_mbc, float* d_coeff, int accumulate, pmf_stream stream) {
    pmf_status st = check_common(grid, P, dtype);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(L >= 1 && L <= kMaxL, "L must be in [1, %d]", kMaxL);
    if ((int64_t)P * L > kNoAllocMaxPL)
        return set_error(PMF_EWORKSPACE, "P*L = %lld exceeds the fixed scratch of the no-allocation variant (P*L <= %d)",
                         (long long)P * L, kNoAllocMaxPL);
    PMF_REQUIRE(mbc && d_mbc && (P == 0 || (coeff && d_dvf && d_coeff)), "null pointer");
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
    if (P == 0) {
        if (!accumulate) cudaMemsetAsync(d_mbc, 0, sizeof(float) * (size_t)(L * 3 * g.n), s);
        return check_launch("mbc_combine_backward_noalloc");
    }
    float* part = nullptr;
    if ((st = noalloc_scratch(&part)) != PMF_OK) return st;
    // every partial slot the reduction reads is written by k_combine_bwd_coeff
    // first, so the array needs no clearing between calls
    k_combine_bwd_mbc<<<stream_blocks(g.n), kThreads, 0, s>>>(g, L, P, coeff, d_dvf, d_mbc, accumulate);
    dim3 gr(kStreamBlocks, (unsigned)(P * 3));
    PMF_DISPATCH_DTYPE(dtype, T, k_combine_bwd_coeff<T><<<gr, kThreads, 0, s>>>(g, L, P, (const T*)mbc, d_dvf, part));
    const int64_t nout = (int64_t)P * L * 3;
    k_reduce_partials<<<(unsigned)((nout + 255) / 256), 256, 0, s>>>(part, nout, kStreamBlocks, d_coeff, accumulate);
    return check_launch("mbc_combine_backward_noalloc");
}
