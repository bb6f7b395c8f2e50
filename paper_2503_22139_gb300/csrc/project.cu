// Cone-beam ray marcher, forward (Eq. 6), and the L1/L2 projection loss
// (Eq. 10/12, Eq. 1) for sm_103a.  The chunk box of every lock-step chunk is
// staged in shared memory with coalesced loads (zero outside the grid), and
// the 8-corner trilinear gathers read shared memory; a chunk whose box does
// not fit falls back to bounds-checked global gathers.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "march.cuh"

namespace pmf {
namespace {

// ----------------------------------------------------------------- forward

// Capacity (floats) of the plain-staging box, in dynamic shared memory: a
// 48-sample chunk's box at the paper geometry, with rows of 33 floats (65 when
// the box is wider than 32 voxels, the same bank pattern).
constexpr int kPlainBox = 13312;

// The staged samples [j0, j1] of one ray on a box with rows PITCH floats apart
// and planes sz floats apart (PITCH a template argument, so the corner offsets
// are immediates).
template <int PITCH>
__device__ __forceinline__ void gather_samples(const Ray& r, const float* box, const Box& bx, int sz, int j0, int j1,
                                               const int ib[3], const float fb[3], float& acc) {
    // positions relative to the anchor cell; the box was bounded with the same
    // expression, so every cell is inside it
    constexpr int sy = PITCH;
    const float syf = (float)sy, szf = (float)sz;
    const float* qa = box + (ib[0] - bx.lx) + (ib[1] - bx.ly) * sy + (ib[2] - bx.lz) * sz;
    float jf = (float)j0;
    for (int j = j0; j <= j1; j++, jf += 1.0f) {
        const float ux = fmaf(jf, r.dh[0], fb[0]), uy = fmaf(jf, r.dh[1], fb[1]), uz = fmaf(jf, r.dh[2], fb[2]);
        const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
        const float fx = ux - flx, fy = uy - fly, fz = uz - flz;
        const float* q = qa + (int)fmaf(flz, szf, fmaf(fly, syf, flx));
        if (!PMF_DCHECK(q >= box && q + sz + sy + 1 < box + kPlainBox)) continue;
        const float c000 = q[0], c100 = q[1], c010 = q[sy], c110 = q[sy + 1];
        const float c001 = q[sz], c101 = q[sz + 1], c011 = q[sz + sy], c111 = q[sz + sy + 1];
        const float a00 = fmaf(fx, c100 - c000, c000), a10 = fmaf(fx, c110 - c010, c010);
        const float a01 = fmaf(fx, c101 - c001, c001), a11 = fmaf(fx, c111 - c011, c011);
        const float b0 = fmaf(fy, a10 - a00, a00), b1 = fmaf(fy, a11 - a01, a01);
        acc += fmaf(fz, b1 - b0, b0);  // into the tile's sum in sample order, as every path does
    }
}

// One 16 x (RPB/16) pixel tile of view p: every thread of the CTA calls it.
template <typename T, int CH, int RPB>
__device__ __forceinline__ void project_tile(const GridD& g, int nu, int nv, int ntu, float step,
                                             const pmf_view* __restrict__ views, const T* __restrict__ vol,
                                             int64_t vol_stride, float* __restrict__ proj, int p, int tile,
                                             float* box, BoxState& bs) {
    int a, b;
    pixel_of<RPB>(tile, ntu, a, b);
    const bool in = a < nu && b < nv;
    tile_view(bs, views[p], g, step);
    Ray r;
    if (in) {
        r = ray_init(bs.vf, nu, nv, a, b, g);
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
        const int pitch = bx.bx <= 32 ? 33 : 65;
        const int sz = pitch * bx.by;
        const bool fits = bx.vol > 0 && bx.bx <= 64 && (long long)bx.bz * sz <= kPlainBox;
        if (threadIdx.x == 0 && bx.vol > 0 && !fits) diag_count(PMF_DIAG_PROJECT_BOX_FALLBACK);
        if (fits) {
            // stage the box: lane = x (two passes when wider than 32), one warp
            // per (y, z) row, zero outside the grid
            for (int col = lane; col < bx.bx; col += 32) {
                const int x = bx.lx + col;
                const bool xin = (unsigned)x < (unsigned)g.nx;
                for (int zz = 0; zz < bx.bz; zz++) {
                    const int z = bx.lz + zz;
                    const bool zin = (unsigned)z < (unsigned)g.nz;
                    for (int yy = warp; yy < bx.by; yy += RPB / 32) {
                        const int y = bx.ly + yy;
                        float val = 0.0f;
                        if (xin && zin && (unsigned)y < (unsigned)g.ny)
                            val = Store<T>::ld(V, ((int64_t)z * g.ny + y) * g.nx + x);
                        const int i = zz * sz + yy * pitch + col;
                        if (PMF_DCHECK(i < kPlainBox)) box[i] = val;
                    }
                }
            }
            __syncthreads();
            if (act) {
                if (pitch == 33) gather_samples<33>(r, box, bx, sz, j0, j1, ib, fb, acc);
                else gather_samples<65>(r, box, bx, sz, j0, j1, ib, fb, acc);
            }
        } else if (act) {
            // the staged loop's own positions and blend, so that every path
            // (staged, bulk-copied, or gathered from global memory) gives the
            // same bits
            float jf = (float)j0;
            for (int j = j0; j <= j1; j++, jf += 1.0f) {
                const float ux = fmaf(jf, r.dh[0], fb[0]), uy = fmaf(jf, r.dh[1], fb[1]),
                            uz = fmaf(jf, r.dh[2], fb[2]);
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
    extern __shared__ __align__(128) float box[];  // kPlainBox floats
    __shared__ BoxState bs;
    project_tile<T, CH, RPB>(g, nu, nv, ntu, step, views, vol, vol_stride, proj, blockIdx.y, blockIdx.x, box, bs);
}

// ------------------------------------------- forward with bulk-copy staging
//
// fp32 volumes whose rows and planes are 16-byte multiples: each chunk's box
// is brought into shared memory by tensor-map bulk copies (cp.async.bulk.tensor)
// of 44 x 8 x 1 voxels, one per (z, 8-row block), issued by one thread and
// completed on an mbarrier; the copy engine fills voxels outside the grid with
// zeros, which is the zero padding of the trilinear interpolation.  The box's
// x origin x0 is rounded down to a multiple of 4 voxels (the copy start must
// be 16-byte aligned) and its y extent up to 8 rows.
//
// Bank layout: rows are 44 floats apart (12 banks) and, where the box is
// narrow enough, planes are S = 8k * 44 + 16 floats apart (16 banks), so the
// 4 x 4 x 2 voxels around any point fall in 32 distinct banks and a warp's
// gathers do not conflict.  Copy destinations must be 128-byte aligned, so
// the +16 is made by shifting odd planes' copies 16 voxels to the left in x:
// plane z lands at z S - 16 (z & 1), and voxel (x, y, z) is always at
// (x - x0) + 44 y + S z.  A box too wide for the shift uses S = 8k * 44;
// one larger than kTmaBox falls back to bounds-checked global gathers (52 KB:
// at the paper geometry no 48-sample chunk's box is larger, and four CTAs of
// 256 rays, the register limit, still fit an SM).  The
// wait is bounded (about one second of clock): a CTA that gives up counts
// PMF_DIAG_TIMEOUT, waits once more for its copies, writes NaN to its pixels
// and returns.
constexpr int kTmaX = 44;                     // floats per staged row (one copy's x extent)
constexpr int kTmaRows = 8;                   // rows per copy
constexpr int kTmaSkew = 16;                  // extra plane stride (floats) of the conflict-free layout
constexpr int kTmaBox = 13312;                // staged floats (52 KB of dynamic shared memory)
constexpr long long kTmaWaitCycles = 2000000000LL;
constexpr long long kStallWaitCycles = 200000LL;  // the test hook's short limit (~0.1 ms)

// Test hook (pmf_debug_stall_bulk_copies): while non-zero, the per-volume
// bulk-copy projector arms its mbarrier for a chunk's bytes but issues no copy,
// so its bounded wait runs out with nothing in flight.  Zero in normal use.
static __device__ int g_stall_copies;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of bar, at most `limit` clock cycles; true if it completed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void tma_load_4d(float* dst, const CUtensorMap* map, int x, int y, int z, int p,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(p), "r"(smem_u32(bar))
        : "memory");
}

// Returns false (after writing NaN to its pixels) when a bulk copy did not
// complete within the bounded wait; the mbarrier's phase is then unknown and
// the CTA must not stage again.  `parity` is the barrier phase the CTA's next
// copy completes, carried across tiles by persistent callers.  `stall` (the
// test hook) arms the barrier without issuing the copies and waits at most
// kStallWaitCycles.
template <int CH, int RPB>
__device__ __forceinline__ bool project_tile_tma(const GridD& g, int nu, int nv, int ntu, float step,
                                                 const pmf_view* __restrict__ views, const CUtensorMap* map,
                                                 const float* __restrict__ vol, int64_t vol_stride,
                                                 float* __restrict__ proj, int p, int tile, float* box,
                                                 unsigned long long* bar, BoxState& bs, unsigned& parity,
                                                 bool stall = false) {
    const long long limit = stall ? kStallWaitCycles : kTmaWaitCycles;
    int a, b;
    pixel_of<RPB>(tile, ntu, a, b);
    const bool in = a < nu && b < nv;
    tile_view(bs, views[p], g, step);
    Ray r;
    if (in) {
        r = ray_init(bs.vf, nu, nv, a, b, g);
    } else {
        r.mlo = 1; r.mhi = 0;
    }
    const bool live = in && r.mlo <= r.mhi;
    const float* V = vol + (int64_t)p * vol_stride;
    const int pv = vol_stride ? p : 0;  // the volume's index along the map's 4th axis
    block_range(bs, r, live);
    const int Mlo = bs.range[0], Mhi = bs.range[1];
    float acc = 0.0f;
    int sel = 0;
    for (int M0 = Mlo; M0 <= Mhi; M0 += CH, sel ^= 1) {
        int j0, j1, ib[3];
        float fb[3];
        const bool act = chunk_begin<CH>(bs, sel, r, live, M0, j0, j1, ib, fb);
        __syncthreads();
        const Box bx = read_box(bs, sel);
        const int x0 = (bx.lx >> 2) << 2;                   // 16-byte aligned copy start (floor)
        const int byr = (bx.by + kTmaRows - 1) & ~(kTmaRows - 1);
        const int span = bx.bx + (bx.lx - x0);              // floats of each row the samples read
        const int skew = span + kTmaSkew <= kTmaX && (long long)bx.bz * (byr * kTmaX + kTmaSkew) <= kTmaBox
                             ? kTmaSkew : 0;
        const int S = byr * kTmaX + skew;                   // plane stride in the box
        const bool fits = bx.vol > 0 && span <= kTmaX && (long long)bx.bz * S <= kTmaBox;
        if (threadIdx.x == 0 && bx.vol > 0 && !fits) diag_count(PMF_DIAG_PROJECT_BOX_FALLBACK);
        if (fits) {
            if (threadIdx.x == 0) {
                // the previous chunk's reads of the box are ordered before the
                // copies into it by the barrier above and this proxy fence
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const int nyb = byr / kTmaRows;
                mbar_expect_tx(bar, (unsigned)(bx.bz * nyb * kTmaRows * kTmaX * sizeof(float)));
                for (int zz = 0; zz < (stall ? 0 : bx.bz); zz++) {
                    const int sh = skew * (zz & 1);  // a multiple of 4 voxels: the copy start stays aligned
                    for (int yb = 0; yb < nyb; yb++) {
                        float* dst = box + zz * S - sh + yb * kTmaRows * kTmaX;
                        // a skipped copy leaves the barrier short of bytes: the bounded wait then reports it
                        if (PMF_DCHECK(dst >= box && dst + kTmaRows * kTmaX <= box + kTmaBox))
                            tma_load_4d(dst, map, x0 - sh, bx.ly + yb * kTmaRows, bx.lz + zz, pv, bar);
                    }
                }
            }
            const bool ok = mbar_wait_bounded(bar, parity, limit);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) diag_count(PMF_DIAG_TIMEOUT);
                // the copies may still be in flight into this CTA's shared
                // memory: wait for them once more, four times as long, before
                // the CTA exits (with the test hook none was issued)
                mbar_wait_bounded(bar, parity ^ 1u, 4 * limit);
                if (in) proj[((int64_t)p * nv + b) * nu + a] = __int_as_float(0x7fc00000);
                return false;
            }
            if (act) {
                const float syf = (float)kTmaX, szf = (float)S;
                const int sy = kTmaX, sz = S;
                const float* qa = box + (ib[0] - x0) + (ib[1] - bx.ly) * sy + (ib[2] - bx.lz) * sz;
                // the staged loop's arithmetic with the x/y position and the
                // z-paired blends in packed fp32 pairs (same bits, fewer
                // instructions): (a00, a01), (a10, a11), then (b0, b1)
                const f32x2 dxy = pack2(r.dh[0], r.dh[1]), bxy = pack2(fb[0], fb[1]), one = pack2(1.0f, 1.0f);
                f32x2 jj = pack2((float)j0, (float)j0);
#pragma unroll 2  // two samples' dependency chains interleave (measured 2% faster)
                for (int j = j0; j <= j1; j++, jj = add2(jj, one)) {
                    const f32x2 uxy = fma2(jj, dxy, bxy);
                    const float ux = lo2(uxy), uy = hi2(uxy), uz = fmaf(lo2(jj), r.dh[2], fb[2]);
                    const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
                    const f32x2 fxy = sub2(uxy, pack2(flx, fly));
                    const float fx = lo2(fxy), fy = hi2(fxy), fz = uz - flz;
                    const float* q = qa + (int)fmaf(flz, szf, fmaf(fly, syf, flx));
                    if (!PMF_DCHECK(q >= box && q + sz + sy + 1 < box + kTmaBox)) continue;
                    const f32x2 c00 = pack2(q[0], q[sz]), c10 = pack2(q[1], q[sz + 1]);
                    const f32x2 c01 = pack2(q[sy], q[sz + sy]), c11 = pack2(q[sy + 1], q[sz + sy + 1]);
                    const f32x2 fx2 = pack2(fx, fx);
                    const f32x2 a0 = fma2(fx2, sub2(c10, c00), c00), a1 = fma2(fx2, sub2(c11, c01), c01);
                    const f32x2 bb = fma2(pack2(fy, fy), sub2(a1, a0), a0);
                    const float b0 = lo2(bb), b1 = hi2(bb);
                    acc += fmaf(fz, b1 - b0, b0);
                }
            }
        } else if (act) {
            // the staged loop's own positions and blend, so that every path
            // (staged, bulk-copied, or gathered from global memory) gives the
            // same bits
            float jf = (float)j0;
            for (int j = j0; j <= j1; j++, jf += 1.0f) {
                const float ux = fmaf(jf, r.dh[0], fb[0]), uy = fmaf(jf, r.dh[1], fb[1]),
                            uz = fmaf(jf, r.dh[2], fb[2]);
                const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
                acc += gather8(V, g, ib[0] + (int)flx, ib[1] + (int)fly, ib[2] + (int)flz, ux - flx, uy - fly,
                               uz - flz);
            }
        }
        __syncthreads();
    }
    if (in) proj[((int64_t)p * nv + b) * nu + a] = step * acc;
    return true;
}

template <int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_project_tma(GridD g, int nu, int nv, int ntu, float step,
                                                                const pmf_view* __restrict__ views,
                                                                const __grid_constant__ CUtensorMap map,
                                                                const float* __restrict__ vol, int64_t vol_stride,
                                                                float* __restrict__ proj) {
    extern __shared__ __align__(128) float box[];  // kTmaBox floats
    __shared__ __align__(8) unsigned long long bar;
    __shared__ BoxState bs;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;
    const bool stall = *(volatile int*)&g_stall_copies != 0;
    project_tile_tma<CH, RPB>(g, nu, nv, ntu, step, views, &map, vol, vol_stride, proj, blockIdx.y, blockIdx.x, box,
                              &bar, bs, parity, stall);
}

// The uneven batch of fp32 volumes with bulk-copy staging: one tensor map per
// item in the launch's parameter block, the mbarrier's phase carried from
// tile to tile.
struct ProjBatchTma {
    ProjBatch B;
    CUtensorMap map[kMaxItems];
};

template <int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_project_batched_tma(const __grid_constant__ ProjBatchTma T) {
    extern __shared__ __align__(128) float box[];  // kTmaBox floats
    __shared__ __align__(8) unsigned long long bar;
    __shared__ BoxState bs;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;
    for (int64_t w = blockIdx.x; w < T.B.total; w += gridDim.x) {
        const int i = find_item(T.B, w);
        const ProjItem& it = T.B.it[i];
        const int local = (int)(w - it.begin);  // < 2^31: checked when the item is filled
        if (!project_tile_tma<CH, RPB>(it.g, it.nu, it.nv, it.ntu, it.step, it.views, &T.map[i], (const float*)it.vol,
                                       it.vol_stride, it.proj, local / it.ntiles, local % it.ntiles, box,
                                       &bar, bs, parity))
            return;
        __syncthreads();
    }
}

template <typename T, int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_project_batched(const __grid_constant__ ProjBatch B) {
    extern __shared__ __align__(128) float box[];  // kPlainBox floats
    __shared__ BoxState bs;
    for (int64_t w = blockIdx.x; w < B.total; w += gridDim.x) {
        const ProjItem it = B.it[find_item(B, w)];  // a copy: the tile code reads registers, not the parameter block
        const int local = (int)(w - it.begin);  // < 2^31: checked when the item is filled
        project_tile<T, CH, RPB>(it.g, it.nu, it.nv, it.ntu, it.step, it.views, (const T*)it.vol, it.vol_stride, it.proj,
                        local / it.ntiles, local % it.ntiles, box, bs);
        __syncthreads();
    }
}

// One work item per CTA (the default launch): the same tiles, without the
// work-list loop.
template <int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_project_batched_tma1(const __grid_constant__ ProjBatchTma T) {
    extern __shared__ __align__(128) float box[];  // kTmaBox floats
    __shared__ __align__(8) unsigned long long bar;
    __shared__ BoxState bs;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;
    const int64_t w = blockIdx.x;
    const int i = find_item(T.B, w);
    const ProjItem& it = T.B.it[i];
    const int local = (int)(w - it.begin);
    project_tile_tma<CH, RPB>(it.g, it.nu, it.nv, it.ntu, it.step, it.views, &T.map[i], (const float*)it.vol,
                              it.vol_stride, it.proj, local / it.ntiles, local % it.ntiles, box, &bar, bs, parity);
}

template <typename T, int CH, int RPB>
__global__ void __launch_bounds__(RPB, 1024 / RPB) k_project_batched1(const __grid_constant__ ProjBatch B) {
    extern __shared__ __align__(128) float box[];  // kPlainBox floats
    __shared__ BoxState bs;
    const int64_t w = blockIdx.x;
    const ProjItem it = B.it[find_item(B, w)];
    const int local = (int)(w - it.begin);
    project_tile<T, CH, RPB>(it.g, it.nu, it.nv, it.ntu, it.step, it.views, (const T*)it.vol, it.vol_stride, it.proj,
                    local / it.ntiles, local % it.ntiles, box, bs);
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return (PFN_cuTensorMapEncodeTiled_v12000)f;
    }();
    return fn;
}

// A 4-D map (x, y, z, volume) over fp32 volumes for the staged forward, or
// false when the layout does not allow bulk copies (base or a stride not a
// multiple of 16 bytes) or the encoder is unavailable.
bool encode_volume_map(CUtensorMap* m, const float* vol, const pmf_grid* g, int32_t P, int64_t vol_stride) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)vol & 15u) != 0) return false;
    const cuuint64_t nx = (cuuint64_t)g->nx, ny = (cuuint64_t)g->ny, nz = (cuuint64_t)g->nz;
    const cuuint64_t vstride = vol_stride ? (cuuint64_t)vol_stride * 4 : nx * ny * nz * 4;
    if ((nx * 4) % 16 || (nx * ny * 4) % 16 || vstride % 16) return false;
    const cuuint64_t dims[4] = {nx, ny, nz, vol_stride ? (cuuint64_t)P : 1};
    const cuuint64_t strides[3] = {nx * 4, nx * ny * 4, vstride};
    const cuuint32_t box[4] = {kTmaX, kTmaRows, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)vol, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// (chunk, rays) -> the projector's kernels, whose chunks may also be 48
// samples long
#define PMF_DISPATCH_PROJ(sh, CH, RPB, ...)                                                                    \
    switch ((sh).chunk * 1000 + (sh).rays) {                                                                \
        case 48256: { constexpr int CH = 48, RPB = 256; __VA_ARGS__; break; }                               \
        case 48128: { constexpr int CH = 48, RPB = 128; __VA_ARGS__; break; }                               \
        case 32256: { constexpr int CH = 32, RPB = 256; __VA_ARGS__; break; }                               \
        case 32128: { constexpr int CH = 32, RPB = 128; __VA_ARGS__; break; }                               \
        case 16256: { constexpr int CH = 16, RPB = 256; __VA_ARGS__; break; }                               \
        case 16128: { constexpr int CH = 16, RPB = 128; __VA_ARGS__; break; }                               \
        default: return set_error(PMF_EINVAL, "unsupported march shape: chunk %d, rays %d", (sh).chunk, (sh).rays); \
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
    CUtensorMap map;
    if (sh.tma && dtype == PMF_F32 && encode_volume_map(&map, (const float*)vol, grid, P, vol_stride)) {
        PMF_DISPATCH_PROJ(sh, CH, RPB, {
            cudaFuncSetAttribute(k_project_tma<CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kTmaBox * sizeof(float)));
            k_project_tma<CH, RPB><<<gr, RPB, kTmaBox * sizeof(float), s>>>(g, det->nu, det->nv, ntu, det->step_mm, views, map,
                                                                           (const float*)vol, vol_stride, proj);
        });
        return check_launch("conebeam_project");
    }
    PMF_DISPATCH_PROJ(sh, CH, RPB, PMF_DISPATCH_DTYPE(dtype, T, {
        cudaFuncSetAttribute(k_project<T, CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kPlainBox * sizeof(float)));
        k_project<T, CH, RPB><<<gr, RPB, kPlainBox * sizeof(float), s>>>(g, det->nu, det->nv, ntu, det->step_mm, views,
                                                                        (const T*)vol, vol_stride, proj);
    }));
    return check_launch("conebeam_project");
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
    int ord[kMaxItems];
    longest_first(n, items, ord);  // work-list position k holds item ord[k]
    for (int k = 0; k < n; k++) {
        const pmf_project_item& in = items[ord[k]];
        if ((st = fill_item(in, total, sh.rays, B.it[k])) != PMF_OK) return st;
        PMF_REQUIRE(in.P == 0 || (in.vol && in.proj), "item %d: null pointer", ord[k]);
        B.it[k].vol = in.vol;
        B.it[k].proj = in.proj;
        total += (int64_t)B.it[k].ntiles * in.P;
    }
    B.total = total;
    if (total == 0) return PMF_OK;
    int ntl[kMaxItems];
    for (int i = 0; i < n; i++) ntl[i] = B.it[i].ntiles;
    const unsigned nc = persistent_ctas(total, ctas, sh.rays, ntl, n);
    if (sh.tma && dtype == PMF_F32) {
        ProjBatchTma tb{};
        bool all = true;
        for (int k = 0; k < n && all; k++) {
            const pmf_project_item& in = items[ord[k]];
            all = in.P == 0 || encode_volume_map(&tb.map[k], (const float*)in.vol, &in.grid, in.P, in.vol_stride);
        }
        if (all) {
            tb.B = B;
            PMF_DISPATCH_PROJ(sh, CH, RPB, {
                if ((int64_t)nc == total) {
                    cudaFuncSetAttribute(k_project_batched_tma1<CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kTmaBox * sizeof(float)));
                    k_project_batched_tma1<CH, RPB><<<nc, RPB, kTmaBox * sizeof(float), s>>>(tb);
                } else {
                    cudaFuncSetAttribute(k_project_batched_tma<CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kTmaBox * sizeof(float)));
                    k_project_batched_tma<CH, RPB><<<nc, RPB, kTmaBox * sizeof(float), s>>>(tb);
                }
            });
            return check_launch("conebeam_project_batched");
        }
    }
    PMF_DISPATCH_PROJ(sh, CH, RPB, PMF_DISPATCH_DTYPE(dtype, T, {
        if ((int64_t)nc == total) {
            cudaFuncSetAttribute(k_project_batched1<T, CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kPlainBox * sizeof(float)));
            k_project_batched1<T, CH, RPB><<<nc, RPB, kPlainBox * sizeof(float), s>>>(B);
        } else {
            cudaFuncSetAttribute(k_project_batched<T, CH, RPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kPlainBox * sizeof(float)));
            k_project_batched<T, CH, RPB><<<nc, RPB, kPlainBox * sizeof(float), s>>>(B);
        }
    }));
    return check_launch("conebeam_project_batched");
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

}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status conebeam_project(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views,
                            pmf_dtype dtype, const void* vol, int64_t vol_stride, float* proj, pmf_stream stream) {
    return project_grid(grid, det, P, views, dtype, vol, vol_stride, proj, default_project_shape(), (cudaStream_t)stream);
}

pmf_status conebeam_project_batched(int32_t n, const pmf_project_item* items, pmf_dtype dtype, pmf_stream stream) {
    return project_batched_impl(n, items, dtype, default_project_shape(), 0, (cudaStream_t)stream);
}

pmf_status pmf_debug_stall_bulk_copies(int32_t on) {
    const int v = on ? 1 : 0;
    cudaError_t e = cudaMemcpyToSymbol(g_stall_copies, &v, sizeof(v));
    if (e != cudaSuccess) return set_error(PMF_ECUDA, "pmf_debug_stall_bulk_copies: %s", cudaGetErrorString(e));
    return PMF_OK;
}

}  // extern "C"
