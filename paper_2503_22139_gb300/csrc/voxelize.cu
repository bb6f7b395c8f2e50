// Tile-binned Gaussian voxelizer (Eq. 4-5 and the signed MBC variant of
// Sec. 2.3.1) and its adjoint, for sm_103a.
//
// Forward: (1) per Gaussian, the inverse covariance and the voxel box of its
// truncation ellipsoid; count the 8x8x8 tiles it overlaps; (2) exclusive scan
// of the per-tile counts; (3) fill per-tile Gaussian lists; (4) one CTA per
// tile stages its list in shared memory and sums every entry at its 512 voxel
// centres.  Sums are exact integers at the scale 2^k with max|value| 2^k < 2^21:
// each term is rounded once to an integer (magic-number add), a batch of at
// most 256 terms is summed in 32 bits (< 2^29) and batches are added in 64
// bits, so the unordered list fill cannot change a bit of the result.
//
// Backward: one CTA per Gaussian walks its voxel box, accumulates
// sum_v dL/dout_c * e, and the moments S1 = sum w d, S2 = sum w d d^T
// (w = e * sum_c value_c dL/dout_c), reduces them in a fixed order, and turns
// them into d mean = A S1, d scale_j = (R^T S2 R)_jj / s_j^3,
// dR = -S2 R diag(1/s^2), then d quaternion through R(q/|q|).
#include "pmf_common.cuh"

namespace pmf {
namespace {

// Bin tiles: the render takes one CTA per tile of TX x TY x TZ voxels, each
// warp a 4 x 4 x 4 sub-block (two voxels per lane), so a tile has
// TX TY TZ / 2 threads; at most 512, so that a batch of that many rounded terms
// stays below 2^30 in 32 bits.  8^3 is the default; plans may take another
// from the autotuner.  Every tile gives the same bits (the sums are exact).
struct VoxTile {
    int x, y, z;
};
constexpr VoxTile kDefaultTile{8, 8, 8};

bool supported_tile(const VoxTile& t) {
    return (t.x == 8 && t.y == 8 && t.z == 8) || (t.x == 16 && t.y == 8 && t.z == 8) ||
           (t.x == 8 && t.y == 8 && t.z == 4) || (t.x == 16 && t.y == 8 && t.z == 4);
}
constexpr int kMaxC = 4;
constexpr float kNegHalfLog2e = -0.72134752044448170368f;  // -log2(e)/2
constexpr float kMagicF = 12582912.0f;  // 1.5 * 2^23: x + kMagicF rounds x to an integer for |x| < 2^22
constexpr int kMagicI = 0x4b400000;     // its bit pattern

// Scale exponent k with m 2^k < 2^21 (m = the largest |value|; 0 if m is 0 or
// not finite).
__device__ __forceinline__ int term_exponent(float m) {
    if (!(m > 0.0f) || !isfinite(m)) return 0;
    int e;
    frexpf(m, &e);  // m < 2^e
    const int k = 21 - e;
    return k > 126 ? 126 : (k < -126 ? -126 : k);
}

struct VoxHeader {
    unsigned int max_abs_bits;  // max |value| over all Gaussians and channels (float bits)
    unsigned int pad;
    long long total_pairs;
};

struct VoxWs {
    VoxHeader* hdr;
    float* prm;        // [10][G]: mx my mz a00 a11 a22 b01 b02 b12 (b = 2 a) and k2
    int* box;          // [6][G]: voxel lo xyz, hi xyz (lo > hi: empty)
    unsigned* tcount;  // [T]
    unsigned* toff;    // [T+1]
    unsigned* cursor;  // [T]
    unsigned* list;    // [capacity]
    int64_t capacity;
};

struct TileGeom {
    int tx, ty, tz;
    int64_t t;
};

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

size_t vox_ws_layout(const GridD& g, int64_t G, int64_t capacity, const VoxTile& tl, VoxWs* w, char* base) {
    int tx = ceil_div(g.nx, tl.x), ty = ceil_div(g.ny, tl.y), tz = ceil_div(g.nz, tl.z);
    int64_t T = (int64_t)tx * ty * tz;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return base ? base + o : nullptr; };
    VoxWs x;
    x.hdr = (VoxHeader*)take(sizeof(VoxHeader));
    x.prm = (float*)take(sizeof(float) * 10 * (size_t)(G > 0 ? G : 1));
    x.box = (int*)take(sizeof(int) * 6 * (size_t)(G > 0 ? G : 1));
    x.tcount = (unsigned*)take(sizeof(unsigned) * (size_t)T);
    x.toff = (unsigned*)take(sizeof(unsigned) * (size_t)(T + 1));
    x.cursor = (unsigned*)take(sizeof(unsigned) * (size_t)T);
    x.list = (unsigned*)take(sizeof(unsigned) * (size_t)(capacity > 0 ? capacity : 1));
    x.capacity = capacity;
    if (w) *w = x;
    return off;
}

// Per-Gaussian setup shared by forward and backward so that both take the
// same truncation decisions: rotation of the normalised quaternion, inverse
// covariance A = R diag(1/s^2) R^T, and the voxel box of {q <= kappa^2}.
struct GaussSetup {
    float mu[3], s[3], qn[4], qnorm, R[9];
    float a00, a11, a22, b01, b02, b12;  // q = a00 dx^2 + a11 dy^2 + a22 dz^2 + b01 dx dy + b02 dx dz + b12 dy dz
    int lo[3], hi[3];
};

__device__ __forceinline__ void gauss_setup(const pmf_gaussians& G, int64_t i, const GridD& g, float kappa,
                                            GaussSetup& o) {
    o.mu[0] = __ldg(G.mean + 3 * i); o.mu[1] = __ldg(G.mean + 3 * i + 1); o.mu[2] = __ldg(G.mean + 3 * i + 2);
    o.s[0] = __ldg(G.scale + 3 * i); o.s[1] = __ldg(G.scale + 3 * i + 1); o.s[2] = __ldg(G.scale + 3 * i + 2);
    float qw = __ldg(G.quat + 4 * i), qx = __ldg(G.quat + 4 * i + 1), qy = __ldg(G.quat + 4 * i + 2),
          qz = __ldg(G.quat + 4 * i + 3);
    float nrm = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    float inv = 1.0f / nrm;
    float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
    o.qn[0] = w; o.qn[1] = x; o.qn[2] = y; o.qn[3] = z; o.qnorm = nrm;
    float* R = o.R;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    float is2[3] = {1.f / (o.s[0] * o.s[0]), 1.f / (o.s[1] * o.s[1]), 1.f / (o.s[2] * o.s[2])};
    float A[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            A[a][b] = R[3 * a] * R[3 * b] * is2[0] + R[3 * a + 1] * R[3 * b + 1] * is2[1] +
                      R[3 * a + 2] * R[3 * b + 2] * is2[2];
    o.a00 = A[0][0]; o.a11 = A[1][1]; o.a22 = A[2][2];
    o.b01 = A[0][1] + A[1][0]; o.b02 = A[0][2] + A[2][0]; o.b12 = A[1][2] + A[2][1];
    const int n[3] = {g.nx, g.ny, g.nz};
    const float iv[3] = {g.ivx, g.ivy, g.ivz};
    for (int a = 0; a < 3; a++) {
        float var = R[3 * a] * R[3 * a] * o.s[0] * o.s[0] + R[3 * a + 1] * R[3 * a + 1] * o.s[1] * o.s[1] +
                    R[3 * a + 2] * R[3 * a + 2] * o.s[2] * o.s[2];
        float half = kappa * sqrtf(var);
        float c = o.mu[a] * iv[a] + 0.5f * (float)n[a] - 0.5f;
        float l = floorf(c - half * iv[a]) - 1.0f, h = ceilf(c + half * iv[a]) + 1.0f;
        // clamp to the grid; fmaxf/fminf drop a NaN operand, so a NaN box comes out empty
        l = fminf(fmaxf(l, 0.0f), (float)n[a]);
        h = fminf(fmaxf(h, -1.0f), (float)(n[a] - 1));
        o.lo[a] = (int)l;
        o.hi[a] = (int)h;
    }
}

// The quadratic form, written with explicit fused multiply-adds so every
// kernel that calls it rounds identically.
__device__ __forceinline__ float qform(float dx, float dy, float dz, float a00, float a11, float a22, float b01,
                                       float b02, float b12) {
    float tx = __fmaf_rn(a00, dx, __fmaf_rn(b01, dy, __fmul_rn(b02, dz)));
    float ty = __fmaf_rn(a11, dy, __fmul_rn(b12, dz));
    return __fmaf_rn(dx, tx, __fmaf_rn(dy, ty, __fmul_rn(__fmul_rn(a22, dz), dz)));
}

// Voxel-centre coordinate (i + 1/2 - n/2) v, rounded the same way everywhere.
__device__ __forceinline__ float centre(int i, int n, float v) {
    return __fmul_rn(__fsub_rn(__fadd_rn((float)i, 0.5f), __fmul_rn(0.5f, (float)n)), v);
}

// ------------------------------------------------------------- forward

// One warp per Gaussian: lane 0 stores the setup, all lanes count tiles.
__global__ void k_prep(pmf_gaussians G, GridD g, float kappa, VoxWs w, VoxTile tl, int ntx, int nty) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= G.n) return;
    GaussSetup s;
    gauss_setup(G, i, g, kappa, s);
    const int64_t n = G.n;
    if (lane == 0) {
        float k2 = isinf(kappa) ? INFINITY : kappa * kappa;
        float* p = w.prm;
        p[0 * n + i] = s.mu[0]; p[1 * n + i] = s.mu[1]; p[2 * n + i] = s.mu[2];
        p[3 * n + i] = s.a00; p[4 * n + i] = s.a11; p[5 * n + i] = s.a22;
        p[6 * n + i] = s.b01; p[7 * n + i] = s.b02; p[8 * n + i] = s.b12; p[9 * n + i] = k2;
        for (int a = 0; a < 3; a++) { w.box[a * n + i] = s.lo[a]; w.box[(3 + a) * n + i] = s.hi[a]; }
        unsigned m = 0u;  // abs_bits keeps a NaN or infinite value visible
        for (int c = 0; c < G.channels; c++) m = max(m, abs_bits(__ldg(G.value + i * G.channels + c)));
        if (m) atomicMax(&w.hdr->max_abs_bits, m);
    }
    if (s.lo[0] > s.hi[0] || s.lo[1] > s.hi[1] || s.lo[2] > s.hi[2]) return;
    const int t0x = s.lo[0] / tl.x, t1x = s.hi[0] / tl.x, t0y = s.lo[1] / tl.y, t1y = s.hi[1] / tl.y,
              t0z = s.lo[2] / tl.z, t1z = s.hi[2] / tl.z;
    const int ex = t1x - t0x + 1, ey = t1y - t0y + 1, ez = t1z - t0z + 1;
    const int cnt = ex * ey * ez;
    for (int c = lane; c < cnt; c += 32) {
        int x = t0x + c % ex, y = t0y + (c / ex) % ey, z = t0z + c / (ex * ey);
        atomicAdd(&w.tcount[((int64_t)z * nty + y) * ntx + x], 1u);
    }
}

// Exclusive scan of the tile counts in one CTA (T is at most a few 1e5).
__global__ void k_scan(VoxWs w, int64_t T) {
    __shared__ unsigned long long part[1024];
    const int tid = threadIdx.x;
    const int64_t per = (T + 1023) / 1024;
    const int64_t b = tid * per, e = b + per < T ? b + per : T;
    unsigned long long s = 0;
    for (int64_t i = b; i < e; i++) s += w.tcount[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < 1024; i++) { unsigned long long v = part[i]; part[i] = run; run += v; }
        w.hdr->total_pairs = (long long)run;
    }
    __syncthreads();
    unsigned long long run = part[tid];
    for (int64_t i = b; i < e; i++) {
        w.toff[i] = (unsigned)(run > 0xffffffffull ? 0xffffffffull : run);
        run += w.tcount[i];
    }
    if (tid == 1023) w.toff[T] = (unsigned)(run > 0xffffffffull ? 0xffffffffull : run);
}

__global__ void k_fill(int64_t n, VoxWs w, VoxTile tl, int ntx, int nty) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) { lo[a] = w.box[a * n + i]; hi[a] = w.box[(3 + a) * n + i]; }
    if (lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2]) return;
    const int t0x = lo[0] / tl.x, t0y = lo[1] / tl.y, t0z = lo[2] / tl.z;
    const int ex = hi[0] / tl.x - t0x + 1, ey = hi[1] / tl.y - t0y + 1, ez = hi[2] / tl.z - t0z + 1;
    const int cnt = ex * ey * ez;
    for (int c = lane; c < cnt; c += 32) {
        int x = t0x + c % ex, y = t0y + (c / ex) % ey, z = t0z + c / (ex * ey);
        int64_t t = ((int64_t)z * nty + y) * ntx + x;
        unsigned pos = atomicAdd(&w.cursor[t], 1u);
        unsigned long long at = (unsigned long long)w.toff[t] + pos;
        if ((long long)at < w.capacity) w.list[at] = (unsigned)i;
    }
}

template <typename T, int C, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ / 2) k_render(pmf_gaussians G, GridD g, VoxWs w, T* out, int ntx,
                                                             int nty) {
    constexpr int NT = TX * TY * TZ / 2;              // threads: two voxels each
    constexpr int SX = TX / 4, SY = TY / 4, SZ = TZ / 4;  // 4^3 sub-blocks per axis, one per warp
    static_assert(TX % 4 == 0 && TY % 4 == 0 && TZ % 4 == 0 && NT <= 512 && SX * SY * SZ <= 32, "bin tile");
    // each staged Gaussian as float4 records, read by the warps with broadcast
    // 16-byte loads; the mean and the quadratic-form coefficients are stored
    // twice, as the packed pairs the two voxels of a thread use:
    // (mx, mx, my, my), (mz, mz, a00, a00), (a11, a11, a22, a22),
    // (b01, b01, b02, b02), (b12, b12, the sub-blocks of the tile its box
    // touches (bits), value_0 2^k), then (value_1..3 2^k) when C > 1
    constexpr int NR = C > 1 ? 6 : 5;
    extern __shared__ float4 vsm[];
    float4* rec = vsm;  // [NR][NT]
    unsigned* sidx = reinterpret_cast<unsigned*>(vsm + NR * NT);
    __shared__ int scount;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t t = blockIdx.x;
    const int tx = (int)(t % ntx), ty = (int)((t / ntx) % nty), tz = (int)(t / ((int64_t)ntx * nty));
    // warp w takes sub-block w of the tile (a 4^3 cube); each lane two voxels
    const int wx = warp % SX, wy = (warp / SX) % SY, wz = warp / (SX * SY);
    const int ix = tx * TX + 4 * wx + (lane & 3), iy = ty * TY + 4 * wy + ((lane >> 2) & 3);
    const int iz0 = tz * TZ + 4 * wz + (lane >> 4), iz1 = iz0 + 2;
    const float cx = centre(ix, g.nx, g.vx), cy = centre(iy, g.ny, g.vy);
    const float cz0 = centre(iz0, g.nz, g.vz), cz1 = centre(iz1, g.nz, g.vz);
    const f32x2 cxx = pack2(cx, cx), cyy = pack2(cy, cy), czz = pack2(cz0, cz1);
    const f32x2 nhl = pack2(kNegHalfLog2e, kNegHalfLog2e);
    const float k2 = isinf(G.kappa) ? INFINITY : G.kappa * G.kappa;  // k_prep's kappa^2

    const float maxabs = __uint_as_float(w.hdr->max_abs_bits);
    const bool bad = !isfinite(maxabs);  // a NaN or infinite value: the output is NaN
    if (bad && t == 0 && tid == 0) diag_count(PMF_DIAG_NONFINITE);
    // every term |value e^{-q/2}| 2^k < 2^21, so it rounds with the magic add
    // and a batch of at most 512 terms stays below 2^30 in 32 bits
    const int kexp = term_exponent(maxabs);
    const float scale = ldexpf(1.0f, kexp), inv_scale = ldexpf(1.0f, -kexp);

    long long acc0[C], acc1[C];
#pragma unroll
    for (int c = 0; c < C; c++) { acc0[c] = 0; acc1[c] = 0; }

    const int64_t n = G.n;
    const unsigned cnt = w.tcount[t];
    const unsigned long long off = w.toff[t];
    const bool listed = (long long)(off + cnt) <= w.capacity && w.toff[t] != 0xffffffffu;
    if (!listed && tid == 0) diag_count(PMF_DIAG_VOXELIZE_LIST_OVERFLOW);
    // Listed tiles walk their own list; overflowed tiles scan every Gaussian's box.
    const int64_t total = listed ? (int64_t)cnt : n;
    const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
    for (int64_t base = 0; base < total; base += NT) {
        __syncthreads();
        if (tid == 0) scount = 0;
        __syncthreads();
        const int64_t k = base + tid;
        if (k < total) {
            unsigned gi;
            bool take;
            if (listed) {
                gi = PMF_DCHECK((long long)(off + k) < w.capacity) ? w.list[off + k] : 0u;
                take = true;
            } else {
                gi = (unsigned)k;
                int lx = w.box[k], ly = w.box[n + k], lz = w.box[2 * n + k];
                int hx = w.box[3 * n + k], hy = w.box[4 * n + k], hz = w.box[5 * n + k];
                take = lx <= hx && ly <= hy && lz <= hz && lx <= x0 + TX - 1 && hx >= x0 && ly <= y0 + TY - 1 &&
                       hy >= y0 && lz <= z0 + TZ - 1 && hz >= z0;
            }
            if (take) {
                int slot = listed ? tid : atomicAdd(&scount, 1);
                if (PMF_DCHECK(slot < NT)) sidx[slot] = gi;
            }
        }
        if (listed) {
            if (tid == 0) scount = (int)((total - base) < NT ? (total - base) : NT);
        }
        __syncthreads();
        const int m = scount;
        if (tid < m) {
            unsigned gi = sidx[tid];
            float f[10], v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 10; k++) f[k] = w.prm[(int64_t)k * n + gi];
#pragma unroll
            for (int c = 0; c < C; c++) v[c] = __ldg(G.value + (int64_t)gi * C + c) * scale;
            // which 4-voxel slices of the tile the box reaches on each axis,
            // then the sub-blocks (bit w: warp w's)
            const int o[3] = {x0, y0, z0}, ns[3] = {SX, SY, SZ};
            unsigned slices[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int lo = w.box[(int64_t)a * n + gi], hi = w.box[(int64_t)(3 + a) * n + gi];
                slices[a] = 0u;
                for (int k = 0; k < ns[a]; k++)
                    if (lo <= o[a] + 4 * k + 3 && hi >= o[a] + 4 * k) slices[a] |= 1u << k;
            }
            unsigned occ = 0u;
#pragma unroll
            for (int q = 0; q < SX * SY * SZ; q++)
                if (((slices[0] >> (q % SX)) & (slices[1] >> ((q / SX) % SY)) & (slices[2] >> (q / (SX * SY)))) & 1u)
                    occ |= 1u << q;
            rec[tid] = make_float4(f[0], f[0], f[1], f[1]);
            rec[NT + tid] = make_float4(f[2], f[2], f[3], f[3]);
            rec[2 * NT + tid] = make_float4(f[4], f[4], f[5], f[5]);
            rec[3 * NT + tid] = make_float4(f[6], f[6], f[7], f[7]);
            rec[4 * NT + tid] = make_float4(f[8], f[8], __uint_as_float(occ), v[0]);
            if (C > 1) rec[5 * NT + tid] = make_float4(v[1], v[2], v[3], 0.f);
        }
        __syncthreads();
        int p0[C], p1[C];
#pragma unroll
        for (int c = 0; c < C; c++) { p0[c] = 0; p1[c] = 0; }
        for (int j = 0; j < m; j++) {
            // a Gaussian whose voxel box misses this warp's sub-block adds
            // nothing there: its q exceeds kappa^2 outside the box (warp-uniform skip)
            const float4 r4 = rec[4 * NT + j];
            if (!((__float_as_uint(r4.z) >> warp) & 1u)) continue;
            const float4 r0 = rec[j], r1 = rec[NT + j], r2 = rec[2 * NT + j], r3 = rec[3 * NT + j];
            float sv[C];
            sv[0] = r4.w;
            if (C > 1) {
                const float4 r5 = rec[5 * NT + j];
                const float rv[3] = {r5.x, r5.y, r5.z};
#pragma unroll
                for (int c = 1; c < C; c++) sv[c] = rv[c - 1];
            }
            // the quadratic form of both voxels on packed pairs, the same
            // operations in the same order as qform() (so the same bits)
            const f32x2 dx = sub2(cxx, pack2(r0.x, r0.y)), dy = sub2(cyy, pack2(r0.z, r0.w));
            const f32x2 dz = sub2(czz, pack2(r1.x, r1.y));
            const f32x2 tx2 = fma2(pack2(r1.z, r1.w), dx, fma2(pack2(r3.x, r3.y), dy, mul2(pack2(r3.z, r3.w), dz)));
            const f32x2 ty2 = fma2(pack2(r2.x, r2.y), dy, mul2(pack2(r4.x, r4.y), dz));
            const f32x2 q = fma2(dx, tx2, fma2(dy, ty2, mul2(mul2(pack2(r2.z, r2.w), dz), dz)));
            const f32x2 qe = mul2(q, nhl);
            if (lo2(q) <= k2) {
                const float e = exp2f(lo2(qe));
#pragma unroll
                for (int c = 0; c < C; c++) p0[c] += __float_as_int(fmaf(sv[c], e, kMagicF)) - kMagicI;
            }
            if (hi2(q) <= k2) {
                const float e = exp2f(hi2(qe));
#pragma unroll
                for (int c = 0; c < C; c++) p1[c] += __float_as_int(fmaf(sv[c], e, kMagicF)) - kMagicI;
            }
        }
#pragma unroll
        for (int c = 0; c < C; c++) { acc0[c] += p0[c]; acc1[c] += p1[c]; }
    }
    const int64_t N = g.n;
    if (ix < g.nx && iy < g.ny) {
        if (iz0 < g.nz) {
            const int64_t v = ((int64_t)iz0 * g.ny + iy) * g.nx + ix;
#pragma unroll
            for (int c = 0; c < C; c++) Store<T>::st(out, c * N + v, bad ? __int_as_float(0x7fc00000) : __ll2float_rn(acc0[c]) * inv_scale);
        }
        if (iz1 < g.nz) {
            const int64_t v = ((int64_t)iz1 * g.ny + iy) * g.nx + ix;
#pragma unroll
            for (int c = 0; c < C; c++) Store<T>::st(out, c * N + v, bad ? __int_as_float(0x7fc00000) : __ll2float_rn(acc1[c]) * inv_scale);
        }
    }
}

__global__ void k_copy_total(const VoxWs w, int64_t* d_pairs) { *d_pairs = w.hdr->total_pairs; }

// ------------------------------------------------------------ backward
//
// Work item = one warp on (Gaussian g, slab s): the warp takes the rows (y, z)
// of g's voxel box with row index = s (mod S), one row per lane, and on each
// row only the x span
// where the quadratic form can be <= kappa^2 (solved analytically, with one
// voxel of slack; the per-voxel test is the forward's).  It accumulates the
// C + 9 moments, reduces them over the warp in a fixed tree, and writes either
// the gradient (S = 1) or a partial that a second pass sums in slab order.

constexpr int kBwdWarps = 8;   // warps per CTA of the slab-merge pass
// One warp per CTA in the adjoint proper: a warp's (Gaussian, slab) item is
// independent of its CTA, and Gaussians of very different sizes in one CTA
// would keep the CTA resident, its finished warps idle, until the largest is
// done; single-warp CTAs let the SM refill each slot at once.  The
// one-channel form fits 64 registers, 32 resident warps (measured 9% faster
// than at 80); the three-channel form would spill there and stays at 24.
constexpr int kBwdItemWarps = 1;
constexpr int kMom = 9;        // S1 (3) + S2 (6)

template <int C>
struct Moments {
    float gv[C], s1[3], s2[6];
};

// Row x-span of {q <= k2} for fixed (dy, dz), as voxel indices clamped to [lo, hi].
__device__ __forceinline__ bool row_span(const GaussSetup& s, float k2, float dy, float dz, const GridD& g, int& xlo,
                                         int& xhi) {
    xlo = s.lo[0];
    xhi = s.hi[0];
    if (isinf(k2)) return true;
    const float B = s.b01 * dy + s.b02 * dz;
    const float C0 = s.a11 * dy * dy + s.b12 * dy * dz + s.a22 * dz * dz - k2;
    const float disc = B * B - 4.0f * s.a00 * C0;
    // skip only rows that are clearly empty; near-tangent rows keep their
    // candidates and the exact per-voxel test decides
    if (disc < -1e-4f * (B * B + fabsf(4.0f * s.a00 * C0))) return false;
    const float r = sqrtf(fmaxf(disc, 0.0f));
    const float inv2a = 0.5f / s.a00;
    const float d0 = (-B - r) * inv2a, d1 = (-B + r) * inv2a;
    const float c = s.mu[0] * g.ivx + 0.5f * (float)g.nx - 0.5f;
    const float f0 = floorf(c + d0 * g.ivx) - 1.0f, f1 = ceilf(c + d1 * g.ivx) + 1.0f;
    xlo = max(xlo, (int)fmaxf(f0, -1.0f));
    xhi = min(xhi, (int)fminf(f1, (float)g.nx));
    return xlo <= xhi;
}

template <int C>
__device__ __forceinline__ void warp_moments(const pmf_gaussians& G, int64_t i, const GaussSetup& s, const GridD& g,
                                             const float* __restrict__ dout, int slab, int S, bool vec, Moments<C>& m) {
    const int lane = threadIdx.x & 31;
    const float k2 = isinf(G.kappa) ? INFINITY : G.kappa * G.kappa;
    float val[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        val[c] = __ldg(G.value + i * C + c);
        m.gv[c] = 0.f;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) m.s1[a] = 0.f;
#pragma unroll
    for (int a = 0; a < 6; a++) m.s2[a] = 0.f;
    if (s.lo[0] > s.hi[0] || s.lo[1] > s.hi[1] || s.lo[2] > s.hi[2]) return;
    const int ey = s.hi[1] - s.lo[1] + 1, ez = s.hi[2] - s.lo[2] + 1;
    const int rows = ey * ez;
    const int64_t N = g.n;
    // one box row per lane (rows slab, slab + S, ... are this warp's), each
    // lane walking its row's x span
    for (int row = slab + S * lane; row < rows; row += 32 * S) {
        const int y = s.lo[1] + row % ey, z = s.lo[2] + row / ey;
        const float dy = centre(y, g.ny, g.vy) - s.mu[1];
        const float dz = centre(z, g.nz, g.vz) - s.mu[2];
        int xlo, xhi;
        if (!row_span(s, k2, dy, dz, g, xlo, xhi)) continue;
        const float* drow = dout + ((int64_t)z * g.ny + y) * g.nx;
        // four voxels per step: their upstream-gradient loads are issued
        // together (the span lies inside the grid), then accumulated in x order.
        // Several channels on 16-byte rows: the steps are the aligned 4-voxel
        // blocks that meet the span, each channel one 16-byte load (a quarter
        // of the L1 sector requests, which bind these calls: 19% faster at the
        // paper's MBC levels); the voxels visited, and their order, are the
        // same.  One channel is not L1-bound, and its short rows would pay
        // for the blocks' extra voxels (13% slower), so it keeps scalar loads.
        const bool v4 = C > 1 && vec;
        const int xs = v4 ? (xlo & ~3) : xlo;
        for (int x0 = xs; x0 <= xhi; x0 += 4) {
            float go[4][C];
            if (v4) {
#pragma unroll
                for (int c = 0; c < C; c++) {
                    const float4 t4 = __ldg(reinterpret_cast<const float4*>(drow + c * N + x0));
                    go[0][c] = t4.x; go[1][c] = t4.y; go[2][c] = t4.z; go[3][c] = t4.w;
                }
            } else {
#pragma unroll
                for (int u = 0; u < 4; u++)
#pragma unroll
                    for (int c = 0; c < C; c++) go[u][c] = x0 + u <= xhi ? __ldg(drow + c * N + x0 + u) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int x = x0 + u;
                if (x > xhi) break;
                if (x < xlo) continue;
                const float dx = centre(x, g.nx, g.vx) - s.mu[0];
                const float q = qform(dx, dy, dz, s.a00, s.a11, s.a22, s.b01, s.b02, s.b12);
                if (!(q <= k2)) continue;
                const float e = exp2f(q * kNegHalfLog2e);
                float sw = 0.f;
#pragma unroll
                for (int c = 0; c < C; c++) {
                    m.gv[c] = fmaf(go[u][c], e, m.gv[c]);
                    sw = fmaf(val[c], go[u][c], sw);
                }
                const float wgt = sw * e;
                m.s1[0] = fmaf(wgt, dx, m.s1[0]); m.s1[1] = fmaf(wgt, dy, m.s1[1]); m.s1[2] = fmaf(wgt, dz, m.s1[2]);
                const float wx = wgt * dx, wy = wgt * dy;
                m.s2[0] = fmaf(wx, dx, m.s2[0]); m.s2[1] = fmaf(wx, dy, m.s2[1]); m.s2[2] = fmaf(wx, dz, m.s2[2]);
                m.s2[3] = fmaf(wy, dy, m.s2[3]); m.s2[4] = fmaf(wy, dz, m.s2[4]); m.s2[5] = fmaf(wgt * dz, dz, m.s2[5]);
            }
        }
    }
}

__device__ __forceinline__ float warp_sum(float r) {
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// Gradients of one Gaussian from its summed moments (thread-local).
template <int C>
__device__ void moments_to_grad(const GaussSetup& s, const float* r, int64_t i, float* d_mean, float* d_scale,
                                float* d_quat, float* d_value, int accumulate) {
    const float* s1 = r + C;
    const float* s2v = r + C + 3;
    const float S2m[3][3] = {{s2v[0], s2v[1], s2v[2]}, {s2v[1], s2v[3], s2v[4]}, {s2v[2], s2v[4], s2v[5]}};
    const float A[3][3] = {{s.a00, 0.5f * s.b01, 0.5f * s.b02},
                           {0.5f * s.b01, s.a11, 0.5f * s.b12},
                           {0.5f * s.b02, 0.5f * s.b12, s.a22}};
    float gmu[3], gs[3], gR[9];
    for (int a = 0; a < 3; a++) gmu[a] = A[a][0] * s1[0] + A[a][1] * s1[1] + A[a][2] * s1[2];
    float S2R[3][3];
    for (int a = 0; a < 3; a++)
        for (int j = 0; j < 3; j++)
            S2R[a][j] = S2m[a][0] * s.R[0 * 3 + j] + S2m[a][1] * s.R[1 * 3 + j] + S2m[a][2] * s.R[2 * 3 + j];
    for (int j = 0; j < 3; j++) {
        float d = s.R[0 * 3 + j] * S2R[0][j] + s.R[1 * 3 + j] * S2R[1][j] + s.R[2 * 3 + j] * S2R[2][j];
        gs[j] = d / (s.s[j] * s.s[j] * s.s[j]);
        for (int a = 0; a < 3; a++) gR[3 * a + j] = -S2R[a][j] / (s.s[j] * s.s[j]);
    }
    // dR/d(w,x,y,z) of R(q/|q|), then the normalisation Jacobian (I - qq^T)/|q|
    const float w = s.qn[0], x = s.qn[1], y = s.qn[2], z = s.qn[3];
    const float dRw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const float dRx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const float dRy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const float dRz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    float gq[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < 9; t++) {
        gq[0] += gR[t] * dRw[t]; gq[1] += gR[t] * dRx[t]; gq[2] += gR[t] * dRy[t]; gq[3] += gR[t] * dRz[t];
    }
    const float dot = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    const float qn[4] = {w, x, y, z};
    const float inv = 1.0f / s.qnorm;
    for (int c = 0; c < 4; c++) {
        const float v = (gq[c] - qn[c] * dot) * inv;
        d_quat[4 * i + c] = accumulate ? d_quat[4 * i + c] + v : v;
    }
    for (int a = 0; a < 3; a++) {
        d_mean[3 * i + a] = accumulate ? d_mean[3 * i + a] + gmu[a] : gmu[a];
        d_scale[3 * i + a] = accumulate ? d_scale[3 * i + a] + gs[a] : gs[a];
    }
    for (int c = 0; c < C; c++) d_value[i * C + c] = accumulate ? d_value[i * C + c] + r[c] : r[c];
}

template <int C>
__global__ void __launch_bounds__(32 * kBwdItemWarps, (C == 1 ? 32 : 24) / kBwdItemWarps) k_vox_bwd(pmf_gaussians G, GridD g, int S,
                                                            const float* __restrict__ dout, float* part,
                                                            float* d_mean, float* d_scale, float* d_quat,
                                                            float* d_value, int accumulate, bool vec) {
    const int64_t item = (int64_t)blockIdx.x * kBwdItemWarps + (threadIdx.x >> 5);
    if (item >= G.n * S) return;
    const int64_t i = item / S;
    const int slab = (int)(item - i * S);
    GaussSetup st;
    gauss_setup(G, i, g, G.kappa, st);
    if (st.lo[0] > st.hi[0] || st.lo[1] > st.hi[1] || st.lo[2] > st.hi[2]) {
        // no voxel of the grid within the truncation box (a Gaussian outside a
        // sub-volume): every moment is zero, so is the gradient (warp-uniform)
        if ((threadIdx.x & 31) != 0) return;
        if (S > 1) {
            for (int k = 0; k < C + kMom; k++) part[item * (C + kMom) + k] = 0.0f;
        } else if (!accumulate) {
            for (int a = 0; a < 3; a++) d_mean[3 * i + a] = d_scale[3 * i + a] = 0.0f;
            for (int a = 0; a < 4; a++) d_quat[4 * i + a] = 0.0f;
            for (int c = 0; c < C; c++) d_value[i * C + c] = 0.0f;
        }
        return;
    }
    Moments<C> m;
    warp_moments<C>(G, i, st, g, dout, slab, S, vec, m);
    float r[C + kMom];
#pragma unroll
    for (int c = 0; c < C; c++) r[c] = warp_sum(m.gv[c]);
#pragma unroll
    for (int a = 0; a < 3; a++) r[C + a] = warp_sum(m.s1[a]);
#pragma unroll
    for (int a = 0; a < 6; a++) r[C + 3 + a] = warp_sum(m.s2[a]);
    if ((threadIdx.x & 31) != 0) return;
    if (S == 1) {
        moments_to_grad<C>(st, r, i, d_mean, d_scale, d_quat, d_value, accumulate);
    } else {
#pragma unroll
        for (int k = 0; k < C + kMom; k++) part[item * (C + kMom) + k] = r[k];
    }
}

// Sum a Gaussian's S slab partials in a fixed order (lane-strided, then a
// fixed tree) and form its gradient.
template <int C>
__global__ void __launch_bounds__(32 * kBwdWarps) k_vox_bwd_final(pmf_gaussians G, GridD g, int S,
                                                                  const float* __restrict__ part, float* d_mean,
                                                                  float* d_scale, float* d_quat, float* d_value,
                                                                  int accumulate) {
    const int64_t i = (int64_t)blockIdx.x * kBwdWarps + (threadIdx.x >> 5);
    if (i >= G.n) return;
    const int lane = threadIdx.x & 31;
    float r[C + kMom];
#pragma unroll
    for (int k = 0; k < C + kMom; k++) r[k] = 0.f;
    for (int sl = lane; sl < S; sl += 32)
#pragma unroll
        for (int k = 0; k < C + kMom; k++) r[k] += part[(i * S + sl) * (C + kMom) + k];
#pragma unroll
    for (int k = 0; k < C + kMom; k++) r[k] = warp_sum(r[k]);
    if (lane != 0) return;
    GaussSetup st;
    gauss_setup(G, i, g, G.kappa, st);
    moments_to_grad<C>(st, r, i, d_mean, d_scale, d_quat, d_value, accumulate);
}

// Slabs per Gaussian: enough warps to fill the GPU a few times over, at most
// 256, a power of two.
int bwd_slabs(int64_t n) {
    int64_t want = (int64_t)152 * 64 * 4;  // warps
    int s = 1;
    while (s < 256 && n * s * 2 <= want) s *= 2;
    return s;
}

pmf_status validate_gaussians(const pmf_gaussians* g) {
    PMF_REQUIRE(g != nullptr, "gaussians is null");
    PMF_REQUIRE(g->n >= 0 && g->n < ((int64_t)1 << 31), "gaussian count %lld out of range", (long long)g->n);
    PMF_REQUIRE(g->channels >= 1, "channels must be >= 1");
    if (g->channels > kMaxC) return set_error(PMF_EUNSUPPORTED, "channels > %d not supported", kMaxC);
    PMF_REQUIRE(g->kappa > 0.0f, "kappa must be > 0 (use INFINITY for no truncation)");
    if (g->n > 0)
        PMF_REQUIRE(g->mean && g->scale && g->quat && g->value, "gaussian arrays must be non-null");
    return PMF_OK;
}

pmf_status run_prep_scan(const pmf_grid* grid, const pmf_gaussians* gs, const VoxWs& w, const GridD& g,
                         const VoxTile& tl, cudaStream_t st, int ntx, int nty, int64_t T) {
    cudaMemsetAsync(w.hdr, 0, sizeof(VoxHeader), st);
    cudaMemsetAsync(w.tcount, 0, sizeof(unsigned) * (size_t)T, st);
    cudaMemsetAsync(w.cursor, 0, sizeof(unsigned) * (size_t)T, st);
    if (gs->n > 0) {
        int64_t threads = gs->n * 32;
        k_prep<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(*gs, g, gs->kappa, w, tl, ntx, nty);
    }
    k_scan<<<1, 1024, 0, st>>>(w, T);
    (void)grid;
    return check_launch("gs_voxelize prep");
}

pmf_status get_tile(const int32_t* tile, VoxTile& tl) {
    PMF_REQUIRE(tile != nullptr, "tile is null");
    tl = VoxTile{tile[0], tile[1], tile[2]};
    if (!supported_tile(tl))
        return set_error(PMF_EUNSUPPORTED, "voxelizer bin tile %dx%dx%d not supported (8x8x8, 16x8x8, 8x8x4, 16x8x4)",
                         tile[0], tile[1], tile[2]);
    return PMF_OK;
}

// Dynamic shared memory of k_render: the records and the staged indices.
template <int C>
constexpr size_t render_smem(int nt) { return (size_t)nt * (16 * (C > 1 ? 6 : 5) + 4); }

template <typename T, int C, int TX, int TY, int TZ>
void render_launch(unsigned blocks, const pmf_gaussians& G, const GridD& g, const VoxWs& w, T* out, int ntx, int nty,
                   cudaStream_t s) {
    constexpr int NT = TX * TY * TZ / 2;
    const size_t smem = render_smem<C>(NT);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_render<T, C, TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_render<T, C, TX, TY, TZ><<<blocks, NT, smem, s>>>(G, g, w, out, ntx, nty);
}

template <typename T, int C>
void render_tiled(const VoxTile& tl, int64_t nt, const pmf_gaussians& G, const GridD& g, const VoxWs& w, T* out,
                  int ntx, int nty, cudaStream_t s) {
    const unsigned blocks = (unsigned)nt;
    if (tl.x == 16 && tl.z == 8)
        render_launch<T, C, 16, 8, 8>(blocks, G, g, w, out, ntx, nty, s);
    else if (tl.x == 16)
        render_launch<T, C, 16, 8, 4>(blocks, G, g, w, out, ntx, nty, s);
    else if (tl.z == 4)
        render_launch<T, C, 8, 8, 4>(blocks, G, g, w, out, ntx, nty, s);
    else
        render_launch<T, C, 8, 8, 8>(blocks, G, g, w, out, ntx, nty, s);
}

}  // namespace

PMF_DIAG_ACCESSOR(diag_voxelize)

}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status gs_voxelize_tiled_workspace(const pmf_grid* grid, int64_t n, int64_t pair_capacity, const int32_t tile[3],
                                      size_t* bytes) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    VoxTile tl;
    if ((st = get_tile(tile, tl)) != PMF_OK) return st;
    PMF_REQUIRE(bytes != nullptr, "bytes is null");
    PMF_REQUIRE(n >= 0 && pair_capacity >= 0 && pair_capacity < ((int64_t)1 << 32), "bad sizes");
    GridD g = make_grid(grid);
    *bytes = vox_ws_layout(g, n, pair_capacity, tl, nullptr, nullptr);
    return PMF_OK;
}

pmf_status gs_voxelize_workspace(const pmf_grid* grid, int64_t n, int64_t pair_capacity, size_t* bytes) {
    const int32_t tile[3] = {kDefaultTile.x, kDefaultTile.y, kDefaultTile.z};
    return gs_voxelize_tiled_workspace(grid, n, pair_capacity, tile, bytes);
}

pmf_status gs_voxelize_tiled_count(const pmf_grid* grid, const pmf_gaussians* gs, const int32_t tile[3],
                                   int64_t* d_pairs, void* ws, size_t ws_bytes, pmf_stream stream) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    if ((st = validate_gaussians(gs)) != PMF_OK) return st;
    VoxTile tl;
    if ((st = get_tile(tile, tl)) != PMF_OK) return st;
    PMF_REQUIRE(d_pairs != nullptr, "d_pairs is null");
    GridD g = make_grid(grid);
    size_t need = vox_ws_layout(g, gs->n, 0, tl, nullptr, nullptr);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    VoxWs w;
    vox_ws_layout(g, gs->n, 0, tl, &w, (char*)ws);
    const int ntx = ceil_div(g.nx, tl.x), nty = ceil_div(g.ny, tl.y), ntz = ceil_div(g.nz, tl.z);
    const int64_t T = (int64_t)ntx * nty * ntz;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = run_prep_scan(grid, gs, w, g, tl, s, ntx, nty, T)) != PMF_OK) return st;
    k_copy_total<<<1, 1, 0, s>>>(w, d_pairs);
    return check_launch("gs_voxelize_count");
}

pmf_status gs_voxelize_count(const pmf_grid* grid, const pmf_gaussians* gs, int64_t* d_pairs, void* ws,
                             size_t ws_bytes, pmf_stream stream) {
    const int32_t tile[3] = {kDefaultTile.x, kDefaultTile.y, kDefaultTile.z};
    return gs_voxelize_tiled_count(grid, gs, tile, d_pairs, ws, ws_bytes, stream);
}

pmf_status gs_voxelize_tiled(const pmf_grid* grid, const pmf_gaussians* gs, pmf_dtype dtype, const int32_t tile[3],
                             void* out, void* ws, size_t ws_bytes, pmf_stream stream) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    if ((st = validate_gaussians(gs)) != PMF_OK) return st;
    if ((st = validate_dtype(dtype)) != PMF_OK) return st;
    VoxTile tl;
    if ((st = get_tile(tile, tl)) != PMF_OK) return st;
    PMF_REQUIRE(out != nullptr, "out is null");
    GridD g = make_grid(grid);
    size_t fixed = vox_ws_layout(g, gs->n, 0, tl, nullptr, nullptr);
    if ((st = validate_ws(ws, ws_bytes, fixed)) != PMF_OK) return st;
    // whatever is left after the fixed part holds the pair list
    int64_t cap = (int64_t)((ws_bytes - fixed) / sizeof(unsigned)) + 1;
    while (cap > 0 && vox_ws_layout(g, gs->n, cap, tl, nullptr, nullptr) > ws_bytes) cap -= 64;
    if (cap < 0) cap = 0;
    if (cap > 0xfffffff0ll) cap = 0xfffffff0ll;
    VoxWs w;
    vox_ws_layout(g, gs->n, cap, tl, &w, (char*)ws);
    const int ntx = ceil_div(g.nx, tl.x), nty = ceil_div(g.ny, tl.y), ntz = ceil_div(g.nz, tl.z);
    const int64_t T = (int64_t)ntx * nty * ntz;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = run_prep_scan(grid, gs, w, g, tl, s, ntx, nty, T)) != PMF_OK) return st;
    if (gs->n > 0) {
        int64_t threads = gs->n * 32;
        k_fill<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(gs->n, w, tl, ntx, nty);
    }
    PMF_DISPATCH_DTYPE(dtype, T_, {
        T_* o = (T_*)out;
        switch (gs->channels) {
            case 1: render_tiled<T_, 1>(tl, T, *gs, g, w, o, ntx, nty, s); break;
            case 2: render_tiled<T_, 2>(tl, T, *gs, g, w, o, ntx, nty, s); break;
            case 3: render_tiled<T_, 3>(tl, T, *gs, g, w, o, ntx, nty, s); break;
            default: render_tiled<T_, 4>(tl, T, *gs, g, w, o, ntx, nty, s); break;
        }
    });
    return check_launch("gs_voxelize");
}

pmf_status gs_voxelize(const pmf_grid* grid, const pmf_gaussians* gs, pmf_dtype dtype, void* out, void* ws,
                       size_t ws_bytes, pmf_stream stream) {
    const int32_t tile[3] = {kDefaultTile.x, kDefaultTile.y, kDefaultTile.z};
    return gs_voxelize_tiled(grid, gs, dtype, tile, out, ws, ws_bytes, stream);
}

pmf_status gs_voxelize_backward_workspace(const pmf_grid* grid, int64_t n, int32_t channels, size_t* bytes) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(bytes != nullptr && n >= 0 && channels >= 1, "bad arguments");
    if (channels > kMaxC) return set_error(PMF_EUNSUPPORTED, "channels > %d not supported", kMaxC);
    const int S = bwd_slabs(n);
    *bytes = S > 1 ? align_up(sizeof(float) * (size_t)n * S * (channels + kMom)) : 0;
    return PMF_OK;
}

pmf_status gs_voxelize_backward(const pmf_grid* grid, const pmf_gaussians* gs, const float* d_out, float* d_mean,
                                float* d_scale, float* d_quat, float* d_value, int accumulate, void* ws,
                                size_t ws_bytes, pmf_stream stream) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    if ((st = validate_gaussians(gs)) != PMF_OK) return st;
    size_t need = 0;
    if ((st = gs_voxelize_backward_workspace(grid, gs->n, gs->channels, &need)) != PMF_OK) return st;
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    if (gs->n == 0) return PMF_OK;
    PMF_REQUIRE(d_out && d_mean && d_scale && d_quat && d_value, "null gradient pointer");
    GridD g = make_grid(grid);
    cudaStream_t s = (cudaStream_t)stream;
    const int S = bwd_slabs(gs->n);
    // 16-byte rows: every row start, and every channel plane, on a 16-byte boundary
    const bool vec = g.nx % 4 == 0 && ((uintptr_t)d_out & 15) == 0;
    float* part = (float*)ws;
    const int64_t items = gs->n * S;
    const unsigned nb = (unsigned)((items + kBwdItemWarps - 1) / kBwdItemWarps);
    const unsigned nf = (unsigned)((gs->n + kBwdWarps - 1) / kBwdWarps);
    const int T = 32 * kBwdWarps, TI = 32 * kBwdItemWarps;
#define PMF_VB(CC)                                                                                               \
    k_vox_bwd<CC><<<nb, TI, 0, s>>>(*gs, g, S, d_out, part, d_mean, d_scale, d_quat, d_value, accumulate, vec); \
    if (S > 1) k_vox_bwd_final<CC><<<nf, T, 0, s>>>(*gs, g, S, part, d_mean, d_scale, d_quat, d_value, accumulate);
    switch (gs->channels) {
        case 1: { PMF_VB(1) break; }
        case 2: { PMF_VB(2) break; }
        case 3: { PMF_VB(3) break; }
        default: { PMF_VB(4) break; }
    }
#undef PMF_VB
    return check_launch("gs_voxelize_backward");
}

}  // extern "C"
