// Stage-1 X-ray rasterizer (Eq. 8-9) for sm_103a: every Gaussian of the
// reference set is projected to a 2-D Gaussian on the detector through the
// local affine approximation of the cone-beam ray-space map, and the 2-D
// Gaussians are summed at pixel centres.
//
//   k_splat_frames  one thread per view: the detector-plane frame in double
//   k_splat_prep    one CTA per (view, Gaussian chunk): p^ (double), Sigma^-1,
//                   rho^, the kappa-ellipse's pixel box, and the chunk's
//                   per-tile counts in a shared-memory histogram
//   k_scan_*        prefix sums over (view, tile, chunk): list offsets
//   k_splat_fill    one CTA per (view, Gaussian chunk): the per-tile lists,
//                   placed through shared-memory cursors (no global atomics)
//   k_splat_render  one CTA per (16x16 tile, view), one pixel per thread: the
//                   tile's list staged in shared memory in batches; each warp
//                   owns an 8x4 pixel block, tests 32 entries at a time (one
//                   per lane, then a ballot) and visits only the Gaussians
//                   whose box reaches the block; per-pixel sums are exact
//                   integers at a per-view scale, so the (unordered) lists
//                   give bit-reproducible projections
//   k_splat_bwd_sums   one warp per (view, Gaussian): each lane walks the runs of
//                      kappa-ellipse pixels in its rows (the render's own test
//                      settles the run ends), six sums by a warp butterfly
//   k_splat_bwd_chain  one thread per Gaussian: the chain rule of every view, in
//                      view order, back to (mean, scale, quaternion, value); no
//                      atomics anywhere, so the adjoint is bit-reproducible
//
// The projection of one Gaussian in one view (all in the view's frame):
//   r = mu - src, z = n.r, ua = ut.r, vb = vt.r (ut, vt: the dual basis of
//   du, dv in the detector plane; n its unit normal; h = n.(det - src)),
//   p^ = (h ua / z - ut.(det - src), h vb / z - vt.(det - src))   (pixels),
//   J rows  Ja = (h/z)(ut - (ua/z) n),  Jb = (h/z)(vt - (vb/z) n),  Jt = r/|r|,
//   Sigma^ = [Ja; Jb] Sigma [Ja; Jb]^T = T^T T with T = [M^T Ja, M^T Jb], M = R diag(s),
//   rho^ = rho sqrt(2 pi |Sigma~| / |Sigma^|) = rho sqrt(2 pi / lambda),
//   lambda = c^T Sigma^-1 c = sum_k (R^T c)_k^2 / s_k^2, c = r / |r|
// (the Schur-complement identity |Sigma~| / |Sigma^| = 1 / (Sigma~^-1)_tt with
// J^-1 e_t = c; it avoids a 3x3 determinant of mixed pixel/mm entries in fp32).
#include <math.h>

#include "pmf_common.cuh"
#include "scan.cuh"

namespace pmf {
namespace {

constexpr int kSplatTile = 16;        // tile side (pixels)
constexpr int kRenderThreads = 256;   // one pixel per thread
constexpr int kBwdWarps = 8;          // Gaussians per backward CTA
constexpr float kMagicF = 12582912.0f;  // 1.5 * 2^23: floats in [2^23, 2^24) are integers
constexpr int kMagicI = 0x4b400000;
constexpr float kTwoPi = 6.283185307179586f;
constexpr float kCullSlack = 0.01f;   // pixels: keeps the warp cull conservative under rounding

struct SplatFrame {
    double src[3], ut[3], vt[3], n[3];
    double h, a0, b0;
    float srcf[3], utf[3], vtf[3], nf[3], hf;  // fp32 copies for the Jacobian and the chain rule
};

// One Gaussian in one view (32 bytes, read as two float4).
struct __align__(16) SplatRec {
    float a, b;        // p^, pixels from the detector centre
    float k0, k1, k2;  // Sigma^-1 entries 00, 01, 11
    float rho;         // rho^
    float wa, wb;      // half-widths of the kappa-ellipse's bounding box (pixels); -1: nothing
};

struct RasterWs {
    SplatFrame* frames;          // [P]
    SplatRec* rec;               // [P][n]
    int4* rect;                  // [P][n] pixel box (i0, j0, i1, j1); empty: i1 < i0
    float* sums;                 // [P][n][8] the adjoint's pixel sums
    unsigned* chist;             // [P][T][C] (view, tile, Gaussian chunk) overlap counts
    unsigned* coff;              // [P*T*C + 1] their exclusive prefix sums: list offsets
    unsigned long long* bsum;    // [scan blocks] the scan's block totals
    unsigned* maxbits;           // [P] largest |rho^| (float bits)
    int chunk, C;                // Gaussians per chunk and chunks per view
    unsigned long long* total;   // pairs the call needs
    unsigned* list;              // [capacity] Gaussian indices, tile-major
    int64_t capacity;
    size_t list_off;             // byte offset of the list in the workspace
};

constexpr int kPrepThreads = 256;
constexpr int kMaxTiles = 12288;  // shared-memory histogram of a view's tiles (48 KB)

// Gaussians per (view, chunk) CTA of the prep and fill: about 8 CTAs per SM in
// total, at least one per thread, at most 8,192.
int chunk_of(int P, int64_t n) {
    const int64_t want = ((int64_t)P * n + 152 * 8 - 1) / (152 * 8);
    int64_t c = (want + kPrepThreads - 1) / kPrepThreads * kPrepThreads;
    return (int)(c < kPrepThreads ? kPrepThreads : (c > 8192 ? 8192 : c));
}

size_t raster_ws_layout(int P, int64_t n, int64_t T, int64_t capacity, RasterWs* w, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return base ? base + o : nullptr;
    };
    RasterWs x;
    const size_t Pn = (size_t)(P > 0 ? P : 1) * (size_t)(n > 0 ? n : 1), PT = (size_t)(P > 0 ? P : 1) * (size_t)T;
    x.frames = (SplatFrame*)take(sizeof(SplatFrame) * (size_t)(P > 0 ? P : 1));
    x.rec = (SplatRec*)take(sizeof(SplatRec) * Pn);
    x.rect = (int4*)take(sizeof(int4) * Pn);
    x.sums = (float*)take(sizeof(float) * 8 * Pn);
    x.chunk = chunk_of(P, n);
    x.C = (int)((n + x.chunk - 1) / x.chunk);
    const size_t N = PT * (size_t)x.C;
    x.chist = (unsigned*)take(sizeof(unsigned) * (N > 0 ? N : 1));
    x.coff = (unsigned*)take(sizeof(unsigned) * (N + 1));
    x.bsum = (unsigned long long*)take(sizeof(unsigned long long) * (N / kScanItems + 2));
    x.maxbits = (unsigned*)take(sizeof(unsigned) * (size_t)(P > 0 ? P : 1));
    x.total = (unsigned long long*)take(sizeof(unsigned long long));
    x.list_off = off;
    x.list = (unsigned*)take(sizeof(unsigned) * (size_t)(capacity > 0 ? capacity : 1));
    x.capacity = capacity;
    if (w) *w = x;
    return off;
}


__global__ void k_splat_frames(const pmf_view* __restrict__ views, int P, SplatFrame* fr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const pmf_view& v = views[p];
    SplatFrame f;
    double D[3], nrm[3];
    for (int t = 0; t < 3; t++) {
        f.src[t] = v.src[t];
        D[t] = v.det[t] - v.src[t];
    }
    nrm[0] = v.du[1] * v.dv[2] - v.du[2] * v.dv[1];
    nrm[1] = v.du[2] * v.dv[0] - v.du[0] * v.dv[2];
    nrm[2] = v.du[0] * v.dv[1] - v.du[1] * v.dv[0];
    const double nn = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    const double sgn = (nrm[0] * D[0] + nrm[1] * D[1] + nrm[2] * D[2]) < 0.0 ? -1.0 : 1.0;
    for (int t = 0; t < 3; t++) f.n[t] = sgn * nrm[t] / nn;
    f.h = f.n[0] * D[0] + f.n[1] * D[1] + f.n[2] * D[2];
    const double uu = v.du[0] * v.du[0] + v.du[1] * v.du[1] + v.du[2] * v.du[2];
    const double vv = v.dv[0] * v.dv[0] + v.dv[1] * v.dv[1] + v.dv[2] * v.dv[2];
    const double uv = v.du[0] * v.dv[0] + v.du[1] * v.dv[1] + v.du[2] * v.dv[2];
    const double del = uu * vv - uv * uv;
    for (int t = 0; t < 3; t++) {
        f.ut[t] = (vv * v.du[t] - uv * v.dv[t]) / del;
        f.vt[t] = (uu * v.dv[t] - uv * v.du[t]) / del;
    }
    f.a0 = f.ut[0] * D[0] + f.ut[1] * D[1] + f.ut[2] * D[2];
    f.b0 = f.vt[0] * D[0] + f.vt[1] * D[1] + f.vt[2] * D[2];
    for (int t = 0; t < 3; t++) {
        f.srcf[t] = (float)f.src[t];
        f.utf[t] = (float)f.ut[t];
        f.vtf[t] = (float)f.vt[t];
        f.nf[t] = (float)f.n[t];
    }
    f.hf = (float)f.h;
    fr[p] = f;
}

// Rotation of the normalised quaternion (w, x, y, z), row-major; the columns
// are the Gaussian's principal axes.
__device__ __forceinline__ void quat_rot(const float q[4], float R[9], float qn[4], float& qnorm) {
    qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float inv = 1.0f / qnorm;
    const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Everything the forward and the adjoint need of one Gaussian in one view, in
// fp32 (relative accuracy is all the Jacobian and the amplitudes need; the
// ~400-pixel coordinates p^ are formed in double by splat_centre).
struct SplatGeo {
    bool ok;                 // mean in front of the source and a finite, positive-definite Sigma^
    float r[3], z, ua, vb, L, h;
    float Ja[3], Jb[3];
    float R[9], s[3], qn[4], qnorm;
    float Ta[3], Tb[3];      // M^T Ja, M^T Jb
    float S00, S01, S11, det;
    float c[3], w[3], lam;   // unit ray direction through the mean, R^T c, c^T Sigma^-1 c
};

__device__ __forceinline__ void splat_geo(const SplatFrame& f, const float mu[3], const float s[3], const float q[4],
                                          SplatGeo& o) {
    for (int t = 0; t < 3; t++) o.r[t] = mu[t] - f.srcf[t];
    o.z = f.nf[0] * o.r[0] + f.nf[1] * o.r[1] + f.nf[2] * o.r[2];
    o.ua = f.utf[0] * o.r[0] + f.utf[1] * o.r[1] + f.utf[2] * o.r[2];
    o.vb = f.vtf[0] * o.r[0] + f.vtf[1] * o.r[1] + f.vtf[2] * o.r[2];
    o.h = f.hf;
    o.ok = o.z > 0.0f;
    o.L = sqrtf(o.r[0] * o.r[0] + o.r[1] * o.r[1] + o.r[2] * o.r[2]);
    const float hz = o.h / o.z, uz = o.ua / o.z, vz = o.vb / o.z;
    for (int t = 0; t < 3; t++) {
        o.Ja[t] = hz * (f.utf[t] - uz * f.nf[t]);
        o.Jb[t] = hz * (f.vtf[t] - vz * f.nf[t]);
        o.c[t] = o.r[t] / o.L;
        o.s[t] = s[t];
    }
    quat_rot(q, o.R, o.qn, o.qnorm);
    o.lam = 0.0f;
    for (int k = 0; k < 3; k++) {
        // (M^T J)_k = s_k sum_i R_ik J_i
        float ta = 0.0f, tb = 0.0f, wk = 0.0f;
        for (int i = 0; i < 3; i++) {
            ta = fmaf(o.R[3 * i + k], o.Ja[i], ta);
            tb = fmaf(o.R[3 * i + k], o.Jb[i], tb);
            wk = fmaf(o.R[3 * i + k], o.c[i], wk);
        }
        o.Ta[k] = ta * s[k];
        o.Tb[k] = tb * s[k];
        o.w[k] = wk;
        o.lam += (wk / s[k]) * (wk / s[k]);
    }
    o.S00 = o.Ta[0] * o.Ta[0] + o.Ta[1] * o.Ta[1] + o.Ta[2] * o.Ta[2];
    o.S01 = o.Ta[0] * o.Tb[0] + o.Ta[1] * o.Tb[1] + o.Ta[2] * o.Tb[2];
    o.S11 = o.Tb[0] * o.Tb[0] + o.Tb[1] * o.Tb[1] + o.Tb[2] * o.Tb[2];
    o.det = o.S00 * o.S11 - o.S01 * o.S01;
    o.ok = o.ok && o.det > 0.0f && isfinite(o.det) && o.lam > 0.0f && isfinite(o.lam);
}

// p^ in double: the source is ~1 m away, so r = mu - src in fp32 would move
// p^ by ~1e-4 pixel.
__device__ __forceinline__ void splat_centre(const SplatFrame& f, const float mu[3], float& a, float& b) {
    double rd[3];
    for (int t = 0; t < 3; t++) rd[t] = (double)mu[t] - f.src[t];
    const double iz = f.h / (f.n[0] * rd[0] + f.n[1] * rd[1] + f.n[2] * rd[2]);
    a = (float)(iz * (f.ut[0] * rd[0] + f.ut[1] * rd[1] + f.ut[2] * rd[2]) - f.a0);
    b = (float)(iz * (f.vt[0] * rd[0] + f.vt[1] * rd[1] + f.vt[2] * rd[2]) - f.b0);
}

// The 2-D quadratic form, with explicit fused multiply-adds so that the
// forward and the adjoint take identical truncation decisions.
__device__ __forceinline__ float splat_q(float k0, float k1, float k2, float da, float db) {
    return __fmaf_rn(da, __fmaf_rn(k0, da, __fmul_rn(2.0f * k1, db)), __fmul_rn(__fmul_rn(k2, db), db));
}

__device__ __forceinline__ float pixel_x(int i, int n) { return (float)i + (0.5f - 0.5f * (float)n); }

// One CTA per (Gaussian chunk, view): the projected Gaussians and their pixel
// boxes; with count_tiles, the chunk's per-tile overlap counts (shared-memory
// histogram, written densely to chist) and the view's largest |rho^|.
__global__ void __launch_bounds__(kPrepThreads) k_splat_prep(pmf_gaussians G, int P, int nu, int nv, int ntu, int T,
                                                             RasterWs w, int count_tiles) {
    extern __shared__ unsigned hist[];
    const int p = blockIdx.y, c = blockIdx.x;
    const int64_t g0 = (int64_t)c * w.chunk, g1 = g0 + w.chunk < G.n ? g0 + w.chunk : G.n;
    if (count_tiles)
        for (int t = threadIdx.x; t < T; t += kPrepThreads) hist[t] = 0u;
    __syncthreads();
    const SplatFrame& fr = w.frames[p];
    unsigned mbits = 0u;
    for (int64_t g = g0 + threadIdx.x; g < g1; g += kPrepThreads) {
        const int64_t idx = (int64_t)p * G.n + g;
        const float mu[3] = {__ldg(G.mean + 3 * g), __ldg(G.mean + 3 * g + 1), __ldg(G.mean + 3 * g + 2)};
        const float s[3] = {__ldg(G.scale + 3 * g), __ldg(G.scale + 3 * g + 1), __ldg(G.scale + 3 * g + 2)};
        const float q[4] = {__ldg(G.quat + 4 * g), __ldg(G.quat + 4 * g + 1), __ldg(G.quat + 4 * g + 2),
                            __ldg(G.quat + 4 * g + 3)};
        const float val = __ldg(G.value + g);
        const bool finite_in = isfinite(mu[0] + mu[1] + mu[2]) && isfinite(s[0] + s[1] + s[2]) &&
                               isfinite(q[0] + q[1] + q[2] + q[3]) && isfinite(val);
        SplatGeo o;
        splat_geo(fr, mu, s, q, o);
        SplatRec rc;
        splat_centre(fr, mu, rc.a, rc.b);
        int4 rt = make_int4(0, 0, -1, -1);
        if (o.ok) {
            const float id = 1.0f / o.det;
            rc.k0 = o.S11 * id; rc.k1 = -o.S01 * id; rc.k2 = o.S00 * id;
            rc.rho = val * sqrtf(kTwoPi / o.lam);
            rc.wa = G.kappa * sqrtf(o.S00);
            rc.wb = G.kappa * sqrtf(o.S11);
            // pixels i with |x(i) - a| <= wa, one pixel of slack; clamped in float
            // first (wa may be +inf), then the per-pixel test decides
            const float ci = rc.a + 0.5f * (float)nu - 0.5f, cj = rc.b + 0.5f * (float)nv - 0.5f;
            const float i0 = fminf(fmaxf(ceilf(ci - rc.wa) - 1.0f, 0.0f), (float)nu);
            const float i1 = fminf(fmaxf(floorf(ci + rc.wa) + 1.0f, -1.0f), (float)(nu - 1));
            const float j0 = fminf(fmaxf(ceilf(cj - rc.wb) - 1.0f, 0.0f), (float)nv);
            const float j1 = fminf(fmaxf(floorf(cj + rc.wb) + 1.0f, -1.0f), (float)(nv - 1));
            if (isfinite(rc.a) && isfinite(rc.b) && isfinite(rc.rho) && i0 <= i1 && j0 <= j1)
                rt = make_int4((int)i0, (int)j0, (int)i1, (int)j1);
        } else {
            rc.k0 = rc.k1 = rc.k2 = 0.0f;
            rc.rho = 0.0f;
        }
        if (rt.z < rt.x) rc.wa = rc.wb = -1.0f;  // nothing to draw: culled everywhere
        w.rec[idx] = rc;
        w.rect[idx] = rt;
        if (!count_tiles) continue;
        if (!finite_in || (o.ok && !isfinite(rc.rho))) {
            // a non-finite parameter makes the whole view undefined: NaN scale, NaN output
            diag_count(PMF_DIAG_NONFINITE);
            mbits = 0x7fc00000u;
        }
        if (rt.z >= rt.x) {
            mbits = max(mbits, abs_bits(rc.rho));
            for (int tj = rt.y / kSplatTile; tj <= rt.w / kSplatTile; tj++)
                for (int ti = rt.x / kSplatTile; ti <= rt.z / kSplatTile; ti++)
                    if (PMF_DCHECK(tj * ntu + ti >= 0 && tj * ntu + ti < T)) atomicAdd(hist + tj * ntu + ti, 1u);
        }
    }
    if (!count_tiles) return;
    mbits = __reduce_max_sync(0xffffffffu, mbits);
    if ((threadIdx.x & 31) == 0 && mbits) atomicMax(w.maxbits + p, mbits);
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += kPrepThreads) w.chist[((int64_t)p * T + t) * w.C + c] = hist[t];
}

// One CTA per (Gaussian chunk, view): every (Gaussian, tile) entry of the chunk
// goes to its tile's list at the chunk's own offset, via shared-memory cursors.
__global__ void __launch_bounds__(kPrepThreads) k_splat_fill(int64_t n, int P, int ntu, int T, RasterWs w) {
    extern __shared__ unsigned cur[];
    const int p = blockIdx.y, c = blockIdx.x;
    for (int t = threadIdx.x; t < T; t += kPrepThreads) cur[t] = w.coff[((int64_t)p * T + t) * w.C + c];
    __syncthreads();
    const int64_t g0 = (int64_t)c * w.chunk, g1 = g0 + w.chunk < n ? g0 + w.chunk : n;
    for (int64_t g = g0 + threadIdx.x; g < g1; g += kPrepThreads) {
        const int4 rt = w.rect[(int64_t)p * n + g];
        if (rt.z < rt.x) continue;
        for (int tj = rt.y / kSplatTile; tj <= rt.w / kSplatTile; tj++)
            for (int ti = rt.x / kSplatTile; ti <= rt.z / kSplatTile; ti++) {
                if (!PMF_DCHECK(tj * ntu + ti >= 0 && tj * ntu + ti < T)) continue;
                const unsigned pos = atomicAdd(cur + tj * ntu + ti, 1u);
                if ((int64_t)pos < w.capacity) w.list[pos] = (unsigned)g;
            }
    }
}

// Scale 2^k with max * 2^k < 2^21 (every term below 2^21 of the scale).
__device__ __forceinline__ int splat_exponent(float m) {
    if (!(m > 0.0f)) return 0;
    int e;
    frexpf(m, &e);
    const int k = 21 - e;
    return k > 100 ? 100 : (k < -100 ? -100 : k);
}

__global__ void __launch_bounds__(kRenderThreads) k_splat_render(int64_t n, int nu, int nv, int ntu, int T, float kappa,
                                                                 RasterWs w, float* __restrict__ proj) {
    __shared__ float4 sr[2][kRenderThreads];
    const int p = blockIdx.y, t = blockIdx.x;
    const int ti = t % ntu, tj = t / ntu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bi = ti * kSplatTile + (warp & 1) * 8, bj = tj * kSplatTile + (warp >> 1) * 4;
    const int i = bi + (lane & 7), j = bj + (lane >> 3);
    const float xa = pixel_x(i, nu), xb = pixel_x(j, nv);
    const float xlo = pixel_x(bi, nu) - kCullSlack, xhi = pixel_x(bi + 7, nu) + kCullSlack;
    const float ylo = pixel_x(bj, nv) - kCullSlack, yhi = pixel_x(bj + 3, nv) + kCullSlack;
    const float k2lim = kappa * kappa;
    const float mx = __uint_as_float(w.maxbits[p]);
    const int kexp = splat_exponent(mx);
    const float fsc = ldexpf(1.0f, kexp);
    const int64_t cell = (int64_t)p * T + t;
    const unsigned beg = w.coff[cell * w.C], end = w.coff[(cell + 1) * w.C];
    const bool overflow = (int64_t)end > w.capacity;
    if (overflow && threadIdx.x == 0) diag_count(PMF_DIAG_RASTER_LIST_OVERFLOW);
    const int64_t cnt = overflow ? n : (int64_t)(end - beg);
    const float4* recs = reinterpret_cast<const float4*>(w.rec + (int64_t)p * n);
    long long acc = 0;
    for (int64_t base = 0; base < cnt; base += kRenderThreads) {
        const int64_t k = base + threadIdx.x;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = make_float4(0.f, 0.f, -1.f, -1.f);
        if (k < cnt) {
            const int64_t g = overflow ? k : (int64_t)w.list[beg + k];
            r0 = __ldg(recs + 2 * g);
            r1 = __ldg(recs + 2 * g + 1);
        }
        sr[0][threadIdx.x] = r0;
        sr[1][threadIdx.x] = r1;
        __syncthreads();
        int part = 0;  // < 256 terms of < 2^21 each
        // each lane tests one entry of every 32 against this warp's 8x4 block;
        // the warp then visits only the entries whose box reaches the block
        for (int e0 = 0; e0 < kRenderThreads; e0 += 32) {
            const float4 a = sr[0][e0 + lane], c = sr[1][e0 + lane];  // (a, b, k0, k1), (k2, rho, wa, wb)
            const bool hit = c.z >= 0.0f && a.x + c.z >= xlo && a.x - c.z <= xhi && a.y + c.w >= ylo &&
                             a.y - c.w <= yhi;
            unsigned m = __ballot_sync(0xffffffffu, hit);
            while (m) {
                const int e = e0 + __ffs(m) - 1;
                m &= m - 1;
                const float4 ea = sr[0][e], ec = sr[1][e];
                const float da = xa - ea.x, db = xb - ea.y;
                const float qq = splat_q(ea.z, ea.w, ec.x, da, db);
                if (qq <= k2lim) {
                    const float v = ec.y * __expf(-0.5f * qq);
                    part += __float_as_int(fmaf(v, fsc, kMagicF)) - kMagicI;
                }
            }
        }
        acc += part;
        __syncthreads();
    }
    if (i < nu && j < nv) {
        const bool bad = !isfinite(mx);
        proj[((int64_t)p * nv + j) * nu + i] = bad ? __int_as_float(0x7fc00000) : __ll2float_rn(acc) * ldexpf(1.0f, -kexp);
    }
}

__device__ __forceinline__ float warp_allsum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adjoint, part 1: one warp per (view, Gaussian); lane l walks rows
// rt.y + l, rt.y + l + 32, ... of the Gaussian's pixel box.  In each row the
// pixels inside the kappa-ellipse form one run: its ends come from the row's
// quadratic and are then settled with the forward's own test (splat_q), so the
// adjoint visits exactly the pixels the render drew.  Along the run,
// e = exp(-q/2) is carried by two products per pixel (q grows by k0 (2 da + 1)
// + 2 k1 db per step: e *= r, r *= exp(-k0)), restarted from exact values every
// 8 pixels, and the six sums
//   sum dY e,  sum c (K d)_a,  sum c (K d)_b,  sum c d_a^2,  sum c d_a d_b,  sum c d_b^2
// (c = dY rho^ e, d = x^ - p^) accumulate per lane; a fixed butterfly reduces
// them and lane 0 writes them to sums[view][Gaussian].
__global__ void __launch_bounds__(32 * kBwdWarps, 4) k_splat_bwd_sums(int64_t n, int P, int nu, int nv, float kappa,
                                                                   RasterWs w, const float* __restrict__ dproj) {
    const int64_t pair = (int64_t)blockIdx.x * kBwdWarps + (threadIdx.x >> 5);
    if (pair >= (int64_t)P * n) return;  // whole warps
    const int lane = threadIdx.x & 31;
    const int p = (int)(pair / n);
    const int4 rt = w.rect[pair];
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f, s5 = 0.f;
    if (rt.z >= rt.x) {
        const SplatRec rc = w.rec[pair];
        // the run of a row is {q <= kappa^2}; beyond q = 170, exp(-q/2) < 2e-37
        // adds nothing to fp32 sums, and starting a run there would underflow
        // the carried exponential, so longer runs (kappa > 13) stop at 170
        const float k2lim = fminf(kappa * kappa, 170.0f);
        const float* dp = dproj + (int64_t)p * nu * nv;
        const float step_r = __expf(-rc.k0);
        const float x0 = pixel_x(0, nu);
        for (int j = rt.y + lane; j <= rt.w; j += 32) {
            const float db = pixel_x(j, nv) - rc.b;
            // q - kappa^2 = k0 da^2 + 2 (k1 db) da + (k2 db^2 - kappa^2)
            const float hb = rc.k1 * db, cc = fmaf(rc.k2 * db, db, -k2lim);
            const float disc = fmaf(hb, hb, -rc.k0 * cc);
            const float c0 = rc.a - x0;  // p^_a in pixel-index units
            int i0, i1;
            if (disc >= 0.0f) {
                const float sd = sqrtf(disc);
                i0 = max(rt.x, (int)fmaxf(ceilf(c0 + (-hb - sd) / rc.k0), -1.0e9f));
                i1 = min(rt.z, (int)fminf(floorf(c0 + (-hb + sd) / rc.k0), 1.0e9f));
            } else {
                // no root in fp32: try the pixel nearest the row's minimum
                i0 = i1 = (int)fminf(fmaxf(rintf(c0 - hb / rc.k0), (float)rt.x), (float)rt.z);
            }
            // settle the ends with the render's test
            while (i0 <= i1 && !(splat_q(rc.k0, rc.k1, rc.k2, pixel_x(i0, nu) - rc.a, db) <= k2lim)) i0++;
            while (i1 >= i0 && !(splat_q(rc.k0, rc.k1, rc.k2, pixel_x(i1, nu) - rc.a, db) <= k2lim)) i1--;
            while (i0 > rt.x && splat_q(rc.k0, rc.k1, rc.k2, pixel_x(i0 - 1, nu) - rc.a, db) <= k2lim) i0--;
            while (i1 < rt.z && splat_q(rc.k0, rc.k1, rc.k2, pixel_x(i1 + 1, nu) - rc.a, db) <= k2lim) i1++;
            if (i0 > i1) continue;
            const float db2 = db * db, kbd = rc.k2 * db;
            const float* row = dp + (int64_t)j * nu;
            // the carried products drift by about k^2/2 ulps after k steps: restart
            // them from exact values every 8 pixels
            for (int ib = i0; ib <= i1; ib += 8) {
                // the block's dY values are loaded before any is used, so the
                // (L2-latency) loads of a block overlap
                const int cnt = min(i1 - ib, 7);
                float gyb[8];
#pragma unroll
                for (int k = 0; k < 8; k++) gyb[k] = k <= cnt ? __ldg(row + ib + k) : 0.0f;
                float da = pixel_x(ib, nu) - rc.a;
                float e = __expf(-0.5f * splat_q(rc.k0, rc.k1, rc.k2, da, db));
                float r = __expf(-fmaf(rc.k0, da + 0.5f, hb));
                float ka = fmaf(rc.k0, da, hb), kb = fmaf(rc.k1, da, kbd);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    if (k > cnt) break;
                    const float gy = gyb[k];
                    const float ge = gy * e, c = ge * rc.rho, cd = c * da;
                    s0 += ge;
                    s1 = fmaf(c, ka, s1);
                    s2 = fmaf(c, kb, s2);
                    s3 = fmaf(cd, da, s3);
                    s4 = fmaf(cd, db, s4);
                    s5 = fmaf(c, db2, s5);
                    e *= r;
                    r *= step_r;
                    da += 1.0f;
                    ka += rc.k0;
                    kb += rc.k1;
                }
            }
        }
    }
    s0 = warp_allsum(s0); s1 = warp_allsum(s1); s2 = warp_allsum(s2);
    s3 = warp_allsum(s3); s4 = warp_allsum(s4); s5 = warp_allsum(s5);
    if (lane == 0) {
        float4* o = reinterpret_cast<float4*>(w.sums + 8 * pair);
        o[0] = make_float4(s0, s1, s2, s3);
        o[1] = make_float4(s4, s5, 0.f, 0.f);
    }
}

// Adjoint, part 2: one thread per Gaussian runs the chain rule of every view
// (in view order) from the pixel sums back to (mean, scale, quaternion, value).
__global__ void __launch_bounds__(128) k_splat_bwd_chain(pmf_gaussians G, int P, RasterWs w, float* d_mean,
                                                         float* d_scale, float* d_quat, float* d_value,
                                                         int accumulate) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G.n) return;
    const float mu[3] = {__ldg(G.mean + 3 * g), __ldg(G.mean + 3 * g + 1), __ldg(G.mean + 3 * g + 2)};
    const float s[3] = {__ldg(G.scale + 3 * g), __ldg(G.scale + 3 * g + 1), __ldg(G.scale + 3 * g + 2)};
    const float q[4] = {__ldg(G.quat + 4 * g), __ldg(G.quat + 4 * g + 1), __ldg(G.quat + 4 * g + 2),
                        __ldg(G.quat + 4 * g + 3)};
    const float val = __ldg(G.value + g);
    float gmu[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gR[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float gval = 0.0f;
    float R[9], qn[4], qnorm;
    quat_rot(q, R, qn, qnorm);
    for (int p = 0; p < P; p++) {
        const int64_t idx = (int64_t)p * G.n + g;
        const int4 rt = w.rect[idx];
        if (rt.z < rt.x) continue;
        const SplatRec rc = w.rec[idx];
        const float4 u0 = reinterpret_cast<const float4*>(w.sums + 8 * idx)[0];
        const float2 u1 = reinterpret_cast<const float2*>(w.sums + 8 * idx)[2];
        const float s_rh = u0.x, s_pa = u0.y, s_pb = u0.z, s_00 = u0.w, s_01 = u1.x, s_11 = u1.y;
        const SplatFrame& f = w.frames[p];
        SplatGeo o;
        splat_geo(f, mu, s, q, o);
        // dL/dK (full symmetric 2x2) = -1/2 sum c d d^T;  dL/dS = -K dL/dK K
        const float K[2][2] = {{rc.k0, rc.k1}, {rc.k1, rc.k2}};
        const float GK[2][2] = {{-0.5f * s_00, -0.5f * s_01}, {-0.5f * s_01, -0.5f * s_11}};
        float KG[2][2], GS[2][2];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) KG[a][b] = K[a][0] * GK[0][b] + K[a][1] * GK[1][b];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) GS[a][b] = -(KG[a][0] * K[0][b] + KG[a][1] * K[1][b]);
        float dTa[3], dTb[3];
        for (int k = 0; k < 3; k++) {
            dTa[k] = 2.0f * (GS[0][0] * o.Ta[k] + GS[0][1] * o.Tb[k]);
            dTb[k] = 2.0f * (GS[1][1] * o.Tb[k] + GS[0][1] * o.Ta[k]);
        }
        // T = M^T J with M = R diag(s):  dM_ik = Ja_i dTa_k + Jb_i dTb_k,  dJ = M dT
        float dJa[3] = {0.f, 0.f, 0.f}, dJb[3] = {0.f, 0.f, 0.f};
        for (int i2 = 0; i2 < 3; i2++)
            for (int k = 0; k < 3; k++) {
                const float dM = o.Ja[i2] * dTa[k] + o.Jb[i2] * dTb[k];
                gR[3 * i2 + k] += dM * s[k];
                gs[k] += dM * R[3 * i2 + k];
                const float M = R[3 * i2 + k] * s[k];
                dJa[i2] += M * dTa[k];
                dJb[i2] += M * dTb[k];
            }
        // rho^ = rho sqrt(2 pi / lambda), lambda = sum_k w_k^2 / s_k^2, w = R^T c
        const float sq = sqrtf(kTwoPi / o.lam);
        gval += s_rh * sq;
        const float dlam = -s_rh * val * sq / (2.0f * o.lam);
        float dw[3];
        for (int k = 0; k < 3; k++) {
            dw[k] = dlam * 2.0f * o.w[k] / (s[k] * s[k]);
            gs[k] += -dlam * 2.0f * o.w[k] * o.w[k] / (s[k] * s[k] * s[k]);
        }
        float dc[3];
        for (int i2 = 0; i2 < 3; i2++) {
            dc[i2] = R[3 * i2] * dw[0] + R[3 * i2 + 1] * dw[1] + R[3 * i2 + 2] * dw[2];
            for (int k = 0; k < 3; k++) gR[3 * i2 + k] += o.c[i2] * dw[k];
        }
        // c = r / |r|
        const float cdc = o.c[0] * dc[0] + o.c[1] * dc[1] + o.c[2] * dc[2];
        // p^ = (h ua / z, h vb / z) - const and J(z, ua, vb)
        const float z = o.z, hz = o.h / z, hz2 = o.h / (z * z), hz3 = 2.0f * o.h / (z * z * z);
        float dua = s_pa * hz, dvb = s_pb * hz;
        float dz = -(s_pa * o.h * o.ua + s_pb * o.h * o.vb) / (z * z);
        for (int t = 0; t < 3; t++) {
            dz += dJa[t] * (-hz2 * f.utf[t] + hz3 * o.ua * f.nf[t]) + dJb[t] * (-hz2 * f.vtf[t] + hz3 * o.vb * f.nf[t]);
            dua += dJa[t] * (-hz2 * f.nf[t]);
            dvb += dJb[t] * (-hz2 * f.nf[t]);
        }
        for (int t = 0; t < 3; t++)
            gmu[t] += (dc[t] - o.c[t] * cdc) / o.L + dua * f.utf[t] + dvb * f.vtf[t] + dz * f.nf[t];
    }
    // dR -> d(unit quaternion) -> d(raw quaternion) through (I - qq^T)/|q|
    const float qw = qn[0], qx = qn[1], qy = qn[2], qz = qn[3];
    const float dRw[9] = {0, -2 * qz, 2 * qy, 2 * qz, 0, -2 * qx, -2 * qy, 2 * qx, 0};
    const float dRx[9] = {0, 2 * qy, 2 * qz, 2 * qy, -4 * qx, -2 * qw, 2 * qz, 2 * qw, -4 * qx};
    const float dRy[9] = {-4 * qy, 2 * qx, 2 * qw, 2 * qx, 0, 2 * qz, -2 * qw, 2 * qz, -4 * qy};
    const float dRz[9] = {-4 * qz, -2 * qw, 2 * qx, 2 * qw, -4 * qz, 2 * qy, 2 * qx, 2 * qy, 0};
    float gq[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < 9; t++) {
        gq[0] += gR[t] * dRw[t]; gq[1] += gR[t] * dRx[t]; gq[2] += gR[t] * dRy[t]; gq[3] += gR[t] * dRz[t];
    }
    const float dot = gq[0] * qw + gq[1] * qx + gq[2] * qy + gq[3] * qz;
    for (int c = 0; c < 4; c++) {
        const float v = (gq[c] - qn[c] * dot) / qnorm;
        d_quat[4 * g + c] = accumulate ? d_quat[4 * g + c] + v : v;
    }
    for (int a = 0; a < 3; a++) {
        d_mean[3 * g + a] = accumulate ? d_mean[3 * g + a] + gmu[a] : gmu[a];
        d_scale[3 * g + a] = accumulate ? d_scale[3 * g + a] + gs[a] : gs[a];
    }
    d_value[g] = accumulate ? d_value[g] + gval : gval;
}

int tiles_of(const pmf_detector* det, int& ntu) {
    ntu = (det->nu + kSplatTile - 1) / kSplatTile;
    return ntu * ((det->nv + kSplatTile - 1) / kSplatTile);
}

pmf_status check_raster(const pmf_detector* det, int32_t P, const pmf_view* views, const pmf_gaussians* g) {
    PMF_REQUIRE(det != nullptr && g != nullptr, "null argument");
    PMF_REQUIRE(det->nu > 0 && det->nv > 0, "detector size must be positive");
    PMF_REQUIRE((int64_t)det->nu * det->nv < ((int64_t)1 << 31), "detector too large");
    int ntu_;
    if (tiles_of(det, ntu_) > kMaxTiles)
        return set_error(PMF_EUNSUPPORTED, "detector has more than %d 16x16 tiles", kMaxTiles);
    PMF_REQUIRE(P >= 0 && P < 65536, "P must be in [0, 65535]");
    PMF_REQUIRE(P == 0 || views != nullptr, "views is null");
    PMF_REQUIRE(g->n >= 0 && g->n < ((int64_t)1 << 32), "n must be in [0, 2^32)");
    PMF_REQUIRE(g->channels == 1, "the rasterizer draws one channel (the reference densities)");
    PMF_REQUIRE(g->kappa > 0.0f, "kappa must be positive");
    PMF_REQUIRE(g->n == 0 || (g->mean && g->scale && g->quat && g->value), "null parameter pointer");
    PMF_REQUIRE((int64_t)P * g->n < ((int64_t)1 << 40), "P * n too large");
    return PMF_OK;
}

// Frames, projected Gaussians and (with count_tiles) per-tile counts, offsets and maxima.
pmf_status raster_prep(const pmf_detector* det, int32_t P, const pmf_view* views, const pmf_gaussians* g,
                       const RasterWs& w, int count_tiles, cudaStream_t s) {
    int ntu;
    const int T = tiles_of(det, ntu);
    if (P == 0) return PMF_OK;
    if (count_tiles) cudaMemsetAsync(w.maxbits, 0, sizeof(unsigned) * (size_t)P, s);
    k_splat_frames<<<(P + 31) / 32, 32, 0, s>>>(views, P, w.frames);
    if (w.C > 0)
        k_splat_prep<<<dim3((unsigned)w.C, (unsigned)P), kPrepThreads, count_tiles ? sizeof(unsigned) * T : 0, s>>>(
            *g, P, det->nu, det->nv, ntu, T, w, count_tiles);
    if (count_tiles) {
        scan_counts(w.chist, (int64_t)P * T * w.C, w.bsum, w.coff, w.total, s);
    }
    return check_launch("gs_rasterize prep");
}

__global__ void k_copy_pairs(const unsigned long long* total, int64_t* out) { *out = (int64_t)*total; }

}  // namespace

PMF_DIAG_ACCESSOR(diag_splat)

}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status gs_rasterize_workspace(const pmf_detector* det, int32_t P, int64_t n, int64_t pair_capacity,
                                  size_t* bytes) {
    PMF_REQUIRE(det != nullptr && bytes != nullptr, "null argument");
    PMF_REQUIRE(det->nu > 0 && det->nv > 0 && P >= 0 && n >= 0 && pair_capacity >= 0, "bad arguments");
    int ntu;
    *bytes = raster_ws_layout(P, n, tiles_of(det, ntu), pair_capacity, nullptr, nullptr);
    return PMF_OK;
}

pmf_status gs_rasterize_count(const pmf_detector* det, int32_t P, const pmf_view* views, const pmf_gaussians* g,
                              int64_t* d_pairs, void* ws, size_t ws_bytes, pmf_stream stream) {
    pmf_status st = check_raster(det, P, views, g);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(d_pairs != nullptr, "d_pairs is null");
    int ntu;
    const int T = tiles_of(det, ntu);
    RasterWs w;
    const size_t need = raster_ws_layout(P, g->n, T, 0, &w, (char*)ws);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (P == 0) return cudaMemsetAsync(d_pairs, 0, sizeof(int64_t), s) == cudaSuccess ? PMF_OK : set_error(PMF_ECUDA, "memset");
    if ((st = raster_prep(det, P, views, g, w, 1, s)) != PMF_OK) return st;
    k_copy_pairs<<<1, 1, 0, s>>>(w.total, d_pairs);
    return check_launch("gs_rasterize_count");
}

pmf_status gs_rasterize(const pmf_detector* det, int32_t P, const pmf_view* views, const pmf_gaussians* g,
                        float* proj, void* ws, size_t ws_bytes, pmf_stream stream) {
    pmf_status st = check_raster(det, P, views, g);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(P == 0 || proj != nullptr, "proj is null");
    if (P == 0) return PMF_OK;
    int ntu;
    const int T = tiles_of(det, ntu);
    // the capacity is whatever the caller's bytes leave after the fixed part
    RasterWs fixed_part;
    const size_t fixed = raster_ws_layout(P, g->n, T, 0, &fixed_part, nullptr);
    if ((st = validate_ws(ws, ws_bytes, fixed)) != PMF_OK) return st;
    const int64_t capacity = (int64_t)((ws_bytes - fixed_part.list_off) / sizeof(unsigned));
    RasterWs w;
    raster_ws_layout(P, g->n, T, capacity, &w, (char*)ws);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = raster_prep(det, P, views, g, w, 1, s)) != PMF_OK) return st;
    if (w.C > 0 && capacity > 0)
        k_splat_fill<<<dim3((unsigned)w.C, (unsigned)P), kPrepThreads, sizeof(unsigned) * T, s>>>(g->n, P, ntu, T, w);
    k_splat_render<<<dim3((unsigned)T, (unsigned)P), kRenderThreads, 0, s>>>(g->n, det->nu, det->nv, ntu, T, g->kappa,
                                                                            w, proj);
    return check_launch("gs_rasterize");
}

pmf_status gs_rasterize_backward(const pmf_detector* det, int32_t P, const pmf_view* views, const pmf_gaussians* g,
                                 const float* d_proj, float* d_mean, float* d_scale, float* d_quat, float* d_value,
                                 int accumulate, void* ws, size_t ws_bytes, pmf_stream stream) {
    pmf_status st = check_raster(det, P, views, g);
    if (st != PMF_OK) return st;
    PMF_REQUIRE(g->n == 0 || (d_mean && d_scale && d_quat && d_value), "null gradient pointer");
    PMF_REQUIRE(P == 0 || d_proj != nullptr, "d_proj is null");
    int ntu;
    const int T = tiles_of(det, ntu);
    RasterWs w;
    const size_t need = raster_ws_layout(P, g->n, T, 0, &w, (char*)ws);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    if (g->n == 0) return PMF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = raster_prep(det, P, views, g, w, 0, s)) != PMF_OK) return st;
    const int64_t pairs = (int64_t)P * g->n;
    if (pairs > 0)
        k_splat_bwd_sums<<<(unsigned)((pairs + kBwdWarps - 1) / kBwdWarps), 32 * kBwdWarps, 0, s>>>(
            g->n, P, det->nu, det->nv, g->kappa, w, d_proj);
    k_splat_bwd_chain<<<(unsigned)((g->n + 127) / 128), 128, 0, s>>>(*g, P, w, d_mean, d_scale, d_quat, d_value,
                                                                    accumulate);
    return check_launch("gs_rasterize_backward");
}

}  // extern "C"
