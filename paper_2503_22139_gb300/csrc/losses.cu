// The terms of the Stage 2-3 objective (Eq. 14) and their gradients, for
// sm_103a:
//  - the L1 (Eq. 10/12) or L2 (Eq. 1) projection loss, the mean over all
//    pixels, with its (sub)gradient;
//  - D-SSIM between rendered and measured projections (Eq. 10/12; SSIM of
//    Zhou et al. 2004 with the customary 11x11 Gaussian window, sigma 1.5,
//    zero padding, C1 = (0.01 range)^2, C2 = (0.03 range)^2);
//  - total variation of a D^3 crop of the reference volume (Eq. 11/14);
//  - the MBC normality loss (Eq. 13).
// Every term follows the same convention: *loss (device scalar) is set to, or
// with accumulate increased by, weight * term, and the gradient buffer
// likewise receives weight * d term.  All reductions run in a fixed order.
//
// D-SSIM: one CTA per 32x8 pixel tile of one projection stages the tile and
// a 5-pixel halo, forms the five windowed moments with two separable passes
// in shared memory and evaluates SSIM and its partial derivatives per pixel.
// The moments are taken about a per-tile shift (the tile's mean) so that
// s^2 = E[x^2] - mu^2 does not cancel in fp32 at projection magnitudes; zero
// padding is honoured exactly through the window mass s inside the image.
// The adjoint blurs the three partial maps with the same (symmetric) window.
#include "pmf_common.cuh"

namespace pmf {
namespace {

constexpr int kTU = 32, kTV = 8;                  // SSIM output tile
constexpr int kHW = 5;                            // window half-width
constexpr int kInU = kTU + 2 * kHW, kInV = kTV + 2 * kHW;
constexpr int kSsimThreads = kTU * kTV;           // one output pixel per thread

// The normalised 1-D Gaussian window (sigma 1.5, 11 taps): w[t] for offset t - 5.
struct Window {
    float w[11];
};

Window make_window() {
    Window W;
    double s = 0.0, v[11];
    for (int t = 0; t < 11; t++) {
        const double d = (double)(t - kHW);
        v[t] = exp(-d * d / (2.0 * 1.5 * 1.5));
        s += v[t];
    }
    for (int t = 0; t < 11; t++) W.w[t] = (float)(v[t] / s);
    return W;
}

// Window mass inside [0, n) for a window centred at i.
__device__ __forceinline__ float inside_mass(const Window& W, int i, int n) {
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < 11; t++) {
        const int j = i + t - kHW;
        if (j >= 0 && j < n) s += W.w[t];
    }
    return s;
}

__device__ __forceinline__ float block_sum_f(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int i = 0; i < nw; i++) t += red[i];  // fixed order, same in every thread
    return t;
}

// Forward: per pixel S and the partials G1 = dS/dmu_x - 2 mu_x G2 - mu_y G3,
// G2 = dS/d s_x^2, G3 = dS/d s_xy (with dS/dmu_x taken at fixed s's), so that
// dS(q)/dx(r) = w(q - r) (G1(q) + 2 x(r) G2(q) + y(r) G3(q)).
__global__ void __launch_bounds__(kSsimThreads) k_dssim_fwd(int nu, int nv, int ntu, const float* __restrict__ X,
                                                           const float* __restrict__ Y, float C1, float C2,
                                                           const Window W, float* G, double* part) {
    __shared__ float sx[kInV][kInU], sy[kInV][kInU];
    __shared__ float h[5][kInV][kTU];
    __shared__ float red[kSsimThreads / 32];
    const int p = blockIdx.y, tu = blockIdx.x % ntu, tv = blockIdx.x / ntu;
    const int u0 = tu * kTU - kHW, v0 = tv * kTV - kHW;
    const int64_t Q = (int64_t)nu * nv;
    const float* Xp = X + (int64_t)p * Q;
    const float* Yp = Y + (int64_t)p * Q;
    // stage the tile and halo (zero outside the image) and its mean over the image part
    float ax = 0.f, ay = 0.f, cnt = 0.f;
    for (int i = threadIdx.x; i < kInU * kInV; i += kSsimThreads) {
        const int r = i / kInU, c = i - r * kInU;
        const int u = u0 + c, v = v0 + r;
        const bool in = u >= 0 && u < nu && v >= 0 && v < nv;
        const float x = in ? __ldg(Xp + (int64_t)v * nu + u) : 0.f, y = in ? __ldg(Yp + (int64_t)v * nu + u) : 0.f;
        sx[r][c] = x;
        sy[r][c] = y;
        ax += x;
        ay += y;
        cnt += in ? 1.f : 0.f;
    }
    const float n_in = block_sum_f(cnt, red);
    const float cx = block_sum_f(ax, red) / n_in, cy = block_sum_f(ay, red) / n_in;
    // shift inside the image (outside stays zero)
    for (int i = threadIdx.x; i < kInU * kInV; i += kSsimThreads) {
        const int r = i / kInU, c = i - r * kInU;
        const int u = u0 + c, v = v0 + r;
        if (u >= 0 && u < nu && v >= 0 && v < nv) {
            sx[r][c] -= cx;
            sy[r][c] -= cy;
        }
    }
    __syncthreads();
    // horizontal pass: 5 sums for every staged row and output column
    for (int i = threadIdx.x; i < kInV * kTU; i += kSsimThreads) {
        const int r = i / kTU, c = i - r * kTU;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
        for (int t = 0; t < 11; t++) {
            const float x = sx[r][c + t], y = sy[r][c + t], wt = W.w[t];
            m0 = fmaf(wt, x, m0);
            m1 = fmaf(wt, y, m1);
            m2 = fmaf(wt * x, x, m2);
            m3 = fmaf(wt * y, y, m3);
            m4 = fmaf(wt * x, y, m4);
        }
        h[0][r][c] = m0; h[1][r][c] = m1; h[2][r][c] = m2; h[3][r][c] = m3; h[4][r][c] = m4;
    }
    __syncthreads();
    const int c = threadIdx.x % kTU, r = threadIdx.x / kTU;
    const int u = tu * kTU + c, v = tv * kTV + r;
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t < 11; t++)
#pragma unroll
        for (int k = 0; k < 5; k++) m[k] = fmaf(W.w[t], h[k][r + t][c], m[k]);
    float S = 0.f;
    if (u < nu && v < nv) {
        // moments about the shift: mu = mu' + c s, s^2 = E'[x^2] - mu'^2 + 2 c mu' (1 - s) + c^2 s (1 - s)
        const float s = inside_mass(W, u, nu) * inside_mass(W, v, nv), s1 = 1.f - s;
        const float mx = fmaf(cx, s, m[0]), my = fmaf(cy, s, m[1]);
        const float vxx = fmaf(cx * s, cx * s1, fmaf(2.f * cx * s1, m[0], m[2] - m[0] * m[0]));
        const float vyy = fmaf(cy * s, cy * s1, fmaf(2.f * cy * s1, m[1], m[3] - m[1] * m[1]));
        const float vxy = fmaf(cx * s, cy * s1, fmaf(s1, fmaf(cx, m[1], cy * m[0]), m[4] - m[0] * m[1]));
        const float A1 = fmaf(2.f * mx, my, C1), A2 = fmaf(2.f, vxy, C2);
        const float B1 = fmaf(mx, mx, fmaf(my, my, C1)), B2 = vxx + vyy + C2;
        const float iB = 1.f / (B1 * B2);
        S = A1 * A2 * iB;
        const float G2 = -S / B2, G3 = 2.f * A1 * iB;
        const float D = 2.f * my * A2 * iB - 2.f * mx * S / B1;  // dS/dmu_x at fixed s's
        const float G1 = D - 2.f * mx * G2 - my * G3;
        const int64_t q = (int64_t)p * Q + (int64_t)v * nu + u;
        const int64_t PQ = Q * gridDim.y;
        G[q] = G1;
        G[PQ + q] = G2;
        G[2 * PQ + q] = G3;
    }
    const float tot = block_sum_f(S, red);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = (double)tot;
}

// Adjoint: d_pred = scale (w * G1 + 2 x w * G2 + y w * G3), scale = -weight / (P Q).
__global__ void __launch_bounds__(kSsimThreads) k_dssim_bwd(int nu, int nv, int ntu, const float* __restrict__ X,
                                                           const float* __restrict__ Y, const float* __restrict__ G,
                                                           const Window W, float scale, float* d_pred,
                                                           int accumulate) {
    __shared__ float sg[3][kInV][kInU];
    __shared__ float h[3][kInV][kTU];
    const int p = blockIdx.y, tu = blockIdx.x % ntu, tv = blockIdx.x / ntu;
    const int u0 = tu * kTU - kHW, v0 = tv * kTV - kHW;
    const int64_t Q = (int64_t)nu * nv, PQ = Q * gridDim.y;
    for (int i = threadIdx.x; i < kInU * kInV; i += kSsimThreads) {
        const int r = i / kInU, c = i - r * kInU;
        const int u = u0 + c, v = v0 + r;
        const bool in = u >= 0 && u < nu && v >= 0 && v < nv;
        const int64_t q = (int64_t)p * Q + (int64_t)v * nu + u;
#pragma unroll
        for (int k = 0; k < 3; k++) sg[k][r][c] = in ? __ldg(G + k * PQ + q) : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kInV * kTU; i += kSsimThreads) {
        const int r = i / kTU, c = i - r * kTU;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int t = 0; t < 11; t++) {
            a0 = fmaf(W.w[t], sg[0][r][c + t], a0);
            a1 = fmaf(W.w[t], sg[1][r][c + t], a1);
            a2 = fmaf(W.w[t], sg[2][r][c + t], a2);
        }
        h[0][r][c] = a0; h[1][r][c] = a1; h[2][r][c] = a2;
    }
    __syncthreads();
    const int c = threadIdx.x % kTU, r = threadIdx.x / kTU;
    const int u = tu * kTU + c, v = tv * kTV + r;
    if (u >= nu || v >= nv) return;
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
    for (int t = 0; t < 11; t++) {
        b0 = fmaf(W.w[t], h[0][r + t][c], b0);
        b1 = fmaf(W.w[t], h[1][r + t][c], b1);
        b2 = fmaf(W.w[t], h[2][r + t][c], b2);
    }
    const int64_t q = (int64_t)p * Q + (int64_t)v * nu + u;
    const float g = scale * fmaf(2.f * __ldg(X + q), b1, fmaf(__ldg(Y + q), b2, b0));
    d_pred[q] = accumulate ? d_pred[q] + g : g;
}

// loss (=/+=) weight * (1 - sum S / (P Q)), partials summed in order in double.
__global__ void k_dssim_final(const double* part, int n, double pq, float weight, float* loss, int accumulate) {
    __shared__ double red[32];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
        const float v = (float)((double)weight * (1.0 - s / pq));
        *loss = accumulate ? *loss + v : v;
    }
}

// ------------------------------------------------------------------- TV

constexpr int kTvThreads = 256;

// The crop origin, clamped so that the D^3 crop lies in the grid.
__device__ __forceinline__ void crop_origin(const int* o, const GridD& g, int D, int c[3]) {
    const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int a = 0; a < 3; a++) c[a] = min(max(o[a], 0), n[a] - D);
}

// One thread per crop voxel: its three forward differences (into the loss)
// and its subgradient (from the differences it takes part in), no atomics.
template <typename T>
__global__ void __launch_bounds__(kTvThreads) k_tv(GridD g, int D, const int* __restrict__ origin,
                                                  const T* __restrict__ V, float gscale, float* d_vol,
                                                  int accumulate, double* part) {
    __shared__ float red[kTvThreads / 32];
    int o[3];
    crop_origin(origin, g, D, o);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n3 = (int64_t)D * D * D;
    float s = 0.f;
    if (t < n3) {
        const int x = (int)(t % D), y = (int)((t / D) % D), z = (int)(t / ((int64_t)D * D));
        const int c[3] = {x, y, z};
        const int64_t v = ((int64_t)(o[2] + z) * g.ny + (o[1] + y)) * g.nx + (o[0] + x);
        const int64_t step[3] = {1, g.nx, (int64_t)g.nx * g.ny};
        const float val = Store<T>::ld(V, v);
        float gsum = 0.f;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (c[a] + 1 < D) {
                const float d = Store<T>::ld(V, v + step[a]) - val;
                s += fabsf(d);
                gsum -= (d > 0.f) ? 1.f : (d < 0.f ? -1.f : 0.f);
            }
            if (c[a] > 0) {
                const float d = val - Store<T>::ld(V, v - step[a]);
                gsum += (d > 0.f) ? 1.f : (d < 0.f ? -1.f : 0.f);
            }
        }
        if (d_vol) {
            const float gv = gscale * gsum;
            d_vol[v] = accumulate ? d_vol[v] + gv : gv;
        }
    }
    const float tot = block_sum_f(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = (double)tot;
}

__global__ void k_sum_final(const double* part, int n, double mult, float* loss, int accumulate) {
    __shared__ double red[32];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
        const float v = (float)(s * mult);
        *loss = accumulate ? *loss + v : v;
    }
}

// ---------------------------------------------------------- normality

constexpr int kNormBlocks = 152;   // partial sums per MBC component (fixed: order independent of the device)

// part[lk][b] = sum of squares of component lk over block b's grid-stride range (double).
template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(const T* __restrict__ E, int64_t N, double* part) {
    __shared__ double red[8];
    const int lk = blockIdx.y;
    const T* e = E + (int64_t)lk * N;
    float sf = 0.f;  // a thread's own few hundred squares in fp32, then double
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const float x = Store<T>::ld(e, v);
        sf = fmaf(x, x, sf);
    }
    double s = (double)sf;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; i++) t += red[i];
        part[(int64_t)lk * gridDim.x + blockIdx.x] = t;
    }
}

// norms[lk] = sum of its partials; loss (=/+=) weight / (3L) sum (norm - 1)^2.
__global__ void k_norm_final(const double* part, int nb, int nlk, double* norms, float weight, float* loss,
                             int accumulate) {
    if (threadIdx.x != 0) return;
    double tot = 0.0;
    for (int lk = 0; lk < nlk; lk++) {
        double n2 = 0.0;
        for (int b = 0; b < nb; b++) n2 += part[(int64_t)lk * nb + b];
        norms[lk] = n2;
        tot += (n2 - 1.0) * (n2 - 1.0);
    }
    const float v = (float)((double)weight * tot / (double)nlk);
    *loss = accumulate ? *loss + v : v;
}

// dE (=/+=) weight * 4 (norm - 1) e / (3L).
template <typename T>
__global__ void __launch_bounds__(256) k_norm_grad(const T* __restrict__ E, int64_t N, int nlk,
                                                   const double* __restrict__ norms, float weight, float* dE,
                                                   int accumulate) {
    const int lk = blockIdx.y;
    const float f = (float)((double)weight * 4.0 * (norms[lk] - 1.0) / (double)nlk);
    const T* e = E + (int64_t)lk * N;
    float* d = dE + (int64_t)lk * N;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const float g = f * Store<T>::ld(e, v);
        d[v] = accumulate ? d[v] + g : g;
    }
}

int ssim_tiles(int nu, int nv) { return ((nu + kTU - 1) / kTU) * ((nv + kTV - 1) / kTV); }

// ------------------------------------------ L1 / L2 projection loss (Eq. 10/12, Eq. 1)

constexpr int kLossThreads = 256;

__device__ __forceinline__ float loss_term(int kind, float r, float invn, float& g) {
    if (kind == 1) {
        g = r > 0.0f ? invn : (r < 0.0f ? -invn : 0.0f);
        return fabsf(r);
    }
    g = 2.0f * r * invn;
    return r * r;
}

// Per-block partial sums of the loss and, optionally, its gradient.  VEC: the
// arrays are 16-byte aligned and each thread takes two float4 groups per
// iteration (more bytes in flight per thread than scalar loads); the n % 4 tail
// goes to block 0.
template <bool VEC>
__global__ void __launch_bounds__(kLossThreads) k_loss(int kind, int64_t n, const float* __restrict__ pred,
                                                       const float* __restrict__ meas, float* d_pred, float* part) {
    __shared__ float red[kLossThreads / 32];
    const float invn = 1.0f / (float)n;
    float s = 0.0f, gr;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    if (VEC) {
        const int64_t n4 = n >> 2;
        const float4* p4 = reinterpret_cast<const float4*>(pred);
        const float4* m4 = reinterpret_cast<const float4*>(meas);
        float4* d4 = reinterpret_cast<float4*>(d_pred);
        for (int64_t t = tid; t < n4; t += 2 * nt) {
            const bool two = t + nt < n4;
            const float4 a = __ldg(p4 + t), b = __ldg(m4 + t);
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f), e = c;
            if (two) { c = __ldg(p4 + t + nt); e = __ldg(m4 + t + nt); }
            float4 g;
            s += loss_term(kind, a.x - b.x, invn, g.x);
            s += loss_term(kind, a.y - b.y, invn, g.y);
            s += loss_term(kind, a.z - b.z, invn, g.z);
            s += loss_term(kind, a.w - b.w, invn, g.w);
            if (d_pred) d4[t] = g;
            if (two) {
                s += loss_term(kind, c.x - e.x, invn, g.x);
                s += loss_term(kind, c.y - e.y, invn, g.y);
                s += loss_term(kind, c.z - e.z, invn, g.z);
                s += loss_term(kind, c.w - e.w, invn, g.w);
                if (d_pred) d4[t + nt] = g;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            const int64_t t = (n4 << 2) + threadIdx.x;
            s += loss_term(kind, __ldg(pred + t) - __ldg(meas + t), invn, gr);
            if (d_pred) d_pred[t] = gr;
        }
    } else {
        for (int64_t t = tid; t < n; t += nt) {
            s += loss_term(kind, __ldg(pred + t) - __ldg(meas + t), invn, gr);
            if (d_pred) d_pred[t] = gr;
        }
    }
    const float tot = block_sum<kLossThreads>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// One CTA: strided partial sums in double, a fixed butterfly per warp and the
// warps in order, so the order of every addition is fixed.
__global__ void k_loss_final(const float* part, int nb, int64_t n, float* loss) {
    __shared__ double red[kLossThreads / 32];
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += (double)part[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kLossThreads / 32; i++) s += red[i];
        *loss = (float)(s / (double)n);
    }
}

}  // namespace
}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status projection_dssim_workspace(int32_t P, int32_t nu, int32_t nv, size_t* bytes) {
    PMF_REQUIRE(bytes != nullptr && P >= 0 && nu >= 0 && nv >= 0, "bad arguments");
    *bytes = align_up(sizeof(float) * 3 * (size_t)P * nu * nv) +
             align_up(sizeof(double) * (size_t)P * ssim_tiles(nu, nv));
    return PMF_OK;
}

pmf_status projection_dssim(int32_t P, int32_t nu, int32_t nv, const float* pred, const float* meas, float data_range,
                            float weight, float* loss, float* d_pred, int accumulate, void* ws, size_t ws_bytes,
                            pmf_stream stream) {
    PMF_REQUIRE(P >= 1 && nu >= 1 && nv >= 1, "P, nu and nv must be positive");
    PMF_REQUIRE(pred && meas && loss, "null pointer");
    PMF_REQUIRE(data_range > 0.f && isfinite(data_range), "data_range must be positive");
    PMF_REQUIRE(isfinite(weight), "weight must be finite");
    PMF_REQUIRE(P <= 65535, "P must be <= 65535");
    size_t need;
    projection_dssim_workspace(P, nu, nv, &need);
    pmf_status st = validate_ws(ws, ws_bytes, need);
    if (st != PMF_OK) return st;
    float* G = (float*)ws;
    double* part = (double*)((char*)ws + align_up(sizeof(float) * 3 * (size_t)P * nu * nv));
    const Window W = make_window();
    const float C1 = (0.01f * data_range) * (0.01f * data_range), C2 = (0.03f * data_range) * (0.03f * data_range);
    const int ntu = (nu + kTU - 1) / kTU, nt = ssim_tiles(nu, nv);
    cudaStream_t s = (cudaStream_t)stream;
    k_dssim_fwd<<<dim3((unsigned)nt, (unsigned)P), kSsimThreads, 0, s>>>(nu, nv, ntu, pred, meas, C1, C2, W, G, part);
    if (d_pred) {
        const float scale = -weight / ((float)P * (float)nu * (float)nv);
        k_dssim_bwd<<<dim3((unsigned)nt, (unsigned)P), kSsimThreads, 0, s>>>(nu, nv, ntu, pred, meas, G, W, scale,
                                                                          d_pred, accumulate);
    }
    k_dssim_final<<<1, 256, 0, s>>>(part, nt * P, (double)P * nu * nv, weight, loss, accumulate);
    return check_launch("projection_dssim");
}

pmf_status tv_loss_workspace(int32_t D, size_t* bytes) {
    PMF_REQUIRE(bytes != nullptr && D >= 0, "bad arguments");
    const int64_t n3 = (int64_t)D * D * D;
    *bytes = align_up(sizeof(double) * (size_t)((n3 + kTvThreads - 1) / kTvThreads + 1));
    return PMF_OK;
}

pmf_status tv_loss(const pmf_grid* grid, pmf_dtype dtype, const void* vol, int32_t D, const int32_t* d_origin,
                   float weight, float* loss, float* d_vol, int accumulate, void* ws, size_t ws_bytes,
                   pmf_stream stream) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    if ((st = validate_dtype(dtype)) != PMF_OK) return st;
    PMF_REQUIRE(vol && d_origin && loss, "null pointer");
    PMF_REQUIRE(D >= 2 && D <= grid->nx && D <= grid->ny && D <= grid->nz, "crop size D must be in [2, min(n)]");
    PMF_REQUIRE(isfinite(weight), "weight must be finite");
    size_t need;
    tv_loss_workspace(D, &need);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    GridD g = make_grid(grid);
    const int64_t n3 = (int64_t)D * D * D;
    const unsigned nb = (unsigned)((n3 + kTvThreads - 1) / kTvThreads);
    const double per_axis = (double)(D - 1) * D * D;
    const float gscale = (float)((double)weight / (3.0 * per_axis));
    cudaStream_t s = (cudaStream_t)stream;
    double* part = (double*)ws;
    if (d_vol && !accumulate) cudaMemsetAsync(d_vol, 0, sizeof(float) * (size_t)g.n, s);
    PMF_DISPATCH_DTYPE(dtype, T, k_tv<T><<<nb, kTvThreads, 0, s>>>(g, D, d_origin, (const T*)vol, gscale, d_vol, accumulate, part));
    k_sum_final<<<1, 256, 0, s>>>(part, (int)nb, (double)weight / (3.0 * per_axis), loss, accumulate);
    return check_launch("tv_loss");
}

pmf_status mbc_normality_workspace(int32_t L, size_t* bytes) {
    PMF_REQUIRE(bytes != nullptr && L >= 0, "bad arguments");
    *bytes = align_up(sizeof(double) * (size_t)3 * L * kNormBlocks) + align_up(sizeof(double) * (size_t)3 * L);
    return PMF_OK;
}

pmf_status mbc_normality(const pmf_grid* grid, int32_t L, pmf_dtype dtype, const void* mbc, float weight, float* loss,
                         float* d_mbc, int accumulate, void* ws, size_t ws_bytes, pmf_stream stream) {
    pmf_status st = validate_grid(grid);
    if (st != PMF_OK) return st;
    if ((st = validate_dtype(dtype)) != PMF_OK) return st;
    PMF_REQUIRE(L >= 1 && L <= 64, "L must be in [1, 64]");
    PMF_REQUIRE(mbc && loss, "null pointer");
    PMF_REQUIRE(isfinite(weight), "weight must be finite");
    size_t need;
    mbc_normality_workspace(L, &need);
    if ((st = validate_ws(ws, ws_bytes, need)) != PMF_OK) return st;
    const int64_t N = (int64_t)grid->nx * grid->ny * grid->nz;
    double* part = (double*)ws;
    double* norms = (double*)((char*)ws + align_up(sizeof(double) * (size_t)3 * L * kNormBlocks));
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 gr(kNormBlocks, (unsigned)(3 * L));
    PMF_DISPATCH_DTYPE(dtype, T, k_sumsq<T><<<gr, 256, 0, s>>>((const T*)mbc, N, part));
    k_norm_final<<<1, 32, 0, s>>>(part, kNormBlocks, 3 * L, norms, weight, loss, accumulate);
    if (d_mbc) {
        const int64_t nb = (N + 255) / 256;
        const dim3 gg((unsigned)(nb < 4 * kStreamBlocks ? nb : 4 * kStreamBlocks), (unsigned)(3 * L));
        PMF_DISPATCH_DTYPE(dtype, T, k_norm_grad<T><<<gg, 256, 0, s>>>((const T*)mbc, N, 3 * L, norms, weight, d_mbc, accumulate));
    }
    return check_launch("mbc_normality");
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
    const bool vec = (((uintptr_t)pred | (uintptr_t)meas | (uintptr_t)d_pred) & 15) == 0;
    if (vec)
        k_loss<true><<<blocks, kLossThreads, 0, s>>>(kind, n, pred, meas, d_pred, (float*)ws);
    else
        k_loss<false><<<blocks, kLossThreads, 0, s>>>(kind, n, pred, meas, d_pred, (float*)ws);
    k_loss_final<<<1, kLossThreads, 0, s>>>((const float*)ws, blocks, n, loss);
    return check_launch("projection_loss");
}
}  // extern "C"
