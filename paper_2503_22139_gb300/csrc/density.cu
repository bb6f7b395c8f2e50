// Adaptive density control of a Gaussian set (Sec. 2.3.2) for sm_103a:
//   k_grad_norm_acc  acc[i] += |dL/dmean_i| over the steps between controls
//   k_select_desc    the densification threshold: the (rank + 1)-th largest
//                    statistic (radix select, one CTA)
//   k_dc_count       per Gaussian the action (remove, keep, clone, split) and
//                    how many Gaussians it leaves (0, 1, 2, 2)
//   scan_counts      output offsets (order-preserving, deterministic)
//   k_dc_emit        the controlled set: kept Gaussians copied, clones as two
//                    copies at half density, splits as two Gaussians drawn from
//                    the parent (mean + R diag(s) z_k, scales s / split_factor)
//                    at half density, in input order
#include "pmf_common.cuh"
#include "scan.cuh"

namespace pmf {
namespace {

constexpr int kDcThreads = 256;

__global__ void k_grad_norm_acc(int64_t n, const float* __restrict__ d_mean, float* __restrict__ acc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = d_mean[3 * i], y = d_mean[3 * i + 1], z = d_mean[3 * i + 2];
        acc[i] += sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
    }
}

__global__ void k_dc_count(pmf_gaussians G, const float* __restrict__ acc, float grad_scale, float grad_threshold,
                           float scale_threshold, float value_threshold, unsigned char* __restrict__ act,
                           unsigned* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    bool empty = true;
    for (int c = 0; c < G.channels; c++) empty = empty && fabsf(__ldg(G.value + i * G.channels + c)) < value_threshold;
    unsigned char a = 1;
    if (empty) {
        a = 0;
    } else if (__ldg(acc + i) * grad_scale > grad_threshold) {
        const float smax = fmaxf(fmaxf(__ldg(G.scale + 3 * i), __ldg(G.scale + 3 * i + 1)), __ldg(G.scale + 3 * i + 2));
        a = smax <= scale_threshold ? 2 : 3;
    }
    act[i] = a;
    cnt[i] = a == 0 ? 0u : (a == 1 ? 1u : 2u);
}

__global__ void k_dc_emit(pmf_gaussians G, const unsigned char* __restrict__ act, const unsigned* __restrict__ off,
                          const float* __restrict__ noise, float split_factor, float* __restrict__ om,
                          float* __restrict__ os, float* __restrict__ oq, float* __restrict__ ov) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    const unsigned char a = act[i];
    if (a == 0) return;
    const int64_t o = off[i];
    const int C = G.channels;
    const float mu[3] = {G.mean[3 * i], G.mean[3 * i + 1], G.mean[3 * i + 2]};
    const float s[3] = {G.scale[3 * i], G.scale[3 * i + 1], G.scale[3 * i + 2]};
    const float q[4] = {G.quat[4 * i], G.quat[4 * i + 1], G.quat[4 * i + 2], G.quat[4 * i + 3]};
    const int copies = a == 1 ? 1 : 2;
    const float vs = a == 1 ? 1.0f : 0.5f;
    float R[9];
    if (a == 3) {
        const float nrm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float w = q[0] / nrm, x = q[1] / nrm, y = q[2] / nrm, z = q[3] / nrm;
        R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
        R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
        R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    }
    for (int k = 0; k < copies; k++) {
        const int64_t j = o + k;
        for (int t = 0; t < 3; t++) {
            float m = mu[t];
            if (a == 3) {
                const float* zk = noise + (i * 2 + k) * 3;
                m = fmaf(R[3 * t], s[0] * zk[0], fmaf(R[3 * t + 1], s[1] * zk[1], fmaf(R[3 * t + 2], s[2] * zk[2], m)));
            }
            om[3 * j + t] = m;
            os[3 * j + t] = a == 3 ? s[t] / split_factor : s[t];
        }
        for (int t = 0; t < 4; t++) oq[4 * j + t] = q[t];
        for (int c = 0; c < C; c++) ov[j * C + c] = vs * G.value[i * C + c];
    }
}

__global__ void k_dc_total(const unsigned long long* total, int64_t* out) { *out = (int64_t)*total; }

// Order-preserving key of a float: larger floats get larger unsigned keys
// (negative values have their bits inverted, the rest the sign bit set).
__device__ __forceinline__ unsigned order_key(float v) {
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_value(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The (rank + 1)-th largest of acc[i] * scale (fp32 products), by a radix
// select on the order keys, eight bits per pass from the top: each pass counts
// the digit of the keys that match the digits chosen so far and keeps the bin
// holding the wanted rank.  One CTA; exact, and independent of thread timing.
constexpr int kSelThreads = 1024;

__global__ void __launch_bounds__(kSelThreads) k_select_desc(int64_t n, const float* __restrict__ acc, float scale,
                                                            int64_t rank, float* out) {
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_want;
    if (threadIdx.x == 0) {
        s_prefix = 0u;
        s_want = (unsigned)rank;
    }
    unsigned mask = 0u;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
        const unsigned prefix = s_prefix;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned k = order_key(__fmul_rn(__ldg(acc + i), scale));
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 0xffu], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned want = s_want, b = 255u;
            for (;; b--) {  // the wanted rank lies in the bin where the count from the top passes it
                if (want < hist[b] || b == 0u) break;
                want -= hist[b];
            }
            s_want = want;
            s_prefix = prefix | (b << shift);
        }
        mask |= 0xffu << shift;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = key_value(s_prefix);
}

struct DcWs {
    unsigned char* act;
    unsigned* cnt;
    unsigned* off;
    unsigned long long* bsum;
    unsigned long long* total;
};

size_t dc_layout(int64_t n, DcWs* w, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return base ? base + o : nullptr;
    };
    const size_t m = (size_t)(n > 0 ? n : 1);
    DcWs x;
    x.act = (unsigned char*)take(m);
    x.cnt = (unsigned*)take(sizeof(unsigned) * m);
    x.off = (unsigned*)take(sizeof(unsigned) * (m + 1));
    x.bsum = (unsigned long long*)take(sizeof(unsigned long long) * (size_t)(scan_blocks(n) + 2));
    x.total = (unsigned long long*)take(sizeof(unsigned long long));
    if (w) *w = x;
    return off;
}

}  // namespace
}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status gs_grad_norm_accumulate(int64_t n, const float* d_mean, float* acc, pmf_stream stream) {
    PMF_REQUIRE(n >= 0, "n must be >= 0");
    PMF_REQUIRE(n == 0 || (d_mean && acc), "null pointer");
    if (n == 0) return PMF_OK;
    const int64_t nb = (n + kDcThreads - 1) / kDcThreads;
    k_grad_norm_acc<<<(unsigned)(nb < 4 * kStreamBlocks ? nb : 4 * kStreamBlocks), kDcThreads, 0,
                      (cudaStream_t)stream>>>(n, d_mean, acc);
    return check_launch("gs_grad_norm_accumulate");
}

pmf_status gs_density_threshold(int64_t n, const float* grad_acc, float grad_scale, int64_t rank, float* d_threshold,
                                pmf_stream stream) {
    PMF_REQUIRE(n > 0 && n < ((int64_t)1 << 31), "n must be in [1, 2^31)");
    PMF_REQUIRE(rank >= 0 && rank < n, "rank must be in [0, n)");
    PMF_REQUIRE(grad_acc != nullptr && d_threshold != nullptr, "null pointer");
    PMF_REQUIRE(isfinite(grad_scale), "grad_scale must be finite");
    k_select_desc<<<1, kSelThreads, 0, (cudaStream_t)stream>>>(n, grad_acc, grad_scale, rank, d_threshold);
    return check_launch("gs_density_threshold");
}

pmf_status gs_density_control_workspace(int64_t n, size_t* bytes) {
    PMF_REQUIRE(bytes != nullptr && n >= 0, "bad arguments");
    *bytes = dc_layout(n, nullptr, nullptr);
    return PMF_OK;
}

pmf_status gs_density_control(const pmf_gaussians* in, const float* grad_acc, float grad_scale, const float* noise,
                              float grad_threshold, float scale_threshold, float value_threshold, float split_factor,
                              float* out_mean, float* out_scale, float* out_quat, float* out_value,
                              int64_t out_capacity, int64_t* d_count, void* ws, size_t ws_bytes, pmf_stream stream) {
    PMF_REQUIRE(in != nullptr && d_count != nullptr, "null argument");
    PMF_REQUIRE(in->n >= 0 && in->n < ((int64_t)1 << 31), "n must be in [0, 2^31)");
    PMF_REQUIRE(in->channels >= 1 && in->channels <= 16, "channels must be in [1, 16]");
    PMF_REQUIRE(in->n == 0 || (in->mean && in->scale && in->quat && in->value && grad_acc && noise), "null pointer");
    PMF_REQUIRE(out_capacity >= 2 * in->n, "out_capacity must be at least 2 n");
    PMF_REQUIRE(in->n == 0 || (out_mean && out_scale && out_quat && out_value), "null output pointer");
    PMF_REQUIRE(isfinite(grad_scale) && isfinite(grad_threshold) && isfinite(scale_threshold) &&
                    isfinite(value_threshold) && split_factor > 0.0f && isfinite(split_factor),
                "thresholds must be finite and split_factor positive");
    DcWs w;
    const size_t need = dc_layout(in->n, &w, (char*)ws);
    pmf_status st = validate_ws(ws, ws_bytes, need);
    if (st != PMF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned nb = (unsigned)((in->n + kDcThreads - 1) / kDcThreads);
    if (in->n > 0)
        k_dc_count<<<nb, kDcThreads, 0, s>>>(*in, grad_acc, grad_scale, grad_threshold, scale_threshold,
                                             value_threshold, w.act, w.cnt);
    scan_counts(w.cnt, in->n, w.bsum, w.off, w.total, s);
    if (in->n > 0)
        k_dc_emit<<<nb, kDcThreads, 0, s>>>(*in, w.act, w.off, noise, split_factor, out_mean, out_scale, out_quat,
                                            out_value);
    k_dc_total<<<1, 1, 0, s>>>(w.total, d_count);
    return check_launch("gs_density_control");
}

}  // extern "C"
