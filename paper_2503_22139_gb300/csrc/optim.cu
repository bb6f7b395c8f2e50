// The optimiser update the training loop of Sec. 2.3.2 uses: Adam (Kingma &
// Ba 2014), one fused element-wise pass per parameter tensor, in place (and a
// translation of Gaussian means, for voxelizing a sub-volume):
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   p = p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
#include "pmf_common.cuh"

namespace pmf {
namespace {

__global__ void __launch_bounds__(256) k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                                              float b2, float eps, float ibc1, float isbc2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * ibc1) / (sqrtf(vi) * isbc2 + eps);
    }
}

__global__ void k_shift_means(int64_t n, const float* __restrict__ mean, const float* __restrict__ off,
                              float* __restrict__ out) {
    const float o[3] = {off[0], off[1], off[2]};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = mean[i] - o[i % 3];
}

}  // namespace
}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status pmf_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                         float beta2, float eps, int32_t t, pmf_stream stream) {
    PMF_REQUIRE(n >= 0, "n must be >= 0");
    PMF_REQUIRE(n == 0 || (param && grad && m && v), "null pointer");
    PMF_REQUIRE(t >= 1, "step t must be >= 1");
    PMF_REQUIRE(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f, "betas must be in [0, 1)");
    PMF_REQUIRE(eps > 0.f && isfinite(lr), "eps must be positive and lr finite");
    if (n == 0) return PMF_OK;
    const double bc1 = 1.0 - pow((double)beta1, (double)t), bc2 = 1.0 - pow((double)beta2, (double)t);
    const int64_t nb = (n + 255) / 256;
    k_adam<<<(unsigned)(nb < 4 * kStreamBlocks ? nb : 4 * kStreamBlocks), 256, 0, (cudaStream_t)stream>>>(
        n, param, grad, m, v, lr, beta1, beta2, eps, (float)(1.0 / bc1), (float)(1.0 / sqrt(bc2)));
    return check_launch("pmf_adam_step");
}

pmf_status pmf_shift_means(int64_t n, const float* mean, const float* offset, float* out, pmf_stream stream) {
    PMF_REQUIRE(n >= 0, "n must be >= 0");
    PMF_REQUIRE(n == 0 || (mean && offset && out), "null pointer");
    if (n == 0) return PMF_OK;
    const int64_t nb = (3 * n + 255) / 256;
    k_shift_means<<<(unsigned)(nb < 4 * kStreamBlocks ? nb : 4 * kStreamBlocks), 256, 0, (cudaStream_t)stream>>>(
        n, mean, offset, out);
    return check_launch("pmf_shift_means");
}

}  // extern "C"
