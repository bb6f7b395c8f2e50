// Exclusive prefix sums of unsigned counts (64-bit running sums, stored
// clamped to 32 bits) in three passes: block totals, a one-CTA scan of the
// totals (which also writes the grand total), and the per-block scans.  The
// order of every sum is fixed, so the offsets are deterministic.  Used by the
// rasterizer's tile lists and by density control's stream compaction.
#pragma once

#include "pmf_common.cuh"

namespace pmf {
namespace {

constexpr int kScanItems = 4096;  // 256 threads x 16 per scan block

__global__ void k_scan_reduce(const unsigned* __restrict__ x, int64_t N, unsigned long long* bsum) {
    __shared__ unsigned long long part[8];
    const int64_t b0 = (int64_t)blockIdx.x * kScanItems + threadIdx.x * 16;
    unsigned long long s = 0;
    for (int k = 0; k < 16; k++)
        if (b0 + k < N) s += x[b0 + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < 8; i++) t += part[i];
        bsum[blockIdx.x] = t;
    }
}

__global__ void k_scan_top(unsigned long long* bsum, int nb, int64_t N, unsigned* coff,
                           unsigned long long* total) {
    __shared__ unsigned long long part[1024];
    const int tid = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    const int b = tid * per, e = b + per < nb ? b + per : nb;
    unsigned long long s = 0;
    for (int i = b; i < e; i++) s += bsum[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < 1024; i++) {
            const unsigned long long v = part[i];
            part[i] = run;
            run += v;
        }
        *total = run;
        coff[N] = (unsigned)(run > 0xffffffffull ? 0xffffffffull : run);
    }
    __syncthreads();
    unsigned long long run = part[tid];
    for (int i = b; i < e; i++) {
        const unsigned long long v = bsum[i];
        bsum[i] = run;
        run += v;
    }
}

__global__ void k_scan_apply(const unsigned* __restrict__ x, int64_t N, const unsigned long long* bsum, unsigned* coff) {
    __shared__ unsigned long long part[256];
    const int64_t b0 = (int64_t)blockIdx.x * kScanItems + threadIdx.x * 16;
    unsigned v[16];
    unsigned long long s = 0;
    for (int k = 0; k < 16; k++) {
        v[k] = b0 + k < N ? x[b0 + k] : 0u;
        s += v[k];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = bsum[blockIdx.x];
        for (int i = 0; i < 256; i++) {
            const unsigned long long t = part[i];
            part[i] = run;
            run += t;
        }
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];
    for (int k = 0; k < 16; k++) {
        if (b0 + k < N) coff[b0 + k] = (unsigned)(run > 0xffffffffull ? 0xffffffffull : run);
        run += v[k];
    }
}

// Host driver: out[0..N) = exclusive prefix sums of x, out[N] = the total (also
// written to *total); bsum holds scan_blocks(N) + 1 words.
inline int scan_blocks(int64_t N) { return (int)((N + kScanItems - 1) / kScanItems); }

inline void scan_counts(const unsigned* x, int64_t N, unsigned long long* bsum, unsigned* out,
                        unsigned long long* total, cudaStream_t s) {
    const int nb = scan_blocks(N);
    if (nb > 0) k_scan_reduce<<<nb, 256, 0, s>>>(x, N, bsum);
    k_scan_top<<<1, 1024, 0, s>>>(bsum, nb, N, out, total);
    if (nb > 0) k_scan_apply<<<nb, 256, 0, s>>>(x, N, bsum, out);
}

}  // namespace
}  // namespace pmf
