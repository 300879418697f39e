// Loss and optimiser kernels of the training step (Algorithm 1: loss,
// Backprop seed and Adam).  Both are HBM-bound elementwise passes.
//
// Device code only (the entry points are in train.cu), so that the same source also builds for the
// host under the test suite's shim.

#pragma once

#include <math.h>
#include <stdint.h>

#include "device_common.cuh"

namespace gsparc {
namespace {

__global__ void __launch_bounds__(256) k_l2_loss(int64_t count, const float2* __restrict__ z,
                                                 const float2* __restrict__ target, float inv_count,
                                                 float* __restrict__ loss, float2* __restrict__ d_z) {
    __shared__ float s_part[8];
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride) {
        const float2 a = z[j], b = target[j];
        const float dr = a.x - b.x, di = a.y - b.y;
        acc = fmaf(dr, dr, fmaf(di, di, acc));
        if (d_z) d_z[j] = make_float2(2.f * dr * inv_count, 2.f * di * inv_count);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += s_part[w];
        atomicAdd(loss, t * inv_count);
    }
}

__global__ void __launch_bounds__(256) k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v, float lr,
                                              float b1, float b2, float eps, float bc1, float bc2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const float gj = g[j];
        const float mj = b1 * m[j] + (1.f - b1) * gj;
        const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
        m[j] = mj;
        v[j] = vj;
        p[j] -= lr * (mj / bc1) / (sqrtf(vj / bc2) + eps);
    }
}

// x[r * per + j] *= w[r]: each sample's block of a batched array scaled by its weight.
__global__ void __launch_bounds__(256) k_scale_rows(int rows, int64_t per, const float* __restrict__ w,
                                                    float* __restrict__ x) {
    const int64_t n = (int64_t)rows * per;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) x[j] *= w[j / per];
}

// Parameter groups of one flat buffer for k_adam_seg: segment s covers [end[s-1], end[s])
// (end[-1] = 0) and takes learning rate lr[s].
constexpr int kAdamMaxSeg = 32;
struct AdamSegments {
    int n_seg;
    int64_t end[kAdamMaxSeg];
    float lr[kAdamMaxSeg];
};

// The same update as k_adam over every group of a flat buffer in one launch: the element's
// group is found by a binary search over the (kernel-parameter) segment ends.
__global__ void __launch_bounds__(256) k_adam_seg(int64_t n, float* __restrict__ p, const float* __restrict__ g,
                                                  float* __restrict__ m, float* __restrict__ v, AdamSegments seg,
                                                  float b1, float b2, float eps, float bc1, float bc2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        int lo = 0, hi = seg.n_seg - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (j < seg.end[mid]) hi = mid;
            else lo = mid + 1;
        }
        const float lr = seg.lr[lo];
        const float gj = g[j];
        const float mj = b1 * m[j] + (1.f - b1) * gj;
        const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
        m[j] = mj;
        v[j] = vj;
        p[j] -= lr * (mj / bc1) / (sqrtf(vj / bc2) + eps);
    }
}

}  // namespace
}  // namespace gsparc
