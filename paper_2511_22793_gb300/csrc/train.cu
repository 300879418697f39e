// Loss and optimiser kernels of the training step (Algorithm 1: loss,
// Backprop seed and Adam).  Both are HBM-bound elementwise passes.

#include <algorithm>
#include <cmath>

#include "internal.cuh"

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

}  // namespace
}  // namespace gsparc

using namespace gsparc;

extern "C" int gsparc_l2_loss(int64_t count, const float* z, const float* target, float* loss, float* d_z,
                              void* stream) {
    if (count < 0 || !loss) return GSPARC_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return GSPARC_ERR_CUDA;
    if (count == 0) return GSPARC_OK;
    if (!z || !target) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(target) |
         reinterpret_cast<uintptr_t>(d_z)) & 7)
        return GSPARC_ERR_INVALID;
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)num_sms() * 8);
    k_l2_loss<<<blocks, 256, 0, s>>>(count, reinterpret_cast<const float2*>(z),
                                     reinterpret_cast<const float2*>(target), (float)(1.0 / (double)count),
                                     loss, reinterpret_cast<float2*>(d_z));
    return launch_status();
}

extern "C" int gsparc_adam(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float b1,
                           float b2, float eps, int32_t step, void* stream) {
    if (n < 0 || step < 1) return GSPARC_ERR_INVALID;
    if (n == 0) return GSPARC_OK;
    if (!param || !grad || !m || !v) return GSPARC_ERR_INVALID;
    const float bc1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float bc2 = (float)(1.0 - std::pow((double)b2, (double)step));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
    k_adam<<<blocks, 256, 0, as_stream(stream)>>>(n, param, grad, m, v, lr, b1, b2, eps, bc1, bc2);
    return launch_status();
}
