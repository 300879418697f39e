// CSI head (Sec. 4.2 "Rendered Spectrum", Eq. 2), channel loss (Eq. 3) and the gradient of
// the head.
//
//   h_hat[b,k] = scale * sum_p z[b,k,p]            (scale = 1/HW: the spatial mean, Eq. 2)
//   L = mean over (b,k) of |h_hat - h|^2,  dL/dh_hat = 2 (h_hat - h) / (B K)      (Eq. 3)
//   dL/dz[b,k,p] = scale * dL/dh_hat[b,k]          (every pixel of the plane)
//
// The head is a row reduction, HBM-bound (8 bytes per pixel and subcarrier): each block sums
// a contiguous chunk of one (b,k) plane with coalesced loads and adds it with one atomic
// pair, so the grid covers the SMs whatever the number of planes.  The order of the atomic
// additions is not fixed (results can differ in the last bits between runs).
//
// Device code only (the entry points are in csi.cu), so that the same source also builds for the
// host under the test suite's shim.

#pragma once

#include <math.h>
#include <stdint.h>

#include "device_common.cuh"

namespace gsparc {
namespace {

constexpr int kCsiThreads = 256;

__device__ __forceinline__ float2 block_sum2(float2 v, float2* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    float2 t = make_float2(0.f, 0.f);
    if (threadIdx.x == 0)
        for (int w = 0; w < kCsiThreads / 32; ++w) {
            t.x += s_warp[w].x;
            t.y += s_warp[w].y;
        }
    return t;   // meaningful in thread 0
}

__global__ void __launch_bounds__(kCsiThreads) k_csi_head(int64_t P, int64_t chunk, const float2* __restrict__ z,
                                                          float scale, float2* __restrict__ csi) {
    __shared__ float2 s_warp[kCsiThreads / 32];
    const int64_t row = blockIdx.y;
    const int64_t p0 = (int64_t)blockIdx.x * chunk;
    const int64_t p1 = p0 + chunk < P ? p0 + chunk : P;
    const float2* zr = z + row * P;
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kCsiThreads) {
        const float2 v = __ldcs(zr + p);
        acc.x += v.x;
        acc.y += v.y;
    }
    const float2 t = block_sum2(acc, s_warp);
    if (threadIdx.x == 0) {
        atomicAdd(&csi[row].x, t.x * scale);
        atomicAdd(&csi[row].y, t.y * scale);
    }
}

__global__ void __launch_bounds__(kCsiThreads) k_csi_loss(int m, const float2* __restrict__ csi,
                                                          const float2* __restrict__ target, float* __restrict__ loss,
                                                          float2* __restrict__ d_csi) {
    __shared__ float2 s_warp[kCsiThreads / 32];
    const float inv = 1.0f / (float)m;
    float2 acc = make_float2(0.f, 0.f);
    for (int e = threadIdx.x; e < m; e += kCsiThreads) {
        const float2 h = csi[e], t = target[e];
        const float dx = h.x - t.x, dy = h.y - t.y;
        acc.x += dx * dx + dy * dy;
        if (d_csi) d_csi[e] = make_float2(2.0f * dx * inv, 2.0f * dy * inv);
    }
    const float2 t = block_sum2(acc, s_warp);
    if (threadIdx.x == 0) loss[0] = t.x * inv;
}

__global__ void __launch_bounds__(kCsiThreads) k_csi_bcast(int64_t P, int64_t total, const float2* __restrict__ d_csi,
                                                           float scale, float2* __restrict__ d_z) {
    const int64_t stride = (int64_t)gridDim.x * kCsiThreads;
    for (int64_t e = (int64_t)blockIdx.x * kCsiThreads + threadIdx.x; e < total; e += stride) {
        const float2 g = d_csi[e / P];
        __stcs(d_z + e, make_float2(g.x * scale, g.y * scale));
    }
}

}  // namespace
}  // namespace gsparc
