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

#include <algorithm>

#include "internal.cuh"

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

using namespace gsparc;

extern "C" int gsparc_csi_head(int32_t B, int32_t K, int64_t P, const float* spectrum, float scale, float* csi,
                               void* stream) {
    if (B <= 0 || K <= 0 || P < 0 || !csi) return GSPARC_ERR_INVALID;
    if ((int64_t)B * K >= 65536) return GSPARC_ERR_INVALID;   // one grid row per plane
    if (P > 0 && !spectrum) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(spectrum) | reinterpret_cast<uintptr_t>(csi)) & 7) return GSPARC_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    const int rows = B * K;
    if (cudaMemsetAsync(csi, 0, (size_t)rows * 2 * sizeof(float), s) != cudaSuccess) return GSPARC_ERR_CUDA;
    if (P == 0) return GSPARC_OK;
    // about four blocks per SM in total, each chunk a multiple of the block size
    const int64_t want = std::max<int64_t>(1, ((int64_t)num_sms() * 4 + rows - 1) / rows);
    int64_t chunk = (P + want - 1) / want;
    chunk = (chunk + kCsiThreads - 1) / kCsiThreads * kCsiThreads;
    const int64_t nchunk = (P + chunk - 1) / chunk;
    dim3 grid((unsigned)nchunk, (unsigned)rows);
    k_csi_head<<<grid, kCsiThreads, 0, s>>>(P, chunk, reinterpret_cast<const float2*>(spectrum), scale,
                                            reinterpret_cast<float2*>(csi));
    return launch_status();
}

extern "C" int gsparc_csi_loss(int32_t B, int32_t K, const float* csi, const float* target, float* loss,
                               float* d_csi, void* stream) {
    if (B <= 0 || K <= 0 || !csi || !target || !loss) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(csi) | reinterpret_cast<uintptr_t>(target) |
         reinterpret_cast<uintptr_t>(d_csi)) & 7)
        return GSPARC_ERR_INVALID;
    const int64_t m = (int64_t)B * K;
    if (m >= (1ll << 31)) return GSPARC_ERR_INVALID;
    k_csi_loss<<<1, kCsiThreads, 0, as_stream(stream)>>>((int)m, reinterpret_cast<const float2*>(csi),
                                                         reinterpret_cast<const float2*>(target), loss,
                                                         reinterpret_cast<float2*>(d_csi));
    return launch_status();
}

extern "C" int gsparc_csi_head_bwd(int32_t B, int32_t K, int64_t P, const float* d_csi, float scale,
                                   float* d_spectrum, void* stream) {
    if (B <= 0 || K <= 0 || P < 0 || !d_csi) return GSPARC_ERR_INVALID;
    if (P > 0 && !d_spectrum) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_csi) | reinterpret_cast<uintptr_t>(d_spectrum)) & 7) return GSPARC_ERR_INVALID;
    const int64_t total = (int64_t)B * K * P;
    if (total == 0) return GSPARC_OK;
    const int64_t blocks = std::min<int64_t>((total + kCsiThreads - 1) / kCsiThreads, (int64_t)num_sms() * 8);
    k_csi_bcast<<<(unsigned)blocks, kCsiThreads, 0, as_stream(stream)>>>(
        P, total, reinterpret_cast<const float2*>(d_csi), scale, reinterpret_cast<float2*>(d_spectrum));
    return launch_status();
}
