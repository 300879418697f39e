// CSI head, channel loss and head backward: entry points (kernels in csi.cuh).

#include <algorithm>

#include "internal.cuh"
#include "csi.cuh"

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
