// Magnitude-spectrum loss (Eq. 4): entry points (kernels and workspace layout in ssim.cuh).

#include <algorithm>

#include "internal.cuh"
#include "ssim.cuh"

using namespace gsparc;

extern "C" int gsparc_spectrum_loss_workspace(int32_t B, int32_t K, int32_t H, int32_t W, size_t* ws_bytes) {
    if (B <= 0 || K <= 0 || H <= 0 || W <= 0 || !ws_bytes) return GSPARC_ERR_INVALID;
    *ws_bytes = ss_layout((int64_t)B * K * H * W).total;
    return GSPARC_OK;
}

extern "C" int gsparc_spectrum_loss(int32_t B, int32_t K, int32_t H, int32_t W, const float* spectrum,
                                    const float* target, float lambda, void* ws, size_t ws_bytes, float* loss,
                                    float* d_spectrum, void* stream) {
    if (B <= 0 || K <= 0 || H <= 0 || W <= 0 || !spectrum || !target || !ws || !loss) return GSPARC_ERR_INVALID;
    if (!(lambda >= 0.f && lambda <= 1.f)) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(spectrum) | reinterpret_cast<uintptr_t>(d_spectrum)) & 7)
        return GSPARC_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return GSPARC_ERR_INVALID;
    const int64_t n = (int64_t)B * K * H * W;
    if ((int64_t)H * W >= (1ll << 31)) return GSPARC_ERR_INVALID;
    const SsLayout SL = ss_layout(n);
    if (ws_bytes < SL.total) return GSPARC_ERR_INVALID;
    const Window win = ss_window();
    char* w = static_cast<char*>(ws);
    double* acc = reinterpret_cast<double*>(w + SL.acc);
    float* t5 = reinterpret_cast<float*>(w + SL.t5);
    float* abc = reinterpret_cast<float*>(w + SL.abc);
    float* t3 = reinterpret_cast<float*>(w + SL.t3);
    const float2* z = reinterpret_cast<const float2*>(spectrum);
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(acc, 0, 2 * sizeof(double), s) != cudaSuccess) return GSPARC_ERR_CUDA;
    const unsigned blocks = (unsigned)((n + kSsThreads - 1) / kSsThreads);
    k_ssim_h<<<blocks, kSsThreads, 0, s>>>(n, H, W, win, z, target, t5);
    k_ssim_v<<<blocks, kSsThreads, 0, s>>>(n, H, W, win, z, target, t5, abc, acc);
    k_ssim_finish<<<1, 1, 0, s>>>(acc, (double)n, (double)lambda, loss);
    if (d_spectrum) {
        k_ssim_bh<<<blocks, kSsThreads, 0, s>>>(n, W, win, abc, t3);
        k_ssim_bv<<<blocks, kSsThreads, 0, s>>>(n, H, W, win, z, target, t3, (float)((1.0 - lambda) / (double)n),
                                                (float)(-(double)lambda / (double)n),
                                                reinterpret_cast<float2*>(d_spectrum));
    }
    return launch_status();
}
