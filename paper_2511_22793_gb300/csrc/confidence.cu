// Confidence-weighted objective (Eq. 5, Sec. 4.2): the C-ABI entry point of the kernel in
// confidence.cuh.
#include "confidence.cuh"
#include "internal.cuh"

using namespace gsparc;

extern "C" int gsparc_confidence(int32_t B, int32_t hidden, const float* pos, const float* task_loss,
                                 const float* weights, float alpha, float* confidence, float* objective,
                                 float* d_task_loss, float* d_weights, void* stream) {
    if (B < 0 || hidden < 1 || hidden > kConfMaxHidden || !weights || !objective) return GSPARC_ERR_INVALID;
    if (B > 0 && (!pos || !task_loss)) return GSPARC_ERR_INVALID;
    if ((int64_t)B * 3 >= (1ll << 31)) return GSPARC_ERR_INVALID;
    if (!(alpha >= 0.0f)) return GSPARC_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    if (B == 0) {
        // the mean over no samples is taken as 0; nothing else is written
        return cudaMemsetAsync(objective, 0, sizeof(float), s) == cudaSuccess ? GSPARC_OK : GSPARC_ERR_CUDA;
    }
    k_confidence<<<1, kConfWarps * 32, 0, s>>>(B, hidden, pos, task_loss, weights, alpha,
                                               (float)(1.0 / (double)B), confidence, objective,
                                               d_task_loss, d_weights);
    return launch_status();
}
