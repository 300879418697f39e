// Loss and optimiser of the training step: entry points (kernels in train.cuh).

#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "train.cuh"

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

extern "C" int gsparc_adam_segments(int64_t n, float* param, const float* grad, float* m, float* v, int32_t n_seg,
                                    const int64_t* seg_end, const float* seg_lr, float b1, float b2, float eps,
                                    int32_t step, void* stream) {
    if (n < 0 || step < 1 || n_seg < 1 || n_seg > kAdamMaxSeg || !seg_end || !seg_lr) return GSPARC_ERR_INVALID;
    AdamSegments seg{};
    seg.n_seg = n_seg;
    int64_t prev = 0;
    for (int s = 0; s < n_seg; ++s) {
        if (seg_end[s] < prev) return GSPARC_ERR_INVALID;
        seg.end[s] = seg_end[s];
        seg.lr[s] = seg_lr[s];
        prev = seg_end[s];
    }
    if (prev != n) return GSPARC_ERR_INVALID;
    if (n == 0) return GSPARC_OK;
    if (!param || !grad || !m || !v) return GSPARC_ERR_INVALID;
    const float bc1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float bc2 = (float)(1.0 - std::pow((double)b2, (double)step));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
    k_adam_seg<<<blocks, 256, 0, as_stream(stream)>>>(n, param, grad, m, v, seg, b1, b2, eps, bc1, bc2);
    return launch_status();
}

extern "C" int gsparc_scale_rows(int32_t rows, int64_t per, const float* w, float* x, void* stream) {
    if (rows < 0 || per < 0) return GSPARC_ERR_INVALID;
    if (rows == 0 || per == 0) return GSPARC_OK;
    if (!w || !x) return GSPARC_ERR_INVALID;
    const int64_t n = (int64_t)rows * per;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
    k_scale_rows<<<blocks, 256, 0, as_stream(stream)>>>(rows, per, w, x);
    return launch_status();
}
