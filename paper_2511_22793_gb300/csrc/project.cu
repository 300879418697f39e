// Entry points of the per-Gaussian projection (kernels in project.cuh).

#include "internal.cuh"
#include "project.cuh"

using namespace gsparc;

extern "C" int32_t gsparc_num_tiles(const gsparc_view* view) {
    if (!view_ok(view)) return 0;
    return tiles_x(*view) * tiles_y(*view);
}

extern "C" int gsparc_project(const gsparc_view* view, int32_t N, const float* means,
                              const float* log_scales, const float* quats, float* proj, int32_t* d_status,
                              void* stream) {
    if (!view_ok(view) || N < 0) return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    if (!means || !log_scales || !quats || !proj) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(quats) | reinterpret_cast<uintptr_t>(proj)) & 15)
        return GSPARC_ERR_INVALID;
    const int threads = 256;
    const int blocks = (N + threads - 1) / threads;
    k_project<<<blocks, threads, 0, as_stream(stream)>>>(to_dev(*view), N, means, log_scales,
                                                         reinterpret_cast<const float4*>(quats),
                                                         reinterpret_cast<float4*>(proj), d_status);
    return launch_status();
}

extern "C" int gsparc_project_bwd(const gsparc_view* view, int32_t N, const float* means,
                                  const float* log_scales, const float* quats, const float* d_proj,
                                  float* d_means, float* d_log_scales, float* d_quats, void* stream) {
    if (!view_ok(view) || N < 0) return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    if (!means || !log_scales || !quats || !d_proj || !d_means || !d_log_scales || !d_quats)
        return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(quats) | reinterpret_cast<uintptr_t>(d_proj)) & 15)
        return GSPARC_ERR_INVALID;
    const int threads = 256;
    const int blocks = (N + threads - 1) / threads;
    k_project_bwd<<<blocks, threads, 0, as_stream(stream)>>>(
        to_dev(*view), N, means, log_scales, reinterpret_cast<const float4*>(quats),
        reinterpret_cast<const float4*>(d_proj), d_means, d_log_scales, d_quats);
    return launch_status();
}
