// Adaptive density control (Algorithm 1, densification branch): the C-ABI entry points of the
// kernels in densify.cuh.
#include <math.h>

#include "densify.cuh"
#include "internal.cuh"

using namespace gsparc;

namespace {

size_t dens_ws_bytes(int N) { return ((size_t)dens_blocks(N) * sizeof(uint32_t) + 255) & ~size_t(255); }

int grid_for(int N) {
    const int want = dens_blocks(N);
    const int cap = num_sms() * 8;
    return want < cap ? (want > 0 ? want : 1) : cap;
}

}  // namespace

extern "C" int gsparc_densify_accumulate(int32_t N, const float* proj, const float* d_means, float* norm_sum,
                                         uint32_t* count, void* stream) {
    if (N < 0) return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    if (!proj || !d_means || !norm_sum || !count || (int64_t)N * 8 >= (1ll << 31)) return GSPARC_ERR_INVALID;
    k_dens_accumulate<<<grid_for(N), kDensThreads, 0, as_stream(stream)>>>(N, proj, d_means, norm_sum, count);
    return launch_status();
}

extern "C" int gsparc_densify_workspace(int32_t N, size_t* ws_bytes) {
    if (N < 0 || !ws_bytes || (int64_t)N * 8 >= (1ll << 31)) return GSPARC_ERR_INVALID;
    *ws_bytes = dens_ws_bytes(N);
    return GSPARC_OK;
}

extern "C" int gsparc_densify(int32_t N, int32_t P, const float* means, const float* log_scales, const float* quats,
                              const float* opacity_logit, const float* payload, const float* proj,
                              const float* norm_sum, const uint32_t* count, const float* xi,
                              const gsparc_densify_params* params, int32_t capacity, void* ws, size_t ws_bytes,
                              float* out_means, float* out_log_scales, float* out_quats, float* out_opacity_logit,
                              float* out_payload, uint32_t* out_parent, uint32_t* n_out, int32_t* d_status,
                              void* stream) {
    if (N < 0 || P < 0 || capacity < 0 || !params || !n_out) return GSPARC_ERR_INVALID;
    const gsparc_densify_params& q = *params;
    if (q.n_split < 1 || q.n_split > kDensMaxSplit) return GSPARC_ERR_INVALID;
    if (!(q.tau_grad >= 0.0f) || !(q.clone_scale >= 0.0f) || !(q.sigma_min >= 0.0f) || !(q.r_max >= 0.0f))
        return GSPARC_ERR_INVALID;
    if ((int64_t)N * 8 >= (1ll << 31) || (int64_t)capacity * (P > 4 ? P : 4) >= (1ll << 40))
        return GSPARC_ERR_INVALID;
    if (N > 0 && (!means || !log_scales || !quats || !opacity_logit || !proj || !norm_sum || !count || !xi ||
                  (P > 0 && !payload)))
        return GSPARC_ERR_INVALID;
    if (capacity > 0 && (!out_means || !out_log_scales || !out_quats || !out_opacity_logit || !out_parent ||
                         (P > 0 && !out_payload)))
        return GSPARC_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    if (N == 0) return cudaMemsetAsync(n_out, 0, sizeof(uint32_t), s) == cudaSuccess ? GSPARC_OK : GSPARC_ERR_CUDA;
    if (!ws || ws_bytes < dens_ws_bytes(N)) return GSPARC_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 3) return GSPARC_ERR_INVALID;

    DensParams p;
    p.tau_grad = q.tau_grad;
    p.clone_scale = q.clone_scale;
    p.sigma_min = q.sigma_min;
    p.r_max = q.r_max;
    p.log_shrink = (float)log(0.8 * (double)q.n_split);
    p.n_split = q.n_split;
    uint32_t* block_rows = static_cast<uint32_t*>(ws);
    const int nb = dens_blocks(N);
    k_dens_count<<<nb, kDensThreads, 0, s>>>(N, p, log_scales, opacity_logit, proj, norm_sum, count, block_rows);
    k_dens_scan<<<1, kDensScanThreads, 0, s>>>(nb, (uint32_t)capacity, block_rows, n_out, d_status);
    DensOut o{out_means, out_log_scales, out_quats, out_opacity_logit, out_payload, out_parent};
    k_dens_scatter<<<nb, kDensThreads, 0, s>>>(N, P, p, means, log_scales, quats, opacity_logit, payload, proj,
                                               norm_sum, count, xi, block_rows, (uint32_t)capacity, o);
    return launch_status();
}

extern "C" int gsparc_opacity_reset(int32_t N, float max_opacity, float* opacity_logit, void* stream) {
    if (N < 0 || !(max_opacity > 0.0f && max_opacity < 1.0f)) return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    if (!opacity_logit) return GSPARC_ERR_INVALID;
    const float cap = (float)log((double)max_opacity / (1.0 - (double)max_opacity));
    k_opacity_reset<<<grid_for(N), kDensThreads, 0, as_stream(stream)>>>(N, cap, opacity_logit);
    return launch_status();
}
