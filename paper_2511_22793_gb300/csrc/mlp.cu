// Attribute network: launches and entry points of the FP32 kernels (mlp_fp32.cuh); the BF16
// tensor-core forms are in mlp_tc.cu and mlp_bwd_tc.cu.

#include <algorithm>

#include "internal.cuh"
#include "mlp_fp32.cuh"

namespace gsparc {

int attr_mlp_bf16(int32_t N, int32_t B, const float* tx, const float* rx, const float* means,
                  const float* opacity_logit, const float* latent, const gsparc_mlp* mlp,
                  int32_t precision, float* attr, cudaStream_t s);

namespace {

// Leading dimension of the stored activations: the rows rounded up to a multiple of 4 (16 bytes).
int64_t hidden_ld(int64_t rows) { return (rows + 3) / 4 * 4; }

bool mlp_ok(const gsparc_mlp* m) {
    if (!m) return false;
    if (!(m->hidden == 8 || m->hidden == 16 || m->hidden == 32 || m->hidden == 64)) return false;
    return m->W1 && m->b1 && m->W2 && m->b2 && m->W3 && m->b3;
}

template <int HD>
void launch_fwd(int N, int B, const float* tx, const float* rx, const float* means, const float* ologit,
                const float* latent, const W& w, float4* attr, float* hidden, cudaStream_t s) {
    const int64_t rows = (int64_t)N * B;
    const int blocks = (int)((rows + 127) / 128);
    if (hidden)
        k_mlp_fwd<HD, true><<<blocks, 128, 0, s>>>(N, B, tx, rx[0], rx[1], rx[2], means, ologit, latent, w, attr,
                                                   hidden, hidden_ld(rows));
    else
        k_mlp_fwd<HD, false><<<blocks, 128, 0, s>>>(N, B, tx, rx[0], rx[1], rx[2], means, ologit, latent, w,
                                                    attr, nullptr, 0);
}

template <int HD>
int launch_bwd(int N, int B, const float* tx, const float* rx, const float* means, const float* ologit,
               const float* latent, const W& w, const float4* d_attr, float* d_means, float* d_ologit,
               float* d_latent, const gsparc_mlp_grad& g, const float* hidden, cudaStream_t s) {
    const size_t smem = (size_t)BwdSmem<HD>::kTotal * sizeof(float);
    if (!ensure_smem_attr(k_mlp_bwd<HD>, (int)smem)) return GSPARC_ERR_CUDA;
    const int64_t rows = (int64_t)N * B;
    const int64_t tiles = (rows + kBwdRows - 1) / kBwdRows;
    const int blocks = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * (HD <= 32 ? 3 : 1));
    return launch_after(GSPARC_OVERLAP_NETWORK, k_mlp_bwd<HD>, dim3(blocks), dim3(kBwdThreads), smem, s, N, B, tx, rx[0], rx[1], rx[2], means,
                        ologit, latent, w, d_attr, d_means, d_ologit, d_latent, g, hidden, hidden_ld(rows));
}

}  // namespace
}  // namespace gsparc

using namespace gsparc;

extern "C" int gsparc_attr_mlp(int32_t N, int32_t B, const float* tx, const float* rx, const float* means,
                               const float* opacity_logit, const float* latent, const gsparc_mlp* mlp,
                               int32_t precision, float* attr, float* hidden, void* stream) {
    if (N < 0 || B <= 0 || !mlp_ok(mlp) || !rx) return GSPARC_ERR_INVALID;
    if (hidden && (precision != GSPARC_FP32 || (reinterpret_cast<uintptr_t>(hidden) & 15)))
        return GSPARC_ERR_INVALID;
    if ((int64_t)N * B >= (1ll << 31)) return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    if (!tx || !means || !opacity_logit || !latent || !attr) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(latent) | reinterpret_cast<uintptr_t>(attr)) & 15)
        return GSPARC_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    if (precision == GSPARC_BF16 || precision == GSPARC_BF16X2)
        return attr_mlp_bf16(N, B, tx, rx, means, opacity_logit, latent, mlp, precision, attr, s);
    if (precision != GSPARC_FP32) return GSPARC_ERR_INVALID;
    W w{mlp->W1, mlp->b1, mlp->W2, mlp->b2, mlp->W3, mlp->b3};
    float4* a4 = reinterpret_cast<float4*>(attr);
    switch (mlp->hidden) {
        case 8: launch_fwd<8>(N, B, tx, rx, means, opacity_logit, latent, w, a4, hidden, s); break;
        case 16: launch_fwd<16>(N, B, tx, rx, means, opacity_logit, latent, w, a4, hidden, s); break;
        case 32: launch_fwd<32>(N, B, tx, rx, means, opacity_logit, latent, w, a4, hidden, s); break;
        default: launch_fwd<64>(N, B, tx, rx, means, opacity_logit, latent, w, a4, hidden, s); break;
    }
    return launch_status();
}

extern "C" int gsparc_attr_mlp_bwd(int32_t N, int32_t B, const float* tx, const float* rx,
                                   const float* means, const float* opacity_logit, const float* latent,
                                   const gsparc_mlp* mlp, const float* d_attr, float* d_means,
                                   float* d_opacity_logit, float* d_latent, const gsparc_mlp_grad* grads,
                                   const float* hidden, void* stream) {
    if (N < 0 || B <= 0 || !mlp_ok(mlp) || !rx || !grads) return GSPARC_ERR_INVALID;
    if ((int64_t)N * B >= (1ll << 31)) return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    if (!tx || !means || !opacity_logit || !latent || !d_attr || !d_means || !d_opacity_logit ||
        !d_latent)
        return GSPARC_ERR_INVALID;
    if (!grads->W1 || !grads->b1 || !grads->W2 || !grads->b2 || !grads->W3 || !grads->b3)
        return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(latent) | reinterpret_cast<uintptr_t>(d_attr) |
         reinterpret_cast<uintptr_t>(hidden)) & 15)
        return GSPARC_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    W w{mlp->W1, mlp->b1, mlp->W2, mlp->b2, mlp->W3, mlp->b3};
    const float4* da = reinterpret_cast<const float4*>(d_attr);
    int rc;
    switch (mlp->hidden) {
        case 8: rc = launch_bwd<8>(N, B, tx, rx, means, opacity_logit, latent, w, da, d_means, d_opacity_logit, d_latent, *grads, hidden, s); break;
        case 16: rc = launch_bwd<16>(N, B, tx, rx, means, opacity_logit, latent, w, da, d_means, d_opacity_logit, d_latent, *grads, hidden, s); break;
        case 32: rc = launch_bwd<32>(N, B, tx, rx, means, opacity_logit, latent, w, da, d_means, d_opacity_logit, d_latent, *grads, hidden, s); break;
        default: rc = launch_bwd<64>(N, B, tx, rx, means, opacity_logit, latent, w, da, d_means, d_opacity_logit, d_latent, *grads, hidden, s); break;
    }
    if (rc != GSPARC_OK) return rc;
    return launch_status();
}
