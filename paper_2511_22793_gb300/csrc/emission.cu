// Per-Gaussian emission network: launches and entry points (kernels in emission.cuh).

#include <algorithm>

#include "internal.cuh"
#include "emission.cuh"

namespace gsparc {
namespace {

template <template <int> class K, typename... Args>
void em_launch(int G, int N, cudaStream_t s, Args... args) {
    const int64_t threads = (int64_t)N * G;
    const unsigned blocks = (unsigned)((threads + kEmThreads - 1) / kEmThreads);
    switch (G) {
        case 1: K<1>::launch(blocks, s, args...); break;
        case 2: K<2>::launch(blocks, s, args...); break;
        case 4: K<4>::launch(blocks, s, args...); break;
        case 8: K<8>::launch(blocks, s, args...); break;
        case 16: K<16>::launch(blocks, s, args...); break;
        default: K<32>::launch(blocks, s, args...); break;
    }
}

template <int G>
struct FwdLaunch {
    template <typename... Args>
    static void launch(unsigned blocks, cudaStream_t s, Args... args) {
        k_emission_fwd<G><<<blocks, kEmThreads, 0, s>>>(args...);
    }
};

template <int G>
struct BwdLaunch {
    template <typename... Args>
    static void launch(unsigned blocks, cudaStream_t s, Args... args) {
        k_emission_bwd<G><<<blocks, kEmThreads, 0, s>>>(args...);
    }
};

bool em_args_ok(int32_t N, int32_t B, int32_t hidden, const float* tx, const float* rx, const float* means,
                const float* ologit, const float* weights) {
    if (N < 0 || B <= 0 || B > 65535 || hidden < 1 || hidden > kEmMaxHidden || !rx) return false;
    if ((int64_t)N * B >= (1ll << 31)) return false;
    if ((int64_t)N * 32 >= (1ll << 31)) return false;   // thread index N * G in 32 bits
    if (N > 0 && (!tx || !means || !ologit || !weights)) return false;
    if (reinterpret_cast<uintptr_t>(weights) & 15) return false;
    return true;
}

}  // namespace
}  // namespace gsparc

using namespace gsparc;

extern "C" int32_t gsparc_emission_stride(int32_t hidden) {
    if (hidden < 1 || hidden > kEmMaxHidden) return 0;
    return em_stride(hidden);
}

extern "C" int gsparc_emission_fwd(int32_t N, int32_t B, int32_t hidden, const float* tx, const float* rx,
                                   const float* means, const float* opacity_logit, const float* weights,
                                   int32_t inv_d, float* attr, void* stream) {
    if (!em_args_ok(N, B, hidden, tx, rx, means, opacity_logit, weights) || (N > 0 && !attr))
        return GSPARC_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(attr) & 15) return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    em_launch<FwdLaunch>(em_group(hidden), N, as_stream(stream), N, B, (int)hidden, em_stride(hidden), tx, rx[0],
                         rx[1], rx[2], means, opacity_logit, weights, inv_d ? 1 : 0,
                         reinterpret_cast<float4*>(attr));
    return launch_status();
}

extern "C" int gsparc_emission_bwd(int32_t N, int32_t B, int32_t hidden, const float* tx, const float* rx,
                                   const float* means, const float* opacity_logit, const float* weights,
                                   int32_t inv_d, const float* d_attr, float* d_means, float* d_opacity_logit,
                                   float* d_weights, void* stream) {
    if (!em_args_ok(N, B, hidden, tx, rx, means, opacity_logit, weights)) return GSPARC_ERR_INVALID;
    if (N > 0 && (!d_attr || !d_means || !d_opacity_logit || !d_weights)) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_attr) | reinterpret_cast<uintptr_t>(d_weights)) & 15)
        return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    em_launch<BwdLaunch>(em_group(hidden), N, as_stream(stream), N, B, (int)hidden, em_stride(hidden), tx, rx[0],
                         rx[1], rx[2], means, opacity_logit, weights, inv_d ? 1 : 0,
                         reinterpret_cast<const float4*>(d_attr), d_means, d_opacity_logit, d_weights);
    return launch_status();
}
