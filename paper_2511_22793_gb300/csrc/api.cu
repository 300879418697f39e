// Status helpers of the C ABI.

#include <atomic>

#include "internal.cuh"

namespace gsparc {
namespace {
std::atomic<uint32_t> g_wait_limit{0};
std::atomic<int32_t> g_overlap{GSPARC_OVERLAP_ALL};
}  // namespace

bool launch_overlap(int32_t group) { return (g_overlap.load(std::memory_order_relaxed) & group) != 0; }

uint32_t wait_limit(uint32_t dflt) {
    const uint32_t v = g_wait_limit.load(std::memory_order_relaxed);
    return v ? v : dflt;
}
}  // namespace gsparc

extern "C" uint32_t gsparc_set_wait_limit(uint32_t polls) {
    return gsparc::g_wait_limit.exchange(polls, std::memory_order_relaxed);
}

extern "C" int32_t gsparc_set_launch_overlap(int32_t groups) {
    return gsparc::g_overlap.exchange(groups & GSPARC_OVERLAP_ALL, std::memory_order_relaxed);
}

extern "C" int gsparc_check(const int32_t* d_status, void* stream) {
    cudaStream_t s = gsparc::as_stream(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return GSPARC_ERR_CUDA;
    if (!d_status) return GSPARC_OK;
    int32_t h = 0;
    if (cudaMemcpy(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return GSPARC_ERR_CUDA;
    return h;
}

extern "C" const char* gsparc_strerror(int status) {
    switch (status) {
        case GSPARC_OK: return "ok";
        case GSPARC_ERR_INVALID: return "invalid argument";
        case GSPARC_ERR_WORKSPACE: return "workspace too small";
        case GSPARC_ERR_CUDA: return "CUDA error";
        case GSPARC_ERR_TIMEOUT: return "bounded device wait expired";
        case GSPARC_ERR_CAPACITY: return "capacity exceeded (tile pairs or densified rows)";
        case GSPARC_ERR_TOO_LARGE: return "size above the fixed scratch limit";
        case GSPARC_ERR_INPUT: return "input out of domain (found on the device)";
        default: return "unknown status";
    }
}
