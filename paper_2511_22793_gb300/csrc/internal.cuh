// Shared definitions of the CUDA library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "gsparc.h"

namespace gsparc {

// Footprint cut-off q_max = 2 ln 255: the kernel exp(-q/2) falls to 1/255.
constexpr float kQMax = 11.082527090f;         // 2 * ln(255)
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kLog2TMin = -13.287712f;      // log2(1e-4)
constexpr float kDilation = 0.3f;             // px^2 added to diag(Sigma')
constexpr float kRhoFloor = 1e-3f;            // zenith floor on rho, relative to r
constexpr float kDMin = 0.01f;                // metres, floor on the transmitter distance
constexpr double kCLight = 299792458.0;       // m/s
constexpr float kPi = 3.14159265358979f;
constexpr int kTile = GSPARC_TILE;

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GSPARC_OK : GSPARC_ERR_CUDA;
}

inline int tiles_x(const gsparc_view& v) { return (v.W + kTile - 1) / kTile; }
inline int tiles_y(const gsparc_view& v) { return (v.H + kTile - 1) / kTile; }

inline bool view_ok(const gsparc_view* v) {
    return v && v->H > 0 && v->W > 0 && v->H <= 32768 && v->W <= 32768;
}

inline int num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (kernel, device): the attribute
// persists, and skipping the repeat keeps launches cheap and capture-friendly.
// Keyed by the kernel's address (kernels of one signature share a type).
template <typename Kernel>
inline bool ensure_smem_attr(Kernel k, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;   // (kernel, device) -> bytes set
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const auto key = std::make_pair(reinterpret_cast<const void*>(k), dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return true;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return false;
    done[key] = bytes;
    return true;
}

// Device-side view constants passed by value to kernels.
struct ViewDev {
    int H, W;
    float rx0, rx1, rx2;
    float V[9];
    float near_dist;
};

inline ViewDev to_dev(const gsparc_view& v) {
    ViewDev d;
    d.H = v.H;
    d.W = v.W;
    d.rx0 = v.rx[0];
    d.rx1 = v.rx[1];
    d.rx2 = v.rx[2];
    for (int i = 0; i < 9; ++i) d.V[i] = v.V[i];
    d.near_dist = v.near_dist;
    return d;
}

}  // namespace gsparc
