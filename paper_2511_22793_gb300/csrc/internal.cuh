// Shared definitions of the CUDA library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "device_common.cuh"
#include "gsparc.h"

namespace gsparc {

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GSPARC_OK : GSPARC_ERR_CUDA;
}


// Whether launch_after launches the kernels of `group` (GSPARC_OVERLAP_*) with programmatic stream
// serialization (gsparc_set_launch_overlap; every group unless switched off).
bool launch_overlap(int32_t group);

// Launches k<<<grid, block, smem, s>>>(args...) as a programmatic dependent of the kernel before it
// on the stream (programmatic stream serialization), for kernels that call grid_dep_wait() in every
// block before they touch what earlier kernels wrote or read: the launch is processed while the
// previous kernel drains, not after it.  Without launch_overlap(group) an ordinary launch.
template <typename... P, typename... A>
inline int launch_after(int32_t group, void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                        A&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = launch_overlap(group) ? 1 : 0;
    if (cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...) != cudaSuccess) {
        (void)cudaGetLastError();
        return GSPARC_ERR_CUDA;
    }
    return launch_status();
}

// Polls before a pipeline wait of the tensor-core compositing kernels gives up: the value set by
// gsparc_set_wait_limit, or dflt when none is set.
uint32_t wait_limit(uint32_t dflt);

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
