// Status helpers of the C ABI.

#include "internal.cuh"

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
        default: return "unknown status";
    }
}
