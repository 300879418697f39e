// Throughput probes of the two pipes that bound the FP32 compositing kernels: FP32 FMA and the
// SFU's ex2.  Measurement infrastructure of the benchmark (libgsparc_probe.so), not part of the
// splatting library's ABI.
//
// Each thread runs kChains independent dependency chains for `iters` iterations, so that the
// pipe, not the latency of one chain, sets the rate; the grid is blocks_per_sm x SMs blocks of
// 256 threads.  The result of every chain is folded into one store per thread so that no
// operation is dead code.

#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma(int iters, float a, float b, float* out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- ex2(-x) keeps every chain in (0.5, 1]; the negation folds into the instruction's operand
__global__ void __launch_bounds__(256) k_ex2(int iters, float* out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.1f * (float)(c + 1);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = ex2a(-x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// kind 0: FMA (returns the FMAs issued), 1: ex2 (returns the ex2 issued).  out must hold
// blocks * 256 floats.  Launches once on `stream` and returns the operation count, or -1 when
// the launch failed.  The caller times it (CUDA events around the call).
extern "C" int64_t gsparc_probe_launch(int kind, int blocks, int iters, float* out, void* stream) {
    if (blocks <= 0 || iters <= 0 || !out) return -1;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (kind == 0)
        k_fma<<<blocks, 256, 0, s>>>(iters, 0.9999f, 1e-4f, out);
    else if (kind == 1)
        k_ex2<<<blocks, 256, 0, s>>>(iters, out);
    else
        return -1;
    if (cudaGetLastError() != cudaSuccess) return -1;
    return (int64_t)blocks * 256 * iters * 4 * kChains;
}

// The paired FP32 operations the FP32 compositing kernels use (the runtime's __ffma2_rn and
// __fadd2_rn) against scalar fmaf and + on the same operands: out_pair[i] = __ffma2_rn(a, b, c) and
// out_scalar[i] = fmaf per element; with add != 0, __fadd2_rn(a, b) against a + b instead.  The two
// must agree bit for bit.
namespace {
__global__ void k_fma2_check(int n, int add, const float2* a, const float2* b, const float2* c, float2* out_pair,
                             float2* out_scalar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 x = a[i], y = b[i], z = c[i];
    if (add) {
        out_pair[i] = __fadd2_rn(x, y);
        out_scalar[i] = make_float2(__fadd_rn(x.x, y.x), __fadd_rn(x.y, y.y));
    } else {
        out_pair[i] = __ffma2_rn(x, y, z);
        out_scalar[i] = make_float2(fmaf(x.x, y.x, z.x), fmaf(x.y, y.y, z.y));
    }
}
}  // namespace

extern "C" int gsparc_probe_fma2_check(int n, int add, const float* a, const float* b, const float* c,
                                       float* out_pair, float* out_scalar, void* stream) {
    if (n < 0 || (n > 0 && (!a || !b || !c || !out_pair || !out_scalar))) return -1;
    if (n == 0) return 0;
    k_fma2_check<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        n, add, reinterpret_cast<const float2*>(a), reinterpret_cast<const float2*>(b), reinterpret_cast<const float2*>(c),
        reinterpret_cast<float2*>(out_pair), reinterpret_cast<float2*>(out_scalar));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
