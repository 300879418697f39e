// Test-only host shim that runs a CUDA kernel's source on CPU threads, one std::thread per
// CUDA thread, blocks one after another.  It exists to check the logic of the library's plain
// (non-tensor-core) kernels on a machine without a GPU: index arithmetic, warp shuffles,
// block barriers and the order of sums.  It is not a CUDA implementation: no memory model
// beyond sequential consistency, no timing, and nothing of the library links against it.
//
// Semantics kept from CUDA: __syncthreads() waits for every thread of the block that has not
// exited (exited threads leave the barrier's count); __shfl_*_sync exchange values among the
// 32 lanes of a warp and record a violation when a lane of the warp has already exited;
// atomics are atomic.  `__shared__` variables are function statics, valid because one block
// runs at a time.
#pragma once

#define GSPARC_HOST_SHIM 1

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <barrier>
#include <memory>
#include <thread>
#include <vector>

using std::max;   // CUDA's device min / max overloads
using std::min;

struct emu_dim3 {
    unsigned x = 1, y = 1, z = 1;
};

inline thread_local emu_dim3 threadIdx, blockIdx;

struct alignas(8) float2 {
    float x, y;
};
struct alignas(16) float4 {
    float x, y, z, w;
};
struct alignas(8) uint2 {
    unsigned x, y;
};
struct alignas(16) uint4 {
    unsigned x, y, z, w;
};
inline float2 make_float2(float x, float y) { return float2{x, y}; }
inline float4 make_float4(float x, float y, float z, float w) { return float4{x, y, z, w}; }
inline uint2 make_uint2(unsigned x, unsigned y) { return uint2{x, y}; }
inline uint4 make_uint4(unsigned x, unsigned y, unsigned z, unsigned w) { return uint4{x, y, z, w}; }
inline emu_dim3 blockDim, gridDim;

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __launch_bounds__(...)
#define __shared__ static
#define __align__(n) __attribute__((aligned(n)))

// dynamic shared memory: one buffer per launch, handed to every block in turn
inline unsigned char* g_emu_dyn_smem = nullptr;
#define GSPARC_DYNAMIC_SMEM(name) unsigned char* name = g_emu_dyn_smem

// single float operations in round-to-nearest (SSE arithmetic on x86-64 and AArch64 alike)
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fmaf_rn(float a, float b, float c) { return fmaf(a, b, c); }
inline void __sincosf(float x, float* s, float* c) { sincosf(x, s, c); }
inline float __int_as_float(int i) {
    float f;
    memcpy(&f, &i, 4);
    return f;
}
inline int __ffsll(long long x) { return __builtin_ffsll(x); }
inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
inline float __uint2float_rz(unsigned x) {
    float f = (float)x;
    if ((double)f > (double)x) f = nextafterf(f, 0.0f);
    return f;
}
inline int __float2int_rz(float f) { return (int)f; }
inline unsigned __float_as_uint(float f) {
    unsigned u;
    memcpy(&u, &f, 4);
    return u;
}
inline int __popc(unsigned x) { return __builtin_popcount(x); }
template <typename T>
inline T __ldcg(const T* p) {
    return *p;
}
template <typename T>
inline T __ldg(const T* p) {
    return *p;
}
template <typename T>
inline T __ldcs(const T* p) {
    return *p;
}
template <typename T>
inline void __stcs(T* p, T v) {
    *p = v;
}
inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }

struct EmuWarp {
    std::unique_ptr<std::barrier<>> bar;
    std::atomic<int> alive{0};
    uint64_t slot[32];
};

struct EmuBlockState {
    std::unique_ptr<std::barrier<>> bar;
    std::vector<std::unique_ptr<EmuWarp>> warps;
    std::atomic<int> vote[3] = {0, 0, 0};  // __syncthreads_or, see below
};

inline EmuBlockState* g_emu_block = nullptr;
inline std::atomic<int> g_emu_violations{0};

inline void __syncthreads() { g_emu_block->bar->arrive_and_wait(); }

// Call c of a block uses slot c % 3; between its two barriers every thread clears slot
// (c + 1) % 3, which nobody reads then and nobody sets before the second barrier.
inline thread_local int tl_vote_calls = 0;
inline int __syncthreads_or(int pred) {
    EmuBlockState& st = *g_emu_block;
    const int c = tl_vote_calls++;
    if (pred) st.vote[c % 3].fetch_or(1);
    st.bar->arrive_and_wait();
    const int r = st.vote[c % 3].load();
    st.vote[(c + 1) % 3].store(0);
    st.bar->arrive_and_wait();
    return r;
}

template <typename T, typename F>
inline T emu_exchange(T v, F src_of) {
    static_assert(sizeof(T) <= 8, "shuffle of a value wider than 64 bits");
    const int t = (int)threadIdx.x, w = t / 32, l = t % 32;
    EmuWarp& wp = *g_emu_block->warps[w];
    if (wp.alive.load() != 32) g_emu_violations.fetch_add(1);
    uint64_t bits = 0;
    memcpy(&bits, &v, sizeof(T));
    wp.slot[l] = bits;
    wp.bar->arrive_and_wait();
    const int src = src_of(l);
    uint64_t got = wp.slot[(src >= 0 && src < 32) ? src : l];
    wp.bar->arrive_and_wait();
    T r;
    memcpy(&r, &got, sizeof(T));
    return r;
}

// every lane's value, for warp-wide votes and reductions
template <typename T>
inline void emu_gather(T v, T out[32]) {
    static_assert(sizeof(T) <= 8, "value wider than 64 bits");
    const int t = (int)threadIdx.x, w = t / 32, l = t % 32;
    EmuWarp& wp = *g_emu_block->warps[w];
    if (wp.alive.load() != 32) g_emu_violations.fetch_add(1);
    uint64_t bits = 0;
    memcpy(&bits, &v, sizeof(T));
    wp.slot[l] = bits;
    wp.bar->arrive_and_wait();
    for (int k = 0; k < 32; ++k) memcpy(&out[k], &wp.slot[k], sizeof(T));
    wp.bar->arrive_and_wait();
}

inline int __any_sync(unsigned, int pred) {
    int all[32];
    emu_gather(pred ? 1 : 0, all);
    for (int k = 0; k < 32; ++k)
        if (all[k]) return 1;
    return 0;
}

inline unsigned __ballot_sync(unsigned, int pred) {
    int all[32];
    emu_gather(pred ? 1 : 0, all);
    unsigned m = 0;
    for (int k = 0; k < 32; ++k) m |= (unsigned)all[k] << k;
    return m;
}
template <typename T>
inline T __reduce_min_sync(unsigned, T v) {
    T all[32];
    emu_gather(v, all);
    return *std::min_element(all, all + 32);
}
template <typename T>
inline T __reduce_max_sync(unsigned, T v) {
    T all[32];
    emu_gather(v, all);
    return *std::max_element(all, all + 32);
}
inline void __syncwarp(unsigned = 0xffffffffu) {
    EmuWarp& wp = *g_emu_block->warps[(int)threadIdx.x / 32];
    if (wp.alive.load() != 32) g_emu_violations.fetch_add(1);
    wp.bar->arrive_and_wait();
}

template <typename T>
inline T __shfl_xor_sync(unsigned, T v, int mask) {
    return emu_exchange(v, [mask](int l) { return l ^ mask; });
}
template <typename T>
inline T __shfl_sync(unsigned, T v, int src) {
    return emu_exchange(v, [src](int) { return src & 31; });
}
template <typename T>
inline T __shfl_up_sync(unsigned, T v, int d) {
    return emu_exchange(v, [d](int l) { return l >= d ? l - d : l; });
}
template <typename T>
inline T __shfl_down_sync(unsigned, T v, int d) {
    return emu_exchange(v, [d](int l) { return l + d < 32 ? l + d : l; });
}

template <typename T>
inline T atomicAdd(T* p, T v) {
    return std::atomic_ref<T>(*p).fetch_add(v);
}

template <typename T>
inline T atomicOr(T* p, T v) {
    return std::atomic_ref<T>(*p).fetch_or(v);
}
template <typename T>
inline T atomicAnd(T* p, T v) {
    return std::atomic_ref<T>(*p).fetch_and(v);
}
template <typename T>
inline T atomicMin(T* p, T v) {
    std::atomic_ref<T> a(*p);
    T cur = a.load();
    while (v < cur && !a.compare_exchange_weak(cur, v)) {
    }
    return cur;
}
template <typename T>
inline T atomicMax(T* p, T v) {
    std::atomic_ref<T> a(*p);
    T cur = a.load();
    while (v > cur && !a.compare_exchange_weak(cur, v)) {
    }
    return cur;
}

template <typename T>
inline T atomicCAS(T* p, T cmp, T val) {
    std::atomic_ref<T>(*p).compare_exchange_strong(cmp, val);
    return cmp;
}

// Runs kernel(args...) over grid x block (1D blocks, a 3D grid), with
// `smem_bytes` of dynamic shared memory.
template <typename K, typename... A>
inline void emu_launch_smem(emu_dim3 grid, unsigned threads, size_t smem_bytes, K kernel, A... args) {
    std::vector<uint64_t> dyn((smem_bytes + 7) / 8 + 2);   // 16-byte aligned start below
    g_emu_dyn_smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn.data()) + 15) & ~uintptr_t(15));
    gridDim = grid;
    blockDim = emu_dim3{threads, 1, 1};
    for (unsigned bz = 0; bz < grid.z; ++bz)
    for (unsigned by = 0; by < grid.y; ++by)
        for (unsigned bx = 0; bx < grid.x; ++bx) {
            EmuBlockState st;
            st.bar = std::make_unique<std::barrier<>>((std::ptrdiff_t)threads);
            for (unsigned w = 0; w < (threads + 31) / 32; ++w) {
                // a last, partial warp has fewer lanes: a full-warp shuffle there counts as a violation
                const int lanes = (int)std::min(32u, threads - 32 * w);
                auto wp = std::make_unique<EmuWarp>();
                wp->bar = std::make_unique<std::barrier<>>(lanes);
                wp->alive = lanes;
                st.warps.push_back(std::move(wp));
            }
            g_emu_block = &st;
            std::vector<std::thread> pool;
            pool.reserve(threads);
            for (unsigned t = 0; t < threads; ++t)
                pool.emplace_back([&, t, bx, by, bz] {
                    threadIdx = emu_dim3{t, 0, 0};
                    blockIdx = emu_dim3{bx, by, bz};
                    kernel(args...);
                    EmuWarp& wp = *st.warps[t / 32];
                    wp.alive.fetch_sub(1);
                    wp.bar->arrive_and_drop();
                    st.bar->arrive_and_drop();
                });
            for (auto& th : pool) th.join();
            g_emu_block = nullptr;
        }
    g_emu_dyn_smem = nullptr;
}

template <typename K, typename... A>
inline void emu_launch(emu_dim3 grid, unsigned threads, K kernel, A... args) {
    emu_launch_smem(grid, threads, 0, kernel, args...);
}
