// Test-only host shim that runs a CUDA kernel's source on the CPU: every CUDA thread of a block
// is a fiber (ucontext) of one host thread, switched at barriers and warp exchanges; blocks run
// one after another.  It exists to check the logic of the library's plain (non-tensor-core)
// kernels on a machine without a GPU: index arithmetic, warp shuffles, block barriers and the
// order of sums.  It is not a CUDA implementation: no memory model beyond sequential
// consistency, no timing, and nothing of the library links against it.
//
// Semantics kept from CUDA: __syncthreads() waits for every thread of the block that has not
// exited (exited threads leave the barrier's count); __shfl_*_sync, votes and __syncwarp
// exchange among the lanes of a warp and record a violation when a lane of the warp has
// already exited; a barrier that can never complete (threads waiting at different barriers)
// records a violation and ends the block.  `__shared__` variables are function statics, valid
// because one block runs at a time.
#pragma once

#define GSPARC_HOST_SHIM 1

#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>

#include <ucontext.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <memory>
#include <vector>

using std::max;   // CUDA's device min / max overloads
using std::min;

struct emu_dim3 {
    unsigned x = 1, y = 1, z = 1;
};

inline emu_dim3 threadIdx, blockIdx;

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
inline float __fdividef(float a, float b) { return a / b; }   // the device's is an approximation
inline void __sincosf(float x, float* s, float* c) { sincosf(x, s, c); }
inline float __int_as_float(int i) {
    float f;
    memcpy(&f, &i, 4);
    return f;
}
inline float __uint_as_float(unsigned u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}
inline int __ffsll(long long x) { return __builtin_ffsll(x); }
inline int __ffs(int x) { return __builtin_ffs(x); }
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

enum EmuState { kEmuRun = 0, kEmuAtBlockBarrier = 1, kEmuAtWarpBarrier = 2, kEmuDone = 3 };

struct EmuFiber {
    ucontext_t ctx;
    std::unique_ptr<char[]> stack;
    int state = kEmuRun;
    int votes = 0;   // __syncthreads_or calls made
};

struct EmuBlockState {
    std::vector<EmuFiber> fib;
    ucontext_t sched;
    int cur = -1;
    std::vector<uint64_t> slot;   // warp exchange slots, 32 per warp
    int vote[3] = {0, 0, 0};      // __syncthreads_or, see below
    std::function<void()> body;
};

inline EmuBlockState* g_emu_block = nullptr;
inline std::atomic<int> g_emu_violations{0};

inline void emu_wait(int state) {
    EmuBlockState& b = *g_emu_block;
    b.fib[b.cur].state = state;
    swapcontext(&b.fib[b.cur].ctx, &b.sched);
}

inline int emu_warp_alive(int w) {
    EmuBlockState& b = *g_emu_block;
    int n = 0;
    const int hi = std::min<int>((int)b.fib.size(), 32 * (w + 1));
    for (int t = 32 * w; t < hi; ++t) n += b.fib[t].state != kEmuDone;
    return n;
}

inline void __syncthreads() { emu_wait(kEmuAtBlockBarrier); }

// Call c of a thread uses slot c % 3; between its two barriers every thread clears slot
// (c + 1) % 3, which nobody reads then and nobody sets before the second barrier.
inline int __syncthreads_or(int pred) {
    EmuBlockState& b = *g_emu_block;
    const int c = b.fib[b.cur].votes++;
    if (pred) b.vote[c % 3] = 1;
    __syncthreads();
    const int r = b.vote[c % 3];
    b.vote[(c + 1) % 3] = 0;
    __syncthreads();
    return r;
}

template <typename T, typename F>
inline T emu_exchange(T v, F src_of) {
    static_assert(sizeof(T) <= 8, "shuffle of a value wider than 64 bits");
    EmuBlockState& b = *g_emu_block;
    const int t = b.cur, w = t / 32, l = t % 32;
    if (emu_warp_alive(w) != 32) g_emu_violations.fetch_add(1);
    uint64_t bits = 0;
    memcpy(&bits, &v, sizeof(T));
    b.slot[32 * w + l] = bits;
    emu_wait(kEmuAtWarpBarrier);
    const int src = src_of(l);
    const uint64_t got = b.slot[32 * w + ((src >= 0 && src < 32) ? src : l)];
    emu_wait(kEmuAtWarpBarrier);
    T r;
    memcpy(&r, &got, sizeof(T));
    return r;
}

// every lane's value, for warp-wide votes and reductions
template <typename T>
inline void emu_gather(T v, T out[32]) {
    static_assert(sizeof(T) <= 8, "value wider than 64 bits");
    EmuBlockState& b = *g_emu_block;
    const int t = b.cur, w = t / 32, l = t % 32;
    if (emu_warp_alive(w) != 32) g_emu_violations.fetch_add(1);
    uint64_t bits = 0;
    memcpy(&bits, &v, sizeof(T));
    b.slot[32 * w + l] = bits;
    emu_wait(kEmuAtWarpBarrier);
    for (int k = 0; k < 32; ++k) memcpy(&out[k], &b.slot[32 * w + k], sizeof(T));
    emu_wait(kEmuAtWarpBarrier);
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
    EmuBlockState& b = *g_emu_block;
    if (emu_warp_alive(b.cur / 32) != 32) g_emu_violations.fetch_add(1);
    emu_wait(kEmuAtWarpBarrier);
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

// the 16-byte vector atomic of sm_90+: one atomic add per element
inline float4 atomicAdd(float4* p, float4 v) {
    float4 old;
    old.x = std::atomic_ref<float>(p->x).fetch_add(v.x);
    old.y = std::atomic_ref<float>(p->y).fetch_add(v.y);
    old.z = std::atomic_ref<float>(p->z).fetch_add(v.z);
    old.w = std::atomic_ref<float>(p->w).fetch_add(v.w);
    return old;
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

// Runs kernel(args...) over grid x block (1D blocks, a 3D grid), with `smem_bytes` of dynamic
// shared memory.  Within a block the fibers run round-robin until each waits or exits; a
// barrier is released when every thread that has not exited waits at it (for a warp barrier,
// every such lane of the warp).
// EMU_ORDER=reverse runs each sweep from the last thread to the first: a read that is missing
// its barrier after another thread's write sees the stale value in one of the two orders.
inline bool emu_reverse_order() {
    static const bool rev = [] {
        const char* e = getenv("EMU_ORDER");
        return e && strcmp(e, "reverse") == 0;
    }();
    return rev;
}

inline void emu_fiber_entry() {
    EmuBlockState& b = *g_emu_block;
    b.body();
    b.fib[b.cur].state = kEmuDone;   // returns to the scheduler through uc_link
}

template <typename K, typename... A>
inline void emu_launch_smem(emu_dim3 grid, unsigned threads, size_t smem_bytes, K kernel, A... args) {
    constexpr size_t kStack = 256 * 1024;
    // exactly the bytes asked for (rounded up to the 16-byte alignment), so that the sanitizer
    // sees an access past them
    const size_t dyn_bytes = smem_bytes ? (smem_bytes + 15) / 16 * 16 : 16;
    std::unique_ptr<unsigned char, void (*)(void*)> dyn(static_cast<unsigned char*>(aligned_alloc(16, dyn_bytes)),
                                                         free);
    g_emu_dyn_smem = dyn.get();
    gridDim = grid;
    blockDim = emu_dim3{threads, 1, 1};
    const int nw = (int)((threads + 31) / 32);
    for (unsigned bz = 0; bz < grid.z; ++bz)
        for (unsigned by = 0; by < grid.y; ++by)
            for (unsigned bx = 0; bx < grid.x; ++bx) {
                EmuBlockState st;
                st.fib.resize(threads);
                st.slot.assign(32 * (size_t)nw, 0);
                st.body = [&] { kernel(args...); };
                blockIdx = emu_dim3{bx, by, bz};
                for (unsigned t = 0; t < threads; ++t) {
                    EmuFiber& f = st.fib[t];
                    f.stack.reset(new char[kStack]);
                    getcontext(&f.ctx);
                    f.ctx.uc_stack.ss_sp = f.stack.get();
                    f.ctx.uc_stack.ss_size = kStack;
                    f.ctx.uc_link = &st.sched;
                    makecontext(&f.ctx, emu_fiber_entry, 0);
                }
                g_emu_block = &st;
                for (;;) {
                    for (unsigned k = 0; k < threads; ++k) {
                        const unsigned t = emu_reverse_order() ? threads - 1 - k : k;
                        if (st.fib[t].state != kEmuRun) continue;
                        st.cur = (int)t;
                        threadIdx = emu_dim3{t, 0, 0};
                        swapcontext(&st.sched, &st.fib[t].ctx);
                    }
                    // release the barriers that every live participant has reached
                    bool alive = false, all_block = true, released = false;
                    for (unsigned t = 0; t < threads; ++t) {
                        const int s = st.fib[t].state;
                        if (s == kEmuDone) continue;
                        alive = true;
                        if (s != kEmuAtBlockBarrier) all_block = false;
                    }
                    if (!alive) break;
                    if (all_block) {
                        for (auto& f : st.fib)
                            if (f.state == kEmuAtBlockBarrier) f.state = kEmuRun;
                        released = true;
                    }
                    for (int w = 0; w < nw && !all_block; ++w) {
                        const unsigned lo = 32u * w, hi = std::min(threads, 32u * (w + 1));
                        bool any = false, all_warp = true;
                        for (unsigned t = lo; t < hi; ++t) {
                            const int s = st.fib[t].state;
                            if (s == kEmuDone) continue;
                            any = true;
                            if (s != kEmuAtWarpBarrier) all_warp = false;
                        }
                        if (any && all_warp) {
                            for (unsigned t = lo; t < hi; ++t)
                                if (st.fib[t].state == kEmuAtWarpBarrier) st.fib[t].state = kEmuRun;
                            released = true;
                        }
                    }
                    if (!released) {   // threads wait at barriers that can never complete
                        g_emu_violations.fetch_add(1);
                        break;
                    }
                }
                g_emu_block = nullptr;
            }
    g_emu_dyn_smem = nullptr;
}

template <typename K, typename... A>
inline void emu_launch(emu_dim3 grid, unsigned threads, K kernel, A... args) {
    emu_launch_smem(grid, threads, 0, kernel, args...);
}
