// Tile binning and directional (receiver-distance) sorting.
//
// Algorithm 1: IntersectGaussians per pixel, then "sort by depth to receiver";
// Sec. 1 names the fully parallel directional sort.  Tiled form: each
// Gaussian's footprint box (azimuth wrapping at +-pi) gives one (Gaussian,
// tile) pair per touched 16x16 tile with key (tile_id << 32) | bits(r); the
// pairs, emitted in Gaussian-index order, are sorted stably by key, so every
// tile's list comes out ordered by (r, index).
//
// Kernels (all on the caller's stream, no host synchronisation):
//   k_count        tiles per Gaussian + block-local exclusive scan
//   k_scan_blocks  scan of block totals, pair count, capacity check
//   k_emit         keys / values in Gaussian-index order
//   k_hist         digit histograms of every pass in one read of the keys,
//                  and zeroing of the look-back flags
//   k_hist_scan    exclusive scan of each pass's 256 bins
//   k_onesweep     one LSD pass over 8 bits: stable in-tile ranking with
//                  warp match, decoupled look-back across tiles (bounded
//                  spins, GSPARC_ERR_TIMEOUT on expiry), scatter
//   k_ranges       [start, end) of each tile from adjacent keys

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "internal.cuh"

namespace gsparc {
namespace {

constexpr int kScanThreads = 256;
constexpr int kOsThreads = 256;
constexpr int kOsWarps = kOsThreads / 32;
constexpr int kOsKpt = 8;                           // keys per thread
constexpr int kOsTile = kOsThreads * kOsKpt;        // 2048 keys per sort tile
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 20;
constexpr int kLookWin = 8;                         // predecessors read per look-back round trip
constexpr int kMaxPasses = 7;

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    if (status) atomicCAS(reinterpret_cast<int*>(status), 0, code);
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Column / row tile ranges touched by one projection record.  Every float
// step is a single correctly rounded operation (explicit _rn intrinsics keep
// the compiler from fusing), so the integer result is reproducible.
struct Foot {
    int ty0, ty1;
    int a0, a1;   // first column-tile range (inclusive)
    int b0, b1;   // second range, empty when b0 > b1
};

__device__ __forceinline__ bool footprint(const float4 p, int H, int W, int TW, Foot& f) {
    const float px = p.x, py = p.y, ex = p.z, ey = p.w;
    if (!(ey >= 0.f) || !(ex >= 0.f)) return false;
    if (!(fabsf(px) <= 1048576.f) || !(fabsf(py) <= 1048576.f)) return false;
    float fy0 = ceilf(__fsub_rn(__fsub_rn(py, ey), 0.5f));
    float fy1 = floorf(__fsub_rn(__fadd_rn(py, ey), 0.5f));
    fy0 = fmaxf(fy0, 0.f);
    fy1 = fminf(fy1, (float)(H - 1));
    if (!(fy0 <= fy1)) return false;
    f.ty0 = ((int)fy0) >> 4;
    f.ty1 = ((int)fy1) >> 4;
    f.b0 = 1;
    f.b1 = 0;
    if (!(ex < 0.5f * (float)W)) {
        f.a0 = 0;
        f.a1 = TW - 1;
        return true;
    }
    const float fx0 = ceilf(__fsub_rn(__fsub_rn(px, ex), 0.5f));
    const float fx1 = floorf(__fsub_rn(__fadd_rn(px, ex), 0.5f));
    if (!(fx0 <= fx1)) return false;
    const int x0 = (int)fx0, x1 = (int)fx1;
    const int a = ((x0 % W) + W) % W;
    const int b = ((x1 % W) + W) % W;
    if (a <= b) {
        f.a0 = a >> 4;
        f.a1 = b >> 4;
    } else if ((a >> 4) <= (b >> 4)) {
        f.a0 = 0;
        f.a1 = TW - 1;
    } else {
        f.a0 = 0;
        f.a1 = b >> 4;
        f.b0 = a >> 4;
        f.b1 = TW - 1;
    }
    return true;
}

__device__ __forceinline__ uint32_t foot_count(const Foot& f) {
    const int cols = (f.a1 - f.a0 + 1) + (f.b1 >= f.b0 ? f.b1 - f.b0 + 1 : 0);
    return (uint32_t)((f.ty1 - f.ty0 + 1) * cols);
}

// Block-wide exclusive scan of one value per thread (blockDim.x == 256).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (kScanThreads / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kScanThreads / 32)) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[kScanThreads / 32 - 1];
    const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0;
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_count(int N, int H, int W, int TW,
                                                        const float4* __restrict__ proj,
                                                        uint32_t* __restrict__ local,
                                                        uint32_t* __restrict__ blk) {
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int i = blockIdx.x * kScanThreads + threadIdx.x;
    uint32_t c = 0;
    if (i < N) {
        Foot f;
        if (footprint(proj[2 * i], H, W, TW, f)) c = foot_count(f);
    }
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(c, s_warp, total);
    if (i < N) local[i] = ex;
    if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// One block of 1024 threads scans the block totals (in place, exclusive).
__global__ void __launch_bounds__(1024) k_scan_blocks(int nblk, uint32_t* __restrict__ blk,
                                                      uint32_t* __restrict__ n_pairs,
                                                      uint32_t* __restrict__ n_sort, uint32_t cap,
                                                      int32_t* status) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nblk; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nblk ? blk[i] : 0;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const uint64_t carry = s_carry;
        const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0;
        const uint64_t ex = carry + before + x - v;
        if (i < nblk) blk[i] = (uint32_t)(ex > 0xffffffffull ? 0xffffffffull : ex);
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint64_t tot = s_carry;
        n_pairs[0] = (uint32_t)(tot > 0xffffffffull ? 0xffffffffull : tot);
        if (tot > cap) set_status(status, GSPARC_ERR_CAPACITY);
        n_sort[0] = (uint32_t)(tot > cap ? cap : tot);
    }
}

__global__ void __launch_bounds__(kScanThreads) k_emit(int N, int H, int W, int TW,
                                                       const float4* __restrict__ proj,
                                                       const uint32_t* __restrict__ local,
                                                       const uint32_t* __restrict__ blk, uint32_t cap,
                                                       uint64_t* __restrict__ keys,
                                                       uint32_t* __restrict__ vals) {
    const int i = blockIdx.x * kScanThreads + threadIdx.x;
    if (i >= N) return;
    Foot f;
    if (!footprint(proj[2 * i], H, W, TW, f)) return;
    const uint32_t rbits = __float_as_uint(proj[2 * i + 1].w);
    uint64_t pos = (uint64_t)blk[blockIdx.x] + local[i];
    for (int ty = f.ty0; ty <= f.ty1; ++ty) {
        for (int tx = f.a0; tx <= f.a1; ++tx, ++pos) {
            if (pos < cap) {
                keys[pos] = ((uint64_t)(ty * TW + tx) << 32) | rbits;
                vals[pos] = (uint32_t)i;
            }
        }
        for (int tx = f.b0; tx <= f.b1; ++tx, ++pos) {
            if (pos < cap) {
                keys[pos] = ((uint64_t)(ty * TW + tx) << 32) | rbits;
                vals[pos] = (uint32_t)i;
            }
        }
    }
}

// Digit histograms for all passes, plus zeroing of the look-back flags.
__global__ void __launch_bounds__(256) k_hist(const uint64_t* __restrict__ keys,
                                              const uint32_t* __restrict__ n_sort, int passes,
                                              uint32_t* __restrict__ hist, uint32_t* __restrict__ look,
                                              int look_tiles_cap) {
    __shared__ uint32_t s_hist[kMaxPasses][256];
    const uint32_t n = n_sort[0];
    for (int t = threadIdx.x; t < passes * 256; t += blockDim.x) (&s_hist[0][0])[t] = 0;
    __syncthreads();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint64_t k = keys[j];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 0xff], 1u);
    }
    // zero the look-back flags of every pass for the tiles this sort uses
    const uint32_t ntiles = (n + kOsTile - 1) / kOsTile;
    const uint64_t zn = (uint64_t)ntiles * 256;
    for (int p = 0; p < passes; ++p) {
        uint32_t* lp = look + (size_t)p * look_tiles_cap * 256;
        for (uint64_t j = blockIdx.x * blockDim.x + threadIdx.x; j < zn; j += stride) lp[j] = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < passes * 256; t += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[t];
        if (c) atomicAdd(&hist[t], c);
    }
}

__global__ void __launch_bounds__(256) k_hist_scan(int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_warp[8];
    for (int p = 0; p < passes; ++p) {
        const uint32_t v = hist[p * 256 + threadIdx.x];
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, s_warp, total);
        hist[p * 256 + threadIdx.x] = ex;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kOsThreads, 2) k_onesweep(
    int pass, const uint64_t* __restrict__ ksrc, const uint32_t* __restrict__ vsrc,
    uint64_t* __restrict__ kdst, uint32_t* __restrict__ vdst, const uint32_t* __restrict__ n_sort,
    uint32_t* __restrict__ ctr, uint32_t* __restrict__ look, const uint32_t* __restrict__ digit_off,
    int32_t* status) {
    __shared__ uint32_t s_whist[kOsWarps][256];
    __shared__ uint32_t s_excl[256];
    __shared__ uint32_t s_tile;
    const uint32_t n = n_sort[0];
    const uint32_t ntiles = (n + kOsTile - 1) / kOsTile;
    const int shift = 8 * pass;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
        for (int t = threadIdx.x; t < kOsWarps * 256; t += kOsThreads) (&s_whist[0][0])[t] = 0;
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t base = tile * kOsTile + warp * (kOsKpt * 32);
        uint64_t k[kOsKpt];
        uint32_t v[kOsKpt];
        uint32_t pos[kOsKpt];
#pragma unroll
        for (int j = 0; j < kOsKpt; ++j) {
            const uint32_t idx = base + j * 32 + lane;
            const bool ok = idx < n;
            k[j] = ok ? ksrc[idx] : ~0ull;
            v[j] = ok ? vsrc[idx] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kOsKpt; ++j) {
            const uint32_t idx = base + j * 32 + lane;
            const uint32_t d = idx < n ? (uint32_t)((k[j] >> shift) & 0xff) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t before = d < 256 ? s_whist[warp][d] : 0u;
            pos[j] = before + __popc(peers & lt_mask);
            __syncwarp();
            if (d < 256 && lane == (__ffs(peers) - 1)) s_whist[warp][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive scan across warps, publish, look back
        {
            const int d = threadIdx.x;
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < kOsWarps; ++w) {
                const uint32_t c = s_whist[w][d];
                s_whist[w][d] = sum;
                sum += c;
            }
            uint32_t* my = look + (size_t)tile * 256 + d;
            uint32_t prefix = 0;
            if (tile == 0) {
                st_relaxed(my, kFlagInc | sum);
            } else {
                st_relaxed(my, kFlagAgg | sum);
                // look back over windows of kLookWin predecessors: the window's flags are
                // loaded together (one L2 round trip per window, not per tile), then summed
                // from the nearest tile down to the first inclusive prefix
                int j = (int)tile - 1;
                int spins = 0;
                bool fin = false;
                while (!fin) {
                    uint32_t v[kLookWin];
#pragma unroll
                    for (int q = 0; q < kLookWin; ++q)
                        v[q] = (j - q >= 0) ? ld_relaxed(look + (size_t)(j - q) * 256 + d) : kFlagInc;
#pragma unroll
                    for (int q = 0; q < kLookWin; ++q) {
                        if (fin) break;
                        uint32_t s = v[q];
                        while ((s & ~kValMask) == 0) {   // that tile has not published yet
                            if (++spins > kSpinLimit) {
                                set_status(status, GSPARC_ERR_TIMEOUT);
                                s = kFlagInc;
                                break;
                            }
                            __nanosleep(32);
                            s = ld_relaxed(look + (size_t)(j - q) * 256 + d);
                        }
                        prefix += s & kValMask;
                        if ((s & ~kValMask) == kFlagInc) fin = true;
                    }
                    j -= kLookWin;
                }
                st_relaxed(my, kFlagInc | ((prefix + sum) & kValMask));
            }
            s_excl[d] = digit_off[d] + prefix;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kOsKpt; ++j) {
            const uint32_t idx = base + j * 32 + lane;
            if (idx < n) {
                const uint32_t d = (uint32_t)((k[j] >> shift) & 0xff);
                const uint32_t dst = s_excl[d] + s_whist[warp][d] + pos[j];
                if (dst < n) {   // always true unless a look-back wait expired
                    kdst[dst] = k[j];
                    vdst[dst] = v[j];
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_ranges(const uint64_t* __restrict__ keys,
                                                const uint32_t* __restrict__ n_sort, uint32_t T,
                                                uint2* __restrict__ ranges) {
    const uint32_t n = n_sort[0];
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint32_t t = (uint32_t)(keys[j] >> 32);
        if (t >= T) continue;   // only after an expired look-back wait
        if (j == 0 || (uint32_t)(keys[j - 1] >> 32) != t) ranges[t].x = j;
        if (j + 1 == n || (uint32_t)(keys[j + 1] >> 32) != t) ranges[t].y = j + 1;
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t local, blk, k0, k1, v0, v1, hist, ctr, misc, look, total;
    int nblk, passes, look_tiles;
};

int num_passes(int ntiles) {
    int bits = 0;
    while ((1ll << bits) < ntiles) ++bits;
    return 4 + (bits + 7) / 8;
}

Layout layout(int N, int64_t cap, int ntiles) {
    Layout L;
    L.nblk = (N + kScanThreads - 1) / kScanThreads;
    L.passes = num_passes(ntiles);
    L.look_tiles = (int)((cap + kOsTile - 1) / kOsTile);
    size_t o = 0;
    L.local = o; o += align256((size_t)N * 4);
    L.blk = o;   o += align256((size_t)(L.nblk + 1) * 4);
    L.k0 = o;    o += align256((size_t)cap * 8);
    L.k1 = o;    o += align256((size_t)cap * 8);
    L.v0 = o;    o += align256((size_t)cap * 4);
    L.v1 = o;    o += align256((size_t)cap * 4);
    L.hist = o;  o += align256((size_t)kMaxPasses * 256 * 4);
    L.ctr = o;   o += align256((size_t)kMaxPasses * 4);
    L.misc = o;  o += align256(16);
    L.look = o;  o += align256((size_t)L.passes * L.look_tiles * 256 * 4);
    L.total = o;
    return L;
}

}  // namespace
}  // namespace gsparc

using namespace gsparc;

extern "C" int gsparc_bin_sort_workspace(const gsparc_view* view, int32_t N, int64_t pair_capacity,
                                         size_t* ws_bytes) {
    if (!view_ok(view) || N < 0 || pair_capacity < 0 || pair_capacity >= (1ll << 31) || !ws_bytes)
        return GSPARC_ERR_INVALID;
    *ws_bytes = layout(N, pair_capacity, tiles_x(*view) * tiles_y(*view)).total;
    return GSPARC_OK;
}

extern "C" int gsparc_bin_sort(const gsparc_view* view, int32_t N, const float* proj,
                               int64_t pair_capacity, void* ws, size_t ws_bytes, uint32_t* sorted_ids,
                               uint64_t* sorted_keys, uint32_t* tile_ranges, uint32_t* n_pairs,
                               int32_t* d_status, void* stream) {
    if (!view_ok(view) || N < 0 || pair_capacity < 0 || pair_capacity >= (1ll << 31))
        return GSPARC_ERR_INVALID;
    if (!tile_ranges || !n_pairs || (N > 0 && !proj) || (pair_capacity > 0 && !sorted_ids))
        return GSPARC_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(proj) & 15) return GSPARC_ERR_INVALID;
    const int TW = tiles_x(*view), TH = tiles_y(*view), T = TW * TH;
    const Layout L = layout(N, pair_capacity, T);
    if (!ws || ws_bytes < L.total) return GSPARC_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return GSPARC_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    char* w = static_cast<char*>(ws);
    uint32_t* local = reinterpret_cast<uint32_t*>(w + L.local);
    uint32_t* blk = reinterpret_cast<uint32_t*>(w + L.blk);
    uint64_t* kb[2] = {reinterpret_cast<uint64_t*>(w + L.k0), reinterpret_cast<uint64_t*>(w + L.k1)};
    uint32_t* vb[2] = {reinterpret_cast<uint32_t*>(w + L.v0), reinterpret_cast<uint32_t*>(w + L.v1)};
    uint32_t* hist = reinterpret_cast<uint32_t*>(w + L.hist);
    uint32_t* ctr = reinterpret_cast<uint32_t*>(w + L.ctr);
    uint32_t* misc = reinterpret_cast<uint32_t*>(w + L.misc);
    uint32_t* look = reinterpret_cast<uint32_t*>(w + L.look);
    const uint32_t cap = (uint32_t)pair_capacity;

    if (cudaMemsetAsync(tile_ranges, 0, (size_t)T * 2 * sizeof(uint32_t), s) != cudaSuccess)
        return GSPARC_ERR_CUDA;
    // hist, ctr and misc are contiguous
    if (cudaMemsetAsync(w + L.hist, 0, L.look - L.hist, s) != cudaSuccess) return GSPARC_ERR_CUDA;
    if (N == 0) {
        if (cudaMemsetAsync(n_pairs, 0, sizeof(uint32_t), s) != cudaSuccess) return GSPARC_ERR_CUDA;
        return GSPARC_OK;
    }
    const float4* p4 = reinterpret_cast<const float4*>(proj);
    k_count<<<L.nblk, kScanThreads, 0, s>>>(N, view->H, view->W, TW, p4, local, blk);
    k_scan_blocks<<<1, 1024, 0, s>>>(L.nblk, blk, n_pairs, misc, cap, d_status);
    k_emit<<<L.nblk, kScanThreads, 0, s>>>(N, view->H, view->W, TW, p4, local, blk, cap, kb[0], vb[0]);
    if (cudaGetLastError() != cudaSuccess) return GSPARC_ERR_CUDA;
    if (cap == 0) return GSPARC_OK;

    const int sms = num_sms();
    const int hist_blocks = sms * 2;
    k_hist<<<hist_blocks, 256, 0, s>>>(kb[0], misc, L.passes, hist, look, L.look_tiles);
    k_hist_scan<<<1, 256, 0, s>>>(L.passes, hist);
    const int os_blocks = (int)std::min<int64_t>(L.look_tiles, (int64_t)sms * 2);
    uint64_t* kfinal = nullptr;
    for (int p = 0; p < L.passes; ++p) {
        const int src = p & 1, dst = src ^ 1;
        const bool last = p == L.passes - 1;
        uint64_t* kd = last ? (sorted_keys ? sorted_keys : kb[dst]) : kb[dst];
        uint32_t* vd = last ? sorted_ids : vb[dst];
        k_onesweep<<<os_blocks, kOsThreads, 0, s>>>(p, kb[src], vb[src], kd, vd, misc, ctr + p,
                                                    look + (size_t)p * L.look_tiles * 256,
                                                    hist + p * 256, d_status);
        if (last) kfinal = kd;
    }
    k_ranges<<<sms * 4, 256, 0, s>>>(kfinal, misc, (uint32_t)T, reinterpret_cast<uint2*>(tile_ranges));
    return launch_status();
}

// ---------------------------------------------------------------------------------------------
// Scratch-free variant for callers that cannot allocate device memory (a real-time loop that
// must not pay cudaMalloc's device-wide synchronisation after start-up, a plugin given buffers
// but no allocator).  Same kernels and launch sequence as gsparc_bin_sort; the scratch lives in
// one file-scope device array instead of a caller workspace.
// ---------------------------------------------------------------------------------------------

namespace gsparc {
namespace {

constexpr size_t kNoAllocBytes = size_t(15) << 20;   // covers layout(65536, 524288, 7 passes)
static_assert(kOsTile == 2048, "the no-alloc budget assumes 2048-key sort tiles");
constexpr int kMaxDevices = 64;

// Host code must not use this symbol as an address: it only names the array.  The device
// address comes from cudaGetSymbolAddress, once per device, with that device current.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::once_flag g_noalloc_once[kMaxDevices];
void* g_noalloc_ptr[kMaxDevices];
cudaError_t g_noalloc_err[kMaxDevices];

}  // namespace
}  // namespace gsparc

extern "C" int gsparc_bin_sort_noalloc(const gsparc_view* view, int32_t N, const float* proj,
                                       int64_t pair_capacity, uint32_t* sorted_ids,
                                       uint64_t* sorted_keys, uint32_t* tile_ranges, uint32_t* n_pairs,
                                       int32_t* d_status, void* stream) {
    if (!view_ok(view) || N < 0 || pair_capacity < 0) return GSPARC_ERR_INVALID;
    if (N > GSPARC_NOALLOC_MAX_N || pair_capacity > GSPARC_NOALLOC_MAX_PAIRS) return GSPARC_ERR_TOO_LARGE;
    if (!tile_ranges || !n_pairs || (N > 0 && !proj) || (pair_capacity > 0 && !sorted_ids))
        return GSPARC_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(proj) & 15) return GSPARC_ERR_INVALID;
    const int TW = tiles_x(*view), TH = tiles_y(*view), T = TW * TH;
    const Layout L = layout(N, pair_capacity, T);
    if (L.total > kNoAllocBytes) return GSPARC_ERR_TOO_LARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GSPARC_ERR_CUDA;
    std::call_once(g_noalloc_once[dev], [dev]() {
        g_noalloc_err[dev] = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
    });
    if (g_noalloc_err[dev] != cudaSuccess || !g_noalloc_ptr[dev]) return GSPARC_ERR_CUDA;

    cudaStream_t s = as_stream(stream);
    char* w = static_cast<char*>(g_noalloc_ptr[dev]);
    uint32_t* local = reinterpret_cast<uint32_t*>(w + L.local);
    uint32_t* blk = reinterpret_cast<uint32_t*>(w + L.blk);
    uint64_t* kb[2] = {reinterpret_cast<uint64_t*>(w + L.k0), reinterpret_cast<uint64_t*>(w + L.k1)};
    uint32_t* vb[2] = {reinterpret_cast<uint32_t*>(w + L.v0), reinterpret_cast<uint32_t*>(w + L.v1)};
    uint32_t* hist = reinterpret_cast<uint32_t*>(w + L.hist);
    uint32_t* ctr = reinterpret_cast<uint32_t*>(w + L.ctr);
    uint32_t* misc = reinterpret_cast<uint32_t*>(w + L.misc);
    uint32_t* look = reinterpret_cast<uint32_t*>(w + L.look);
    const uint32_t cap = (uint32_t)pair_capacity;

    // the array keeps the previous call's contents: clear the counters, histograms and
    // pass counters here (the look-back flags are cleared by k_hist)
    if (cudaMemsetAsync(tile_ranges, 0, (size_t)T * 2 * sizeof(uint32_t), s) != cudaSuccess)
        return GSPARC_ERR_CUDA;
    if (cudaMemsetAsync(w + L.hist, 0, L.look - L.hist, s) != cudaSuccess) return GSPARC_ERR_CUDA;
    if (N == 0) {
        if (cudaMemsetAsync(n_pairs, 0, sizeof(uint32_t), s) != cudaSuccess) return GSPARC_ERR_CUDA;
        return GSPARC_OK;
    }
    const float4* p4 = reinterpret_cast<const float4*>(proj);
    k_count<<<L.nblk, kScanThreads, 0, s>>>(N, view->H, view->W, TW, p4, local, blk);
    k_scan_blocks<<<1, 1024, 0, s>>>(L.nblk, blk, n_pairs, misc, cap, d_status);
    k_emit<<<L.nblk, kScanThreads, 0, s>>>(N, view->H, view->W, TW, p4, local, blk, cap, kb[0], vb[0]);
    if (cudaGetLastError() != cudaSuccess) return GSPARC_ERR_CUDA;
    if (cap == 0) return GSPARC_OK;
    const int sms = num_sms();
    k_hist<<<sms * 2, 256, 0, s>>>(kb[0], misc, L.passes, hist, look, L.look_tiles);
    k_hist_scan<<<1, 256, 0, s>>>(L.passes, hist);
    const int os_blocks = (int)std::min<int64_t>(L.look_tiles, (int64_t)sms * 2);
    uint64_t* kfinal = nullptr;
    for (int p = 0; p < L.passes; ++p) {
        const int src = p & 1, dst = src ^ 1;
        const bool last = p == L.passes - 1;
        uint64_t* kd = last ? (sorted_keys ? sorted_keys : kb[dst]) : kb[dst];
        uint32_t* vd = last ? sorted_ids : vb[dst];
        k_onesweep<<<os_blocks, kOsThreads, 0, s>>>(p, kb[src], vb[src], kd, vd, misc, ctr + p,
                                                    look + (size_t)p * L.look_tiles * 256,
                                                    hist + p * 256, d_status);
        if (last) kfinal = kd;
    }
    k_ranges<<<sms * 4, 256, 0, s>>>(kfinal, misc, (uint32_t)T, reinterpret_cast<uint2*>(tile_ranges));
    return launch_status();
}
