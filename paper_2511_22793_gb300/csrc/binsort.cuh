// Tile binning and directional (receiver-distance) sorting.
//
// Algorithm 1: IntersectGaussians per pixel followed by its depth sort step
// (depth = distance to the receiver); Sec. 1: the fully parallel directional
// sort.  Tiled form: each
// Gaussian's footprint box (azimuth wrapping at +-pi) gives one (Gaussian,
// tile) pair per touched 16x16 tile, and every tile's list is ordered by
// (r, index).
//
// The pairs go straight into per-tile buckets and each bucket is sorted on its
// own, so no pass ever runs over the whole pair array:
//   k_tile_count  pairs per tile (block-aggregated atomics); the last block to
//                 finish scans the counts into bucket offsets, tile ranges and
//                 the pair count, and checks the capacity
//   k_tile_emit   every pair, as the 64-bit sort key (bits(r) << 32) | index,
//                 into its tile's bucket (block-aggregated cursor atomics, so
//                 the order inside a bucket is arbitrary)
//   k_tile_sort   one CTA per tile: a distribution sort by depth (each key ranked
//                 against the few keys of its sub-bucket), up to kSortCap keys in
//                 shared memory over kSubBuckets sub-buckets; a bucket above kSortCap keys
//                 is cut into slices of about kSlice keys at boundaries of kSubBig depth
//                 sub-buckets, each slice sorted in shared memory by its own CTA (the
//                 tile's block and blocks past the tiles, from a work list of k_tile_count);
//                 when a sub-bucket holds too many keys (many equal depths), an
//                 LSD radix sort (8-bit digits, warp-match ranking, only the
//                 bytes that vary in the bucket), in a global ping-pong buffer
//                 for a bucket above kSortCap keys; writes the ids (and keys)
// The keys are unique (the index is part of the key), so any arrangement of a
// bucket sorts to the same list: the (r, index) order, bit for bit.
//
// Device code only (the entry points are in binsort.cu), so that the same source also builds for
// the host under the test suite's shim.

#pragma once

#include <math.h>
#include <stdint.h>

#include "device_common.cuh"

namespace gsparc {
namespace {

constexpr int kBinThreads = 256;
constexpr int kSmemTiles = 4096;                    // tile counters kept in shared memory up to this T
constexpr int kSortThreads = 1024;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortCap = 24576;                     // keys per bucket sorted in shared memory
constexpr int kSubBuckets = 8192;                   // sub-buckets of the in-tile distribution sort
constexpr int kSubMax = 64;                         // largest sub-bucket ranked by comparison
constexpr int kSubBig = 16384;                      // sub-buckets of a bucket above kSortCap keys
constexpr int kSubMaxBig = 256;                     // largest such sub-bucket ranked by comparison
constexpr int kSlice = 12288;                       // keys per slice of such a bucket, about

// Slices of a bucket of n keys beyond its first (its tile's own block takes slice 0): none up to
// kSortCap keys.
__device__ __host__ __forceinline__ uint32_t extra_slices(uint32_t n) {
    return n > (uint32_t)kSortCap ? (n + kSlice - 1) / kSlice - 1u : 0u;
}
// Buckets above kSortCap keys are sliced only when the tiles alone leave SMs idle; otherwise each
// is sorted by its tile's block (keys scattered in global memory), which moves fewer bytes.
inline bool slice_big_buckets(int T, int sms) { return T < sms; }
// Blocks of a k_tile_sort launch: one per SM (each holds 200+ KB of shared memory), or fewer when
// a list of cap pairs has fewer work items (its tiles and the extra slices of its buckets).
inline uint32_t sort_grid(int T, uint32_t cap, int sms) {
    const uint64_t most = (uint64_t)T + (slice_big_buckets(T, sms) ? cap / kSlice : 0u);
    return (uint32_t)(most < (uint64_t)sms ? most : (uint64_t)sms);
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

// Every (Gaussian, tile) pair of the 32 lanes' Gaussians, spread evenly over the lanes
// (a wide footprint would otherwise keep one lane looping while the others idle).  Pair
// k of the warp belongs to the lane whose exclusive..inclusive pair prefix holds k,
// found by a binary search over the lanes' prefixes; fn(tile, owner, active) runs on
// every lane in rounds of 32 pairs (active false past the warp's last pair).
template <class F>
__device__ __forceinline__ void warp_pairs(bool valid, const Foot& f, int TW, F&& fn) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wa = valid ? f.a1 - f.a0 + 1 : 0;
    const int cols = valid ? wa + (f.b1 >= f.b0 ? f.b1 - f.b0 + 1 : 0) : 0;
    const int c = valid ? (f.ty1 - f.ty0 + 1) * cols : 0;
    // ceil(2^32 / cols): the row of pair q is the high word of q * inv, or one less (fixed below)
    const uint64_t inv = cols > 0 ? ((1ull << 32) + (uint64_t)cols - 1) / (uint64_t)cols : 0ull;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(full, incl, 31);
    const int excl = incl - c;
    for (int base = 0; base < total; base += 32) {
        const int k = base + lane;
        int owner = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int v = __shfl_sync(full, incl, owner + st - 1);
            if (v <= k) owner += st;
        }
        const int q = k - __shfl_sync(full, excl, owner);
        const int ocols = __shfl_sync(full, cols, owner);
        const uint64_t oinv = __shfl_sync(full, inv, owner);
        const int owa = __shfl_sync(full, wa, owner);
        const int oty0 = __shfl_sync(full, valid ? f.ty0 : 0, owner);
        const int oa0 = __shfl_sync(full, valid ? f.a0 : 0, owner);
        const int ob0 = __shfl_sync(full, valid ? f.b0 : 0, owner);
        const bool active = k < total;
        int tile = 0;
        if (active) {
            // q / ocols without a division: q * ceil(2^32 / ocols) / 2^32 exceeds q / ocols by
            // less than q / 2^32 < 1, so it is the quotient or one above it
            int row = (int)(((uint64_t)(uint32_t)q * oinv) >> 32);
            if (row * ocols > q) --row;
            const int cc = q - row * ocols;
            const int tx = cc < owa ? oa0 + cc : ob0 + (cc - owa);
            tile = (oty0 + row) * TW + tx;
        }
        fn(tile, owner, active);
    }
}

// Pairs per tile, and with bcnt also per (block, tile) (bcnt[block * T + t], for emit to skip its
// own counting pass; only when the counts are kept in shared memory, T <= kSmemTiles).  The last
// block to finish turns the counts into bucket offsets:
// cursor[t] = start of tile t, tile_ranges[t] = [start, end) ([0, 0) when the bucket is
// empty or does not fit below cap), n_pairs = total (saturated at 2^32-1), GSPARC_ERR_CAPACITY if the
// total exceeds cap, and the sort's extra slices (none unless slice_big): extra[t] = the first extra
// slice of tile t (an exclusive scan of extra_slices over the tile ranges), extra[T] = their number.
__global__ void __launch_bounds__(kBinThreads) k_tile_count(int N, int H, int W, int TW, int T,
                                                            const float4* __restrict__ proj,
                                                            uint32_t* __restrict__ cnt,
                                                            uint32_t* __restrict__ bcnt,
                                                            uint32_t* __restrict__ cursor,
                                                            uint32_t* __restrict__ done, uint32_t cap,
                                                            uint2* __restrict__ ranges,
                                                            uint32_t* __restrict__ n_pairs,
                                                            uint32_t* __restrict__ extra, int slice_big,
                                                            int32_t* status) {
    __shared__ uint32_t s_cnt[kSmemTiles];
    __shared__ uint32_t s_warp[kBinThreads / 32];
    __shared__ uint64_t s_carry;
    __shared__ bool s_last;
    grid_dep_wait();
    const bool local = T <= kSmemTiles;
    if (local) {
        for (int t = threadIdx.x; t < T; t += kBinThreads) s_cnt[t] = 0;
        __syncthreads();
    }
    const int i = blockIdx.x * kBinThreads + threadIdx.x;
    Foot f;
    const bool valid = i < N && footprint(proj[2 * i], H, W, TW, f);
    warp_pairs(valid, f, TW, [&](int t, int, bool active) {
        if (active) atomicAdd(local ? &s_cnt[t] : &cnt[t], 1u);
    });
    if (local) {
        __syncthreads();
        uint32_t* mine = bcnt ? bcnt + (size_t)blockIdx.x * T : nullptr;
        for (int t = threadIdx.x; t < T; t += kBinThreads) {
            const uint32_t c = s_cnt[t];
            if (c) atomicAdd(&cnt[t], c);
            if (mine) mine[t] = c;
        }
    }
    grid_dep_launch();   // the emit pass may become resident while the last block scans
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < T; base += kBinThreads) {
        const int t = base + threadIdx.x;
        const uint32_t v = t < T ? __ldcg(&cnt[t]) : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint64_t before = s_carry;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        const uint64_t start = before + x - v, end = start + v;
        if (t < T) {
            const bool fits = v > 0 && end <= cap;
            const uint32_t s0 = (uint32_t)(start < cap ? start : cap);
            ranges[t] = fits ? make_uint2((uint32_t)start, (uint32_t)end) : make_uint2(0u, 0u);
            cursor[t] = s0;
        }
        __syncthreads();
        if (threadIdx.x == kBinThreads - 1) s_carry = end;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint64_t tot = s_carry;
        n_pairs[0] = (uint32_t)(tot > 0xffffffffull ? 0xffffffffull : tot);
        if (tot > cap) set_status(status, GSPARC_ERR_CAPACITY);
        s_carry = 0;
    }
    __syncthreads();
    // the extra slices of buckets above kSortCap keys (ranges written above by this thread)
    for (int base = 0; base < T; base += kBinThreads) {
        const int t = base + threadIdx.x;
        uint32_t v = 0;
        if (t < T) {
            const uint2 rg = ranges[t];
            v = slice_big ? extra_slices(rg.y - rg.x) : 0u;
        }
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint64_t before = s_carry;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        if (t < T) extra[t] = (uint32_t)(before + x - v);
        const uint64_t end = before + x;
        __syncthreads();
        if (threadIdx.x == kBinThreads - 1) s_carry = end;
        __syncthreads();
    }
    if (threadIdx.x == 0) extra[T] = (uint32_t)s_carry;
}

// Every pair's key (bits(r) << 32) | index into its tile's bucket.  A block reserves one
// run of each bucket with a single atomic per touched tile and fills it through shared
// counters; the block's count per tile comes from k_tile_count (bcnt) or, without it, from a
// counting pass of its own.  Positions at or above cap are dropped (their tiles have empty
// ranges).
__global__ void __launch_bounds__(kBinThreads) k_tile_emit(int N, int H, int W, int TW, int T,
                                                           const float4* __restrict__ proj,
                                                           const uint32_t* __restrict__ bcnt,
                                                           uint32_t* __restrict__ cursor, uint32_t cap,
                                                           uint64_t* __restrict__ keys) {
    __shared__ uint32_t s_cnt[kSmemTiles];
    __shared__ uint32_t s_base[kSmemTiles];
    const bool local = T <= kSmemTiles;
    const int i = blockIdx.x * kBinThreads + threadIdx.x;
    Foot f;
    const bool valid = i < N && footprint(proj[2 * i], H, W, TW, f);
    const uint64_t key = valid ? ((uint64_t)__float_as_uint(proj[2 * i + 1].w) << 32) | (uint32_t)i : 0;
    // the footprints above read only the projection, complete before k_tile_count began; the
    // counts, offsets and buckets below come from k_tile_count
    grid_dep_wait();
    if (!local) {
        warp_pairs(valid, f, TW, [&](int t, int owner, bool active) {
            const uint64_t k = __shfl_sync(0xffffffffu, key, owner);
            if (active) {
                const uint32_t pos = atomicAdd(&cursor[t], 1u);
                if (pos < cap) keys[pos] = k;
            }
        });
        return;
    }
    if (bcnt) {
        const uint32_t* mine = bcnt + (size_t)blockIdx.x * T;
        for (int t = threadIdx.x; t < T; t += kBinThreads) {
            const uint32_t c = mine[t];
            if (c) s_base[t] = atomicAdd(&cursor[t], c);
            s_cnt[t] = 0;
        }
    } else {
        for (int t = threadIdx.x; t < T; t += kBinThreads) s_cnt[t] = 0;
        __syncthreads();
        warp_pairs(valid, f, TW, [&](int t, int, bool active) {
            if (active) atomicAdd(&s_cnt[t], 1u);
        });
        __syncthreads();
        for (int t = threadIdx.x; t < T; t += kBinThreads) {
            const uint32_t c = s_cnt[t];
            if (c) {
                s_base[t] = atomicAdd(&cursor[t], c);
                s_cnt[t] = 0;
            }
        }
    }
    __syncthreads();
    warp_pairs(valid, f, TW, [&](int t, int owner, bool active) {
        const uint64_t k = __shfl_sync(0xffffffffu, key, owner);
        if (active) {
            const uint32_t pos = s_base[t] + atomicAdd(&s_cnt[t], 1u);
            if (pos < cap) keys[pos] = k;
        }
    });
}

struct SortShared {
    uint32_t hist[kSortWarps * 256];   // radix: [warp][digit] counts; distribution: sub-bucket offsets
    uint32_t warp_sum[kSortWarps];
    unsigned long long or_all, and_all;
    uint32_t dmin, dmax, maxb;
};

// Block-wide exclusive scan of one value per thread (kSortThreads threads).
__device__ __forceinline__ uint32_t sort_block_scan(uint32_t v, uint32_t* warp_sum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];
    __syncthreads();
    return before + x - v;
}

// Lanes of the warp whose 8-bit digit equals this lane's (d == 256 marks a lane without an
// element; such lanes match only each other): one ballot per digit bit.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bal : ~bal;
    }
    return peers;
}

// One stable LSD pass over the 8-bit digit at `shift`: src[0, n) -> dst[0, n).  Warp w
// owns the contiguous chunk [w*C, (w+1)*C) (C a multiple of 32) and walks it in rows of
// 32, ranking equal digits within a row by ballots.  The per-warp histograms are stored
// warp-major (lanes of a warp touch banks by digit) and scanned digit by digit across
// warps, then over digits, which gives every (digit, warp) run its place.
__device__ __forceinline__ void lsd_pass(const uint64_t* src, uint64_t* dst, int n, int shift,
                                         SortShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int C = ((n + kSortThreads - 1) / kSortThreads) * 32;
    const int lo = warp * C, hi = min(n, lo + C);
    uint32_t* wh = sh.hist + warp * 256;
    for (int e = threadIdx.x; e < 256 * kSortWarps; e += kSortThreads) sh.hist[e] = 0;
    __syncthreads();
    for (int idx = lo + lane; idx < hi; idx += 32) atomicAdd(&wh[(uint32_t)(src[idx] >> shift) & 0xffu], 1u);
    __syncthreads();
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
        if (d < 256) {
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = sh.hist[w * 256 + d];
                sh.hist[w * 256 + d] = run;
                run += c;
            }
        }
        const uint32_t off = sort_block_scan(run, sh.warp_sum);
        if (d < 256) {
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) sh.hist[w * 256 + d] += off;
        }
    }
    __syncthreads();
    for (int row = lo; row < hi; row += 32) {
        const int idx = row + lane;
        const uint64_t k = idx < hi ? src[idx] : 0ull;
        const uint32_t d = idx < hi ? (uint32_t)(k >> shift) & 0xffu : 256u;
        const uint32_t peers = digit_peers(d);
        uint32_t base = 0;
        if (d < 256) base = wh[d];
        __syncwarp();
        if (d < 256) {
            dst[base + __popc(peers & lt)] = k;
            if ((peers & lt) == 0) wh[d] = base + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
}

// Sort keys[0, n) (ping-pong with alt) over the bytes that vary; returns the buffer that
// holds the result.
__device__ __forceinline__ uint64_t* sort_bucket(uint64_t* a, uint64_t* b, int n, SortShared& sh) {
    unsigned long long o = 0, z = ~0ull;
    for (int j = threadIdx.x; j < n; j += kSortThreads) {
        o |= a[j];
        z &= a[j];
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, s);
        z &= __shfl_xor_sync(0xffffffffu, z, s);
    }
    if (threadIdx.x == 0) {
        sh.or_all = 0;
        sh.and_all = ~0ull;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicOr(&sh.or_all, o);
        atomicAnd(&sh.and_all, z);
    }
    __syncthreads();
    const uint64_t vary = sh.or_all ^ sh.and_all;
    __syncthreads();
    for (int byte = 0; byte < 8; ++byte) {
        if (((vary >> (8 * byte)) & 0xffu) == 0) continue;
        lsd_pass(a, b, n, 8 * byte, sh);
        uint64_t* t = a;
        a = b;
        b = t;
    }
    return a;
}

// Sub-buckets of a tile's distribution sort over its depth range [dmin, dmax] (float bits of r).
// When every depth is a finite non-negative float (bits below those of +inf), the sub-bucket is
// linear in r: (r - r_min) * nsub / (r_max - r_min).  Otherwise (or when that scale would not
// be finite) it is linear in the bits, (bits - dmin) * nsub / (dmax - dmin + 1).  Receiver
// distances in a volume have a density that grows with r, so a map linear in r (rather than in
// the bits, i.e. nearly in log r) keeps the sub-buckets of the far end small.
struct SubMap {
    uint32_t dmin;
    float rmin, scale;
    bool lin;
};

__device__ __forceinline__ SubMap sub_map(uint32_t dmin, uint32_t dmax, int nsub) {
    SubMap m;
    m.dmin = dmin;
    m.rmin = __uint_as_float(dmin);
    m.lin = false;
    if (dmax < 0x7f800000u) {
        const float range = __fsub_rn(__uint_as_float(dmax), m.rmin);
        const float sc = (float)nsub / range;
        if (range > 0.f && sc < 1e30f) {
            m.scale = sc;
            m.lin = true;
            return m;
        }
    }
    m.scale = (float)nsub / ((float)(dmax - dmin) + 1.0f);
    return m;
}

// Every step (offset, conversion, multiplication, clamp, truncation) is monotone
// non-decreasing, so a key never lands in an earlier sub-bucket than a smaller key; the clamp
// keeps the truncated value in [0, nsub - 1].
__device__ __forceinline__ int sub_bucket(uint64_t k, const SubMap& m, int nsub = kSubBuckets) {
    const uint32_t d = (uint32_t)(k >> 32);
    const float x = m.lin ? __fmul_rn(__fsub_rn(__uint_as_float(d), m.rmin), m.scale)
                          : __fmul_rn(__uint2float_rz(d - m.dmin), m.scale);
    return __float2int_rz(fminf(x, (float)(nsub - 1)));
}

// The distribution sort of a bucket above kSortCap keys: the same steps as the in-tile sort,
// with kSubBig sub-buckets counted in shared memory (hist, the block's key buffer) and the keys
// scattered into their sub-buckets in global memory (alt); each key's place is its sub-bucket's
// start plus the number of smaller keys there.  Returns false, having written nothing, when a
// sub-bucket holds more than kSubMaxBig keys (then the radix sort takes the bucket).
__device__ __forceinline__ bool sort_big_bucket(const uint64_t* src, uint64_t* alt, int n, uint32_t base,
                                                int tile, SortShared& sh, uint32_t* hist, uint32_t* sorted_ids,
                                                uint64_t* sorted_keys) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        sh.dmin = 0xffffffffu;
        sh.dmax = 0u;
        sh.maxb = 0u;
    }
    for (int e = threadIdx.x; e < kSubBig; e += kSortThreads) hist[e] = 0;
    __syncthreads();
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int j = threadIdx.x; j < n; j += kSortThreads) {
        const uint32_t d = (uint32_t)(src[j] >> 32);
        lo = min(lo, d);
        hi = max(hi, d);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
        atomicMin(&sh.dmin, lo);
        atomicMax(&sh.dmax, hi);
    }
    __syncthreads();
    const SubMap sm = sub_map(sh.dmin, sh.dmax, kSubBig);
    for (int j = threadIdx.x; j < n; j += kSortThreads) atomicAdd(&hist[sub_bucket(src[j], sm, kSubBig)], 1u);
    __syncthreads();
    {
        constexpr int kPer = kSubBig / kSortThreads;
        uint32_t sum = 0, mx = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t c = hist[threadIdx.x * kPer + q];
            sum += c;
            mx = max(mx, c);
        }
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) atomicMax(&sh.maxb, mx);
        uint32_t off = sort_block_scan(sum, sh.warp_sum);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t c = hist[threadIdx.x * kPer + q];
            hist[threadIdx.x * kPer + q] = off;
            off += c;
        }
    }
    __syncthreads();
    if (sh.maxb > (uint32_t)kSubMaxBig) {
        __syncthreads();
        return false;
    }
    for (int j = threadIdx.x; j < n; j += kSortThreads) {
        const uint64_t k = src[j];
        alt[atomicAdd(&hist[sub_bucket(k, sm, kSubBig)], 1u)] = k;
    }
    __syncthreads();
    // hist[b] is now the end of sub-bucket b (= the start of b + 1)
    for (int p = threadIdx.x; p < n; p += kSortThreads) {
        const uint64_t k = alt[p];
        const int b = sub_bucket(k, sm, kSubBig);
        const int s0 = b > 0 ? (int)hist[b - 1] : 0, e0 = (int)hist[b];
        int rank = 0;
        for (int q = s0; q < e0; ++q) rank += alt[q] < k;
        const uint32_t dst = base + (uint32_t)(s0 + rank);
        sorted_ids[dst] = (uint32_t)k;
        if (sorted_keys) sorted_keys[dst] = ((uint64_t)tile << 32) | (k >> 32);
    }
    __syncthreads();
    return true;
}

// fn(key) over the keys src[0, n), four loads in flight per thread.
template <class F>
__device__ __forceinline__ void for_keys4(const uint64_t* src, int n, F&& fn) {
    for (int j0 = threadIdx.x; j0 < n; j0 += 4 * kSortThreads) {
        uint64_t k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * kSortThreads;
            k[u] = j < n ? __ldcg(src + j) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (j0 + u * kSortThreads < n) fn(k[u]);
    }
}

// Slice c of a bucket of n > kSortCap keys (src, its first list position base): the keys are
// counted into kSubBig depth sub-buckets (hist, in the block's key buffer; the map over the
// bucket's depth range, the same in every slice), the counts scanned, and the slice is the run
// of sub-buckets whose starts fall in [c n / P, (c + 1) n / P) for P slices.  Its keys are
// gathered into shared memory (buf) by sub-bucket and each is placed at its sub-bucket's start
// plus the number of smaller keys there.  Returns false, having written nothing, when a
// sub-bucket holds more than kSubMaxBig keys (then slice 0 takes the radix sort and the others
// nothing).
__device__ __forceinline__ bool sort_slice(const uint64_t* src, int n, uint32_t c, uint32_t base, int tile,
                                           SortShared& sh, uint32_t* hist, uint64_t* buf, uint32_t* sorted_ids,
                                           uint64_t* sorted_keys) {
    const int lane = threadIdx.x & 31;
    const uint32_t P = extra_slices((uint32_t)n) + 1u;
    if (threadIdx.x == 0) {
        sh.dmin = 0xffffffffu;
        sh.dmax = 0u;
        sh.maxb = 0u;
    }
    for (int e = threadIdx.x; e < kSubBig; e += kSortThreads) hist[e] = 0;
    __syncthreads();
    uint32_t lo = 0xffffffffu, hi = 0u;
    for_keys4(src, n, [&](uint64_t k) {
        const uint32_t d = (uint32_t)(k >> 32);
        lo = min(lo, d);
        hi = max(hi, d);
    });
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
        atomicMin(&sh.dmin, lo);
        atomicMax(&sh.dmax, hi);
    }
    __syncthreads();
    const SubMap sm = sub_map(sh.dmin, sh.dmax, kSubBig);
    for_keys4(src, n, [&](uint64_t k) { atomicAdd(&hist[sub_bucket(k, sm, kSubBig)], 1u); });
    __syncthreads();
    constexpr int kPer = kSubBig / kSortThreads;
    {
        uint32_t sum = 0, mx = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t v = hist[threadIdx.x * kPer + q];
            sum += v;
            mx = max(mx, v);
        }
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) atomicMax(&sh.maxb, mx);
        uint32_t off = sort_block_scan(sum, sh.warp_sum);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t v = hist[threadIdx.x * kPer + q];
            hist[threadIdx.x * kPer + q] = off;   // the start of the sub-bucket
            off += v;
        }
    }
    if (threadIdx.x == 0) {
        sh.dmin = (uint32_t)kSubBig;   // first sub-bucket of the slice
        sh.dmax = (uint32_t)kSubBig;   // first sub-bucket of the next slice
    }
    __syncthreads();
    if (sh.maxb > (uint32_t)kSubMaxBig) {
        __syncthreads();
        return false;
    }
    // sub-bucket b opens slice s when its start times P first reaches s n (empty sub-buckets
    // hold no keys, so which slice they fall in does not matter)
    {
        const uint64_t t0 = (uint64_t)c * (uint32_t)n, t1 = (uint64_t)(c + 1) * (uint32_t)n;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int b = threadIdx.x * kPer + q;
            const uint64_t st = (uint64_t)hist[b] * P;
            const uint64_t pv = b > 0 ? (uint64_t)hist[b - 1] * P : 0ull;
            if (st >= t0 && (b == 0 || pv < t0)) sh.dmin = (uint32_t)b;
            if (st >= t1 && (b == 0 || pv < t1)) sh.dmax = (uint32_t)b;
        }
    }
    __syncthreads();
    const int b_lo = (int)sh.dmin, b_hi = (int)sh.dmax;
    const uint32_t s_lo = b_lo < kSubBig ? hist[b_lo] : (uint32_t)n;
    const uint32_t s_hi = b_hi < kSubBig ? hist[b_hi] : (uint32_t)n;
    const int m = (int)(s_hi - s_lo);   // <= n / P + kSubMaxBig
    __syncthreads();   // every thread has read the slice's starts before the gather moves them
    for_keys4(src, n, [&](uint64_t k) {
        const int b = sub_bucket(k, sm, kSubBig);
        if (b >= b_lo && b < b_hi) buf[atomicAdd(&hist[b], 1u) - s_lo] = k;
    });
    __syncthreads();
    // hist[b] is now the end of sub-bucket b (= the start of b + 1) inside the slice
    for (int p = threadIdx.x; p < m; p += kSortThreads) {
        const uint64_t k = buf[p];
        const int b = sub_bucket(k, sm, kSubBig);
        const int s0 = (b > b_lo ? (int)hist[b - 1] : (int)s_lo) - (int)s_lo;
        const int e0 = (int)hist[b] - (int)s_lo;
        int rank = 0;
        for (int q = s0; q < e0; ++q) rank += buf[q] < k;
        const uint32_t dst = base + s_lo + (uint32_t)(s0 + rank);
        sorted_ids[dst] = (uint32_t)k;
        if (sorted_keys) sorted_keys[dst] = ((uint64_t)tile << 32) | (k >> 32);
    }
    __syncthreads();
    return true;
}

// Item tile < T of k_tile_sort: the tile's bucket.
__device__ __forceinline__ void sort_tile(int tile, const uint2* __restrict__ ranges, const uint32_t* __restrict__ extra,
                                          uint64_t* __restrict__ keys, uint64_t* __restrict__ alt,
                                          uint32_t* __restrict__ sorted_ids, uint64_t* __restrict__ sorted_keys,
                                          SortShared& sh, uint64_t* buf) {
    const int lane = threadIdx.x & 31;
    {
        const uint2 r = ranges[tile];
        const int n = (int)(r.y - r.x);
        if (n <= 0) return;
        const uint64_t* src = keys + r.x;
        if (n > kSortCap) {
            // the slice's keys in the front of the buffer, the kSubBig counters behind them
            static_assert((size_t)(kSlice + kSubMaxBig) * 8 + kSubBig * 4 <= (size_t)kSortCap * 8,
                          "slice keys and large-bucket histogram in the key buffer");
            uint32_t* hist = reinterpret_cast<uint32_t*>(buf + kSlice + kSubMaxBig);
            const bool sliced = __ldg(&extra[tile + 1]) > __ldg(&extra[tile]);
            if (sliced ? sort_slice(src, n, 0u, r.x, tile, sh, hist, buf, sorted_ids, sorted_keys)
                       : sort_big_bucket(src, alt + r.x, n, r.x, tile, sh, reinterpret_cast<uint32_t*>(buf),
                                         sorted_ids, sorted_keys))
                return;
            const uint64_t* res = sort_bucket(keys + r.x, alt + r.x, n, sh);
            for (int j = threadIdx.x; j < n; j += kSortThreads) {
                const uint64_t k = res[j];
                sorted_ids[r.x + j] = (uint32_t)k;
                if (sorted_keys) sorted_keys[r.x + j] = ((uint64_t)tile << 32) | (k >> 32);
            }
            return;
        }
        bool radix = false;
        {
            if (threadIdx.x == 0) {
                sh.dmin = 0xffffffffu;
                sh.dmax = 0u;
                sh.maxb = 0u;
            }
            for (int e = threadIdx.x; e < kSubBuckets; e += kSortThreads) sh.hist[e] = 0;
            __syncthreads();
            uint32_t lo = 0xffffffffu, hi = 0u;
            for (int j = threadIdx.x; j < n; j += kSortThreads) {
                const uint32_t d = (uint32_t)(src[j] >> 32);
                lo = min(lo, d);
                hi = max(hi, d);
            }
            lo = __reduce_min_sync(0xffffffffu, lo);
            hi = __reduce_max_sync(0xffffffffu, hi);
            if (lane == 0) {
                atomicMin(&sh.dmin, lo);
                atomicMax(&sh.dmax, hi);
            }
            __syncthreads();
            const SubMap sm = sub_map(sh.dmin, sh.dmax, kSubBuckets);
            for (int j = threadIdx.x; j < n; j += kSortThreads)
                atomicAdd(&sh.hist[sub_bucket(src[j], sm)], 1u);
            __syncthreads();
            {
                constexpr int kPer = kSubBuckets / kSortThreads;
                uint32_t c[kPer], sum = 0, mx = 0;
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    c[q] = sh.hist[threadIdx.x * kPer + q];
                    sum += c[q];
                    mx = max(mx, c[q]);
                }
                mx = __reduce_max_sync(0xffffffffu, mx);
                if (lane == 0) atomicMax(&sh.maxb, mx);
                uint32_t off = sort_block_scan(sum, sh.warp_sum);
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    sh.hist[threadIdx.x * kPer + q] = off;
                    off += c[q];
                }
            }
            __syncthreads();
            radix = sh.maxb > (uint32_t)kSubMax;
            if (!radix) {
                for (int j = threadIdx.x; j < n; j += kSortThreads) {
                    const uint64_t k = src[j];
                    buf[atomicAdd(&sh.hist[sub_bucket(k, sm)], 1u)] = k;
                }
                __syncthreads();
                // hist[b] is now the end of sub-bucket b (= the start of b + 1)
                for (int p = threadIdx.x; p < n; p += kSortThreads) {
                    const uint64_t k = buf[p];
                    const int b = sub_bucket(k, sm);
                    const int s0 = b > 0 ? (int)sh.hist[b - 1] : 0, e0 = (int)sh.hist[b];
                    int rank = 0;
                    for (int q = s0; q < e0; ++q) rank += buf[q] < k;
                    const uint32_t dst = r.x + (uint32_t)(s0 + rank);
                    sorted_ids[dst] = (uint32_t)k;
                    if (sorted_keys) sorted_keys[dst] = ((uint64_t)tile << 32) | (k >> 32);
                }
            }
            __syncthreads();
        }
        if (radix) {
            const uint64_t* res = sort_bucket(keys + r.x, alt + r.x, n, sh);
            for (int j = threadIdx.x; j < n; j += kSortThreads) {
                const uint64_t k = res[j];
                sorted_ids[r.x + j] = (uint32_t)k;
                if (sorted_keys) sorted_keys[r.x + j] = ((uint64_t)tile << 32) | (k >> 32);
            }
        }
    }
}

// Persistent blocks that take work items from a counter (work[0], zero-initialised): item t < T
// sorts tile t's bucket, up to kSortCap keys by distribution (keys counted into kSubBuckets
// sub-buckets by depth, scattered to their sub-bucket in shared memory in arbitrary order inside
// it, each key's final place its sub-bucket's start plus the number of smaller keys in the same
// sub-bucket; the keys are unique, so the places are distinct); above kSortCap keys slice 0 of the
// bucket (sort_slice) when the bucket is sliced, else the whole bucket with its keys scattered in
// global memory (sort_big_bucket).  Items T + e are the extra slices e of the work list of
// k_tile_count.  A bucket whose largest sub-bucket is too large (many equal depths) takes the LSD
// radix sort in global memory with `alt` as the second buffer (its tile's item; its extra slices
// are skipped).
__global__ void __launch_bounds__(kSortThreads, 1) k_tile_sort(int T, const uint2* __restrict__ ranges,
                                                               const uint32_t* __restrict__ extra,
                                                               uint32_t* __restrict__ work,
                                                               uint64_t* __restrict__ keys,
                                                               uint64_t* __restrict__ alt,
                                                               uint32_t* __restrict__ sorted_ids,
                                                               uint64_t* __restrict__ sorted_keys) {
    GSPARC_DYNAMIC_SMEM(smem_raw);
    SortShared& sh = *reinterpret_cast<SortShared*>(smem_raw);
    uint64_t* buf = reinterpret_cast<uint64_t*>(smem_raw + ((sizeof(SortShared) + 15) & ~size_t(15)));
    __shared__ uint32_t s_item;
    grid_dep_wait();
    const uint32_t n_items = (uint32_t)T + __ldg(&extra[T]);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();   // every thread has its item before thread 0 takes the next
        if (item >= n_items) return;   // the whole block
        if (item < (uint32_t)T) {
            sort_tile((int)item, ranges, extra, keys, alt, sorted_ids, sorted_keys, sh, buf);
        } else {
            const uint32_t e = item - (uint32_t)T;
            // the tile: the last t with extra[t] <= e (tiles without extra slices repeat the next offset)
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&extra[mid]) <= e) lo = mid;
                else hi = mid - 1;
            }
            const uint2 r = ranges[lo];
            uint32_t* hist = reinterpret_cast<uint32_t*>(buf + kSlice + kSubMaxBig);
            sort_slice(keys + r.x, (int)(r.y - r.x), 1u + e - __ldg(&extra[lo]), r.x, lo, sh, hist, buf, sorted_ids,
                       sorted_keys);
        }
        __syncthreads();   // the next item reuses the shared memory
    }
}

constexpr size_t kSortSmem = ((sizeof(SortShared) + 15) & ~size_t(15)) + kSortCap * sizeof(uint64_t);
static_assert(kSubBig * sizeof(uint32_t) <= kSortCap * sizeof(uint64_t), "large-bucket histogram in the key buffer");
static_assert(kSubBig % kSortThreads == 0, "histogram scan: a whole number of entries per thread");
static_assert(kSortSmem <= 232448, "tile sort shared memory above the per-block limit");

}  // namespace
}  // namespace gsparc
