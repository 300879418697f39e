// Schedule of the tensor-core backward (k_bwd_schedule) and its workspace layout: device code
// with no runtime API, so that the same source also builds for the host under the test suite's
// shim.  The launch is in render.cu (gsparc_render_bwd_tc_balanced).

#pragma once

#include <stdint.h>

#include "device_common.cuh"

namespace gsparc {
namespace {

constexpr int kTbE = 16;   // entries per backward batch

// ---------------------------------------------------------------------------------------------
// Schedule of the tensor-core backward.  Its cost per (transmitter, tile, strip) is the walk,
// the largest n_contrib among the tile's pixels, in batches of kTbE entries, and it varies by
// a factor of two or more between tiles, so one block per tile leaves most SMs idle while the
// longest walks finish.  The schedule splits each long walk into a front chunk [0, m) and a
// back chunk [m, walk) that run as independent blocks: the back chunk starts from the final
// state as before, the front chunk from T = 1 with the suffix taken as s_tot minus the prefix
// sum (no state at m is needed).  The items are ordered by decreasing batch count; the block
// scheduler hands out blocks in index order, which makes this longest-first list scheduling.
// ---------------------------------------------------------------------------------------------

constexpr int kSchedThreads = 256;
constexpr int kSchedKeys = kSchedThreads;   // cost buckets (batches, clamped), one per thread
constexpr int kSplitMinDefault = 3;        // batches: a longer walk is split in two

struct SchedLayout {
    size_t hdr, walks, items, total;
};

inline SchedLayout sched_layout(int B, int T, int strips) {
    SchedLayout L;
    size_t o = 0;
    L.hdr = o;   o += 16;                                          // ticket, item count
    L.walks = o; o += ((size_t)B * T * 4 + 15) & ~size_t(15);
    L.items = o; o += (size_t)2 * B * T * strips * sizeof(uint4);
    L.total = o;
    return L;
}

inline int strips_of(int K) { return K <= 64 ? 1 : (K + 63) / 64; }

// Without walks_in: one block per (transmitter, tile) takes the walk from n_contrib, and the
// last block to finish builds the items.  With walks_in (written by the tensor-core forward):
// one block builds the items from them.  BT = transmitters x tiles.
__global__ void __launch_bounds__(kSchedThreads) k_bwd_schedule(int H, int W, int TW, int T, int BT, int strips,
                                                                int split_min, int allow_split,
                                                                const uint2* __restrict__ ranges,
                                                                const uint32_t* __restrict__ n_contrib,
                                                                const uint32_t* __restrict__ walks_in,
                                                                uint32_t* __restrict__ hdr,
                                                                uint32_t* __restrict__ walks,
                                                                uint4* __restrict__ items) {
    __shared__ uint32_t s_max;
    __shared__ uint32_t s_off[kSchedKeys];
    __shared__ uint32_t s_warp[kSchedThreads / 32];
    __shared__ bool s_last;
    grid_dep_wait();     // the forward's walks or n_contrib
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (!walks_in) {
        const int tile = (int)(blockIdx.x % (uint32_t)T), b = (int)(blockIdx.x / (uint32_t)T);
        if (tid == 0) s_max = 0u;
        __syncthreads();
        const int x = (tile % TW) * kTile + (tid & 15), y = (tile / TW) * kTile + (tid >> 4);
        uint32_t v = (x < W && y < H) ? n_contrib[(size_t)b * H * W + (size_t)y * W + x] : 0u;
        v = __reduce_max_sync(0xffffffffu, v);
        if (lane == 0) atomicMax(&s_max, v);
        __syncthreads();
        if (tid == 0) {
            const uint2 r = ranges[tile];
            walks[blockIdx.x] = min(s_max, r.y - r.x);
            __threadfence();
            s_last = atomicAdd(&hdr[0], 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
    }
    const uint32_t* wsrc = walks_in ? walks_in : walks;
    // batch counts of the one or two chunks of a walk (n1 = 0: not split)
    auto chunks = [&](uint32_t w, uint32_t& n0, uint32_t& n1) {
        const uint32_t nb = (w + kTbE - 1) / kTbE;
        if (allow_split && split_min >= 0 && nb > (uint32_t)split_min) {
            n0 = nb / 2;
            n1 = nb - n0;
        } else {
            n0 = nb;
            n1 = 0u;
        }
    };
    auto key = [](uint32_t n) { return (uint32_t)kSchedKeys - 1u - min(n, (uint32_t)kSchedKeys - 1u); };
    const int units = BT * strips;
    s_off[tid] = 0u;
    __syncthreads();
    for (int u = tid; u < units; u += kSchedThreads) {
        uint32_t n0, n1;
        chunks(__ldcg(&wsrc[u / strips]), n0, n1);
        if (n0) atomicAdd(&s_off[key(n0)], 1u);
        if (n1) atomicAdd(&s_off[key(n1)], 1u);
    }
    __syncthreads();
    // exclusive scan of the bucket counts: bucket 0 holds the longest items
    const uint32_t c = s_off[tid];
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y2 = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y2;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t before = 0u;
    for (int w2 = 0; w2 < warp; ++w2) before += s_warp[w2];
    s_off[tid] = before + incl - c;
    if (tid == kSchedThreads - 1) hdr[1] = before + incl;   // the item count
    __syncthreads();
    for (int u = tid; u < units; u += kSchedThreads) {
        const uint32_t bt = (uint32_t)(u / strips), strip = (uint32_t)(u % strips);
        const uint32_t w = __ldcg(&wsrc[bt]);
        uint32_t n0, n1;
        chunks(w, n0, n1);
        if (n1) {
            const uint32_t m = n0 * kTbE;
            items[atomicAdd(&s_off[key(n0)], 1u)] = make_uint4(bt, strip | 0x80000000u, 0u, m);
            items[atomicAdd(&s_off[key(n1)], 1u)] = make_uint4(bt, strip, m, w);
        } else if (n0) {
            items[atomicAdd(&s_off[key(n0)], 1u)] = make_uint4(bt, strip, 0u, w);
        }
    }
    if (tid == 0 && !walks_in) hdr[0] = 0u;   // every block has taken its ticket: reset for the next call
}

}  // namespace
}  // namespace gsparc
