// Tile binning and directional sorting: workspace layout, launch sequence and entry points
// (kernels in binsort.cuh).

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "internal.cuh"
#include "binsort.cuh"

namespace gsparc {
namespace {

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// bcnt (the per-block tile counts that spare k_tile_emit its counting pass) is laid out when the
// counts are kept in shared memory (ntiles <= kSmemTiles) and with_bcnt is set; bcnt == 0 then
// means "not laid out".
struct Layout {
    size_t cnt, cursor, done, keys, alt, extra, bcnt, total;
    int nblk;
};

Layout layout(int N, int64_t cap, int ntiles, bool with_bcnt = true) {
    Layout L;
    L.nblk = (N + kBinThreads - 1) / kBinThreads;
    size_t o = 0;
    L.cnt = o;    o += align256((size_t)ntiles * 4);
    L.done = o;   o += align256(16);
    L.cursor = o; o += align256((size_t)ntiles * 4);
    L.keys = o;   o += align256((size_t)cap * 8);
    L.alt = o;    o += align256((size_t)cap * 8);
    L.extra = o;  o += align256((size_t)(ntiles + 1) * 4);
    L.bcnt = 0;
    if (with_bcnt && ntiles <= kSmemTiles && N > 0) {
        L.bcnt = o;
        o += align256((size_t)L.nblk * (size_t)ntiles * 4);
    }
    L.total = o;
    return L;
}

// The launch sequence shared by both entry points.  `w` is a workspace laid out by layout().
int bin_sort_launch(const gsparc_view* view, int N, const float* proj, int64_t pair_capacity, char* w,
                    const Layout& L, uint32_t* sorted_ids, uint64_t* sorted_keys, uint32_t* tile_ranges,
                    uint32_t* n_pairs, int32_t* d_status, cudaStream_t s) {
    const int TW = tiles_x(*view), TH = tiles_y(*view), T = TW * TH;
    uint32_t* cnt = reinterpret_cast<uint32_t*>(w + L.cnt);
    uint32_t* done = reinterpret_cast<uint32_t*>(w + L.done);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(w + L.cursor);
    uint64_t* keys = reinterpret_cast<uint64_t*>(w + L.keys);
    uint64_t* alt = reinterpret_cast<uint64_t*>(w + L.alt);
    uint32_t* extra = reinterpret_cast<uint32_t*>(w + L.extra);
    uint32_t* bcnt = L.bcnt ? reinterpret_cast<uint32_t*>(w + L.bcnt) : nullptr;
    const uint32_t cap = (uint32_t)pair_capacity;
    if (N == 0) {
        if (cudaMemsetAsync(tile_ranges, 0, (size_t)T * 2 * sizeof(uint32_t), s) != cudaSuccess)
            return GSPARC_ERR_CUDA;
        if (cudaMemsetAsync(n_pairs, 0, sizeof(uint32_t), s) != cudaSuccess) return GSPARC_ERR_CUDA;
        return GSPARC_OK;
    }
    // tile counters, the block ticket and the sort's work counter are contiguous
    if (cudaMemsetAsync(w + L.cnt, 0, L.cursor - L.cnt, s) != cudaSuccess) return GSPARC_ERR_CUDA;
    if (!ensure_smem_attr(k_tile_sort, (int)kSortSmem)) return GSPARC_ERR_CUDA;
    const float4* p4 = reinterpret_cast<const float4*>(proj);
    uint2* ranges = reinterpret_cast<uint2*>(tile_ranges);
    k_tile_count<<<L.nblk, kBinThreads, 0, s>>>(N, view->H, view->W, TW, T, p4, cnt, bcnt, cursor, done, cap,
                                                ranges, n_pairs, extra, slice_big_buckets(T, num_sms()) ? 1 : 0,
                                                d_status);
    if (launch_status() != GSPARC_OK) return GSPARC_ERR_CUDA;
    if (launch_after(GSPARC_OVERLAP_BIN_SORT, k_tile_emit, dim3(L.nblk), dim3(kBinThreads), 0, s, N, view->H, view->W, TW, T, p4, bcnt,
                     cursor, cap, keys) != GSPARC_OK)
        return GSPARC_ERR_CUDA;
    return launch_after(GSPARC_OVERLAP_BIN_SORT, k_tile_sort, dim3(sort_grid(T, cap, num_sms())), dim3(kSortThreads), kSortSmem, s, T,
                        ranges, extra, done + 1, keys, alt, sorted_ids, sorted_keys);
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
    const int T = tiles_x(*view) * tiles_y(*view);
    const Layout L = layout(N, pair_capacity, T);
    if (!ws || ws_bytes < L.total) return GSPARC_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return GSPARC_ERR_INVALID;
    return bin_sort_launch(view, N, proj, pair_capacity, static_cast<char*>(ws), L, sorted_ids,
                           sorted_keys, tile_ranges, n_pairs, d_status, as_stream(stream));
}

// ---------------------------------------------------------------------------------------------
// Scratch-free variant for callers that cannot allocate device memory (a real-time loop that
// must not pay cudaMalloc's device-wide synchronisation after start-up, a plugin given buffers
// but no allocator).  Same kernels and launch sequence as gsparc_bin_sort; the scratch lives in
// one file-scope device array instead of a caller workspace.
// ---------------------------------------------------------------------------------------------

namespace gsparc {
namespace {

// covers layout(N, GSPARC_NOALLOC_MAX_PAIRS, T) for up to 65536 tiles
constexpr size_t kNoAllocBytes = size_t(9) << 20;
static_assert(size_t(GSPARC_NOALLOC_MAX_PAIRS) * 16 + 65536 * 12 + 8192 <= kNoAllocBytes,
              "no-alloc scratch below the documented limits");
constexpr int kMaxDevices = 64;

// Host code must not use this symbol as an address: it only names the array.  The device
// address comes from cudaGetSymbolAddress, once per device, with that device current.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array per device, stored only once a lookup succeeded: a failed lookup
// (an earlier asynchronous error reported by the runtime call, or a lookup inside a stream
// capture) is retried by the next call instead of being kept for the life of the process.
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices];

void* noalloc_scratch(int dev) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            (void)cudaGetLastError();   // clear a non-sticky error so that a retry can succeed
            return nullptr;
        }
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

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
    const int T = tiles_x(*view) * tiles_y(*view);
    Layout L = layout(N, pair_capacity, T);
    if (L.total > kNoAllocBytes) L = layout(N, pair_capacity, T, false);   // emit counts for itself
    if (L.total > kNoAllocBytes) return GSPARC_ERR_TOO_LARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GSPARC_ERR_CUDA;
    char* scratch = static_cast<char*>(noalloc_scratch(dev));
    if (!scratch) return GSPARC_ERR_CUDA;
    // the array keeps the previous call's contents; bin_sort_launch clears the tile
    // counters and the block ticket, and everything else is written before it is read
    return bin_sort_launch(view, N, proj, pair_capacity, scratch, L,
                           sorted_ids, sorted_keys, tile_ranges, n_pairs, d_status, as_stream(stream));
}
