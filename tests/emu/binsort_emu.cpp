// Runs the library's binning and sorting kernels (csrc/binsort.cuh) under the host shim with the
// launch sequence of gsparc_bin_sort: tile counters and ticket zeroed, k_tile_count and
// k_tile_emit over blocks of kBinThreads records, k_tile_sort over sort_grid(T, capacity, 4)
// persistent blocks (as on a GPU of 4 SMs: the tiles and the extra slices of buckets above kSortCap
// keys taken from a work counter) with the kernel's dynamic shared memory.
// With with_bcnt (bit 0 of the fifth header word), k_tile_count also writes the per-(block, tile)
// counts and k_tile_emit takes them instead of counting for itself (the library's path when
// T <= kSmemTiles).  Bit 1 turns off the slicing of buckets above kSortCap keys (the library's
// choice when there are at least as many tiles as SMs): each is then sorted whole by its tile's
// block.
// Input: int32 N, H, W, capacity, flags; float proj[8N].  Output: uint32 n_pairs; int32
// status; uint32 tile_ranges[2T]; uint32 sorted_ids[capacity]; uint64 sorted_keys[capacity];
// int32 violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "binsort.cuh"

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t hdr[5];
    if (fread(hdr, 4, 5, f) != 5) return 2;
    const int N = hdr[0], H = hdr[1], W = hdr[2];
    const uint32_t cap = (uint32_t)hdr[3];
    std::vector<float4> proj(2 * (size_t)N);
    if (N && fread(proj.data(), 16, 2 * (size_t)N, f) != 2 * (size_t)N) return 2;
    fclose(f);
    const int TW = (W + 15) / 16, TH = (H + 15) / 16, T = TW * TH;
    std::vector<uint32_t> cnt(T, 0u), cursor(T, 0u), ids(cap, 0xffffffffu), done(4, 0u), extra(T + 1, 0xdeadbeefu);
    std::vector<uint2> ranges(T, uint2{0xffffffffu, 0xffffffffu});
    std::vector<uint64_t> keys(cap > 0 ? cap : 1), alt(cap > 0 ? cap : 1), skeys(cap, ~0ull);
    uint32_t n_pairs = 0xffffffffu;
    int32_t status = 0;
    if (N == 0) {
        for (auto& r : ranges) r = uint2{0u, 0u};
        n_pairs = 0;
    } else {
        using namespace gsparc;
        const unsigned nblk = (unsigned)((N + kBinThreads - 1) / kBinThreads);
        const bool with_bcnt = (hdr[4] & 1) != 0 && T <= kSmemTiles;
        // bit 1: sort large buckets whole (the library's choice when the tiles outnumber the SMs)
        const int slice_big = (hdr[4] & 2) ? 0 : 1;
        std::vector<uint32_t> bcnt(with_bcnt ? (size_t)nblk * T : 1, 0xdeadbeefu);   // written before read
        uint32_t* bc = with_bcnt ? bcnt.data() : nullptr;
        emu_launch(emu_dim3{nblk, 1, 1}, kBinThreads, k_tile_count, N, H, W, TW, T, (const float4*)proj.data(),
                   cnt.data(), bc, cursor.data(), done.data(), cap, ranges.data(), &n_pairs, extra.data(), slice_big, &status);
        emu_launch(emu_dim3{nblk, 1, 1}, kBinThreads, k_tile_emit, N, H, W, TW, T, (const float4*)proj.data(),
                   (const uint32_t*)bc, cursor.data(), cap, keys.data());
        emu_launch_smem(emu_dim3{sort_grid(T, cap, 4), 1, 1}, kSortThreads, kSortSmem, k_tile_sort, T,
                        (const uint2*)ranges.data(), (const uint32_t*)extra.data(), done.data() + 1, keys.data(), alt.data(), ids.data(),
                        skeys.data());
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(&n_pairs, 4, 1, o);
    fwrite(&status, 4, 1, o);
    fwrite(ranges.data(), 8, T, o);
    fwrite(ids.data(), 4, cap, o);
    fwrite(skeys.data(), 8, cap, o);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
