// Runs the tensor-core backward's schedule (csrc/bwd_schedule.cuh) under the host shim with the
// launch of gsparc_render_bwd_tc_balanced: one block per (transmitter, tile) taking the walks
// from n_contrib when no walks are given, else one block.
// Input: int32 H, W, B, strips, split_min, allow_split, have_walks; uint32 ranges[2T],
// n_contrib[B H W], walks_in[B T].  Output: uint32 hdr[4], walks[B T], items[4 * 2 B T strips];
// int32 shim violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "bwd_schedule.cuh"

template <typename T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

int main(int argc, char** argv) {
    using namespace gsparc;
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    auto hdr_in = rd<int32_t>(f, 7);
    const int H = hdr_in[0], W = hdr_in[1], B = hdr_in[2], strips = hdr_in[3], split_min = hdr_in[4],
              allow = hdr_in[5], have_walks = hdr_in[6];
    const int TW = (W + 15) / 16, T = TW * ((H + 15) / 16);
    auto ranges = rd<uint2>(f, T);
    auto nc = rd<uint32_t>(f, (size_t)B * H * W);
    auto walks_in = rd<uint32_t>(f, (size_t)B * T);
    fclose(f);
    std::vector<uint32_t> hdr(4, 0u), walks((size_t)B * T, 0xffffffffu);
    std::vector<uint4> items((size_t)2 * B * T * strips, uint4{~0u, ~0u, ~0u, ~0u});
    emu_launch(emu_dim3{have_walks ? 1u : (unsigned)(B * T), 1, 1}, kSchedThreads, k_bwd_schedule, H, W, TW, T, B * T,
               strips, split_min, allow, (const uint2*)ranges.data(), (const uint32_t*)nc.data(),
               (const uint32_t*)(have_walks ? walks_in.data() : nullptr), hdr.data(), walks.data(), items.data());
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(hdr.data(), 4, 4, o);
    fwrite(walks.data(), 4, walks.size(), o);
    fwrite(items.data(), 16, items.size(), o);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
