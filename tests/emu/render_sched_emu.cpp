// Runs the library's FP32 training-step compositing under the host shim with the arguments and
// launch shapes of gsparc_render_fwd_l2 and gsparc_render_bwd_balanced: the forward with the
// complex L2 loss fused (dL/dz, loss, s_tot, tile walks), then k_bwd_schedule building the work
// items from the walks (split_min batches: every longer walk split into a front and a back
// chunk), then the backward over those items.
// Input: int32 H, W, K, N, B, n_ids, split_min; double f_c, df; float proj[8N]; uint32
// ranges[2T], ids[n_ids]; float attr[4BN], target[2BKHW].  Output: float loss, d_spectrum
// [2BKHW], s_tot[B strips HW], final_logT[BHW]; uint32 n_contrib[BHW], walks[BT], n_items,
// items[4 * n_items]; float d_attr[4BN], d_proj[8N]; int32 shim violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "render_common.cuh"
#include "bwd_schedule.cuh"

template <typename T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

template <int S>
static void fwd(const gsparc::RenderArgs& a, int T) {
    const emu_dim3 grid{(unsigned)((a.K + S - 1) / S), (unsigned)T, (unsigned)a.B};
    emu_launch_smem(grid, gsparc::kThreads, gsparc::F32Smem<S>::kTotal, gsparc::k_render_fwd<S>, a);
}
template <int S>
static void bwd(const gsparc::RenderArgs& a, unsigned items) {
    emu_launch_smem(emu_dim3{items, 1, 1}, gsparc::kThreads, gsparc::F32BwdSmem<S>::kTotal, gsparc::k_render_bwd<S>, a);
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    auto hdr = rd<int32_t>(f, 7);
    const int H = hdr[0], W = hdr[1], K = hdr[2], N = hdr[3], B = hdr[4], n_ids = hdr[5], split_min = hdr[6];
    auto fr = rd<double>(f, 2);
    gsparc_view view{};
    view.H = H;
    view.W = W;
    gsparc_band band{};
    band.K = K;
    band.f_c = fr[0];
    band.df = fr[1];
    const int TW = gsparc::tiles_x(view), T = TW * gsparc::tiles_y(view);
    auto proj = rd<float4>(f, 2 * (size_t)N);
    auto ranges = rd<uint32_t>(f, 2 * (size_t)T);
    auto ids = rd<uint32_t>(f, n_ids);
    auto attr = rd<float4>(f, (size_t)B * N);
    const size_t P = (size_t)H * W;
    auto target = rd<float2>(f, (size_t)B * K * P);
    fclose(f);
    const int S = gsparc::pick_strip(K, (int64_t)T * B);
    const int strips = (K + S - 1) / S;
    std::vector<float2> dspec((size_t)B * K * P, float2{nanf(""), nanf("")});
    std::vector<float> stot((size_t)B * strips * P, nanf("")), logT((size_t)B * P, nanf(""));
    std::vector<uint32_t> nc((size_t)B * P, 0xffffffffu), walks((size_t)B * T, 0xffffffffu);
    std::vector<float4> dattr((size_t)B * N, float4{0, 0, 0, 0});
    std::vector<float> dproj(8 * (size_t)N, 0.0f);
    float loss = 0.f;

    gsparc::RenderArgs a{};
    gsparc::fill_args(&view, &band, B, N, reinterpret_cast<const float*>(proj.data()), ranges.data(), ids.data(),
                      reinterpret_cast<const float*>(attr.data()), a);
    a.final_logT = logT.data();
    a.n_contrib = nc.data();
    a.l2_target = target.data();
    a.l2_loss = &loss;
    a.l2_grad = dspec.data();
    a.l2_inv = (float)(1.0 / ((double)B * K * P));
    a.s_tot = stot.data();
    a.tile_walk = walks.data();
    switch (S) {
        case 1: fwd<1>(a, T); break;
        case 2: fwd<2>(a, T); break;
        case 4: fwd<4>(a, T); break;
        case 8: fwd<8>(a, T); break;
        case 16: fwd<16>(a, T); break;
        default: fwd<32>(a, T); break;
    }
    // the schedule, from the forward's tile walks
    const gsparc::SchedLayout SL = gsparc::sched_layout(B, T, strips);
    std::vector<unsigned char> ws(SL.total, 0);
    uint32_t* hdrw = reinterpret_cast<uint32_t*>(ws.data() + SL.hdr);
    emu_launch(emu_dim3{1, 1, 1}, gsparc::kSchedThreads, gsparc::k_bwd_schedule, H, W, TW, T, B * T, strips, split_min,
               1, reinterpret_cast<const uint2*>(ranges.data()), (const uint32_t*)nc.data(),
               (const uint32_t*)walks.data(), hdrw, reinterpret_cast<uint32_t*>(ws.data() + SL.walks),
               reinterpret_cast<uint4*>(ws.data() + SL.items));
    const uint32_t n_items = hdrw[1];
    gsparc::RenderArgs g = a;
    g.l2_target = nullptr;
    g.l2_loss = nullptr;
    g.l2_grad = nullptr;
    g.tile_walk = nullptr;
    g.d_spectrum = dspec.data();
    g.d_attr = dattr.data();
    g.d_proj = dproj.data();
    g.items = reinterpret_cast<const uint4*>(ws.data() + SL.items);
    g.n_items = hdrw + 1;
    const unsigned launched = (unsigned)(2 * B * T * strips);
    switch (S) {
        case 1: bwd<1>(g, launched); break;
        case 2: bwd<2>(g, launched); break;
        case 4: bwd<4>(g, launched); break;
        case 8: bwd<8>(g, launched); break;
        case 16: bwd<16>(g, launched); break;
        default: bwd<32>(g, launched); break;
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(&loss, 4, 1, o);
    fwrite(dspec.data(), 8, dspec.size(), o);
    fwrite(stot.data(), 4, stot.size(), o);
    fwrite(logT.data(), 4, logT.size(), o);
    fwrite(nc.data(), 4, nc.size(), o);
    fwrite(walks.data(), 4, walks.size(), o);
    fwrite(&n_items, 4, 1, o);
    fwrite(ws.data() + SL.items, 16, n_items, o);
    fwrite(dattr.data(), 16, dattr.size(), o);
    fwrite(dproj.data(), 4, dproj.size(), o);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
