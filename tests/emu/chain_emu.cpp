// One FP32 training step of the library, stage after stage, under the host shim: projection,
// binning and sort, attribute network, compositing, complex L2 loss, compositing backward,
// network backward, projection backward -- the kernels of gsparc_project, gsparc_bin_sort,
// gsparc_attr_mlp (FP32), gsparc_render_fwd, gsparc_l2_loss, gsparc_render_bwd,
// gsparc_attr_mlp_bwd and gsparc_project_bwd with their launch shapes (152 SMs), each stage
// reading what the previous one wrote.
// Input: int32 n, H, W, K, hidden, B; double f_c, df; float means[3n], log_scales[3n],
// quats[4n], ologit[n], latent[16n], W1, b1, W2, b2, W3, b3, tx[3B], target[2 B K H W].
// Output: float loss, spectrum[2 B K H W], d_means[3n], d_log_scales[3n], d_quats[4n],
// d_ologit[n], d_latent[16n], dW1, db1, dW2, db2, dW3, db3; uint32 n_pairs; int32 violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "binsort.cuh"
#include "mlp_fp32.cuh"
#include "project.cuh"
#include "render_common.cuh"
#include "train.cuh"

template <typename T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

template <int S>
static void render_fwd(const gsparc::RenderArgs& a, int T) {
    emu_launch_smem(emu_dim3{(unsigned)((a.K + S - 1) / S), (unsigned)T, (unsigned)a.B}, gsparc::kThreads,
                    gsparc::F32Smem<S>::kTotal, gsparc::k_render_fwd<S>, a);
}
template <int S>
static void render_bwd(const gsparc::RenderArgs& a, int T) {
    emu_launch_smem(emu_dim3{(unsigned)((a.K + S - 1) / S), (unsigned)T, (unsigned)a.B}, gsparc::kThreads,
                    gsparc::F32BwdSmem<S>::kTotal, gsparc::k_render_bwd<S>, a);
}
template <int HD>
static void mlp(int n, int B, const float* tx, const float* means, const float* ologit, const float* latent,
                const gsparc::W& w, float4* attr, const float4* dattr, float* dm, float* dol, float* dlat,
                const gsparc_mlp_grad& g, bool backward) {
    const int64_t rows = (int64_t)n * B;
    if (!backward) {
        emu_launch(emu_dim3{(unsigned)((rows + 127) / 128), 1, 1}, 128, gsparc::k_mlp_fwd<HD>, n, B, tx, 0.f, 0.f,
                   0.f, means, ologit, latent, w, attr, static_cast<float*>(nullptr), (int64_t)0);
        return;
    }
    const int64_t tiles = (rows + gsparc::kBwdRows - 1) / gsparc::kBwdRows;
    emu_launch_smem(emu_dim3{(unsigned)std::min<int64_t>(tiles, 152 * 3), 1, 1}, gsparc::kBwdThreads,
                    (size_t)gsparc::BwdSmem<HD>::kTotal * sizeof(float), gsparc::k_mlp_bwd<HD>, n, B, tx, 0.f, 0.f,
                    0.f, means, ologit, latent, w, dattr, dm, dol, dlat, g, static_cast<const float*>(nullptr), (int64_t)0);
}

int main(int argc, char** argv) {
    using namespace gsparc;
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    auto hdr = rd<int32_t>(f, 6);
    const int n = hdr[0], H = hdr[1], W = hdr[2], K = hdr[3], h = hdr[4], B = hdr[5];
    auto fr = rd<double>(f, 2);
    auto means = rd<float>(f, 3 * (size_t)n), ls = rd<float>(f, 3 * (size_t)n);
    auto quats = rd<float4>(f, n);
    auto ologit = rd<float>(f, n), latent = rd<float>(f, 16 * (size_t)n);
    auto W1 = rd<float>(f, 20 * (size_t)h), b1 = rd<float>(f, h), W2 = rd<float>(f, (size_t)h * h),
         b2 = rd<float>(f, h), W3 = rd<float>(f, 3 * (size_t)h), b3 = rd<float>(f, 3);
    auto tx = rd<float>(f, 3 * (size_t)B);
    const size_t P = (size_t)H * W, count = (size_t)B * K * P;
    auto target = rd<float2>(f, count);
    fclose(f);

    gsparc_view view{};
    view.H = H;
    view.W = W;
    view.V[0] = view.V[4] = view.V[8] = 1.0f;
    view.near_dist = 0.1f;
    gsparc_band band{};
    band.K = K;
    band.f_c = fr[0];
    band.df = fr[1];
    ViewDev vd{};
    vd.H = H;
    vd.W = W;
    for (int i = 0; i < 9; ++i) vd.V[i] = view.V[i];
    vd.near_dist = view.near_dist;

    // projection
    std::vector<float4> proj(2 * (size_t)n);
    const unsigned pblk = (unsigned)((n + 255) / 256);
    emu_launch(emu_dim3{pblk, 1, 1}, 256, k_project, vd, n, (const float*)means.data(), (const float*)ls.data(),
               (const float4*)quats.data(), proj.data(), static_cast<int32_t*>(nullptr));
    // binning and sort
    const int TW = tiles_x(view), T = TW * tiles_y(view);
    const uint32_t cap = 64u * (uint32_t)n + 64u;
    std::vector<uint32_t> cnt(T, 0u), cursor(T, 0u), done(4, 0u), ids(cap, 0u), extra(T + 1, 0u);
    std::vector<uint2> ranges(T);
    std::vector<uint64_t> keys(cap), alt(cap);
    uint32_t n_pairs = 0;
    int32_t status = 0;
    const unsigned nblk = (unsigned)((n + kBinThreads - 1) / kBinThreads);
    std::vector<uint32_t> bcnt((size_t)nblk * T);   // T <= kSmemTiles here: emit takes the blocks' counts
    emu_launch(emu_dim3{nblk, 1, 1}, kBinThreads, k_tile_count, n, H, W, TW, T, (const float4*)proj.data(), cnt.data(),
               bcnt.data(), cursor.data(), done.data(), cap, ranges.data(), &n_pairs, extra.data(), 1, &status);
    emu_launch(emu_dim3{nblk, 1, 1}, kBinThreads, k_tile_emit, n, H, W, TW, T, (const float4*)proj.data(),
               (const uint32_t*)bcnt.data(), cursor.data(), cap, keys.data());
    emu_launch_smem(emu_dim3{sort_grid(T, cap, 4), 1, 1}, kSortThreads, kSortSmem, k_tile_sort, T,
                    (const uint2*)ranges.data(), (const uint32_t*)extra.data(), done.data() + 1, keys.data(), alt.data(), ids.data(),
                    (uint64_t*)nullptr);
    // attribute network
    gsparc::W w{W1.data(), b1.data(), W2.data(), b2.data(), W3.data(), b3.data()};
    std::vector<float4> attr((size_t)B * n);
    std::vector<float4> dattr((size_t)B * n, float4{0, 0, 0, 0});
    std::vector<float> dm(3 * (size_t)n, 0.f), dl(3 * (size_t)n, 0.f), dq(4 * (size_t)n, 0.f), dol(n, 0.f),
        dlat(16 * (size_t)n, 0.f);
    std::vector<float> gW1(W1.size(), 0.f), gb1(b1.size(), 0.f), gW2(W2.size(), 0.f), gb2(b2.size(), 0.f),
        gW3(W3.size(), 0.f), gb3(b3.size(), 0.f);
    gsparc_mlp_grad mg{gW1.data(), gb1.data(), gW2.data(), gb2.data(), gW3.data(), gb3.data()};
    auto run_mlp = [&](bool backward) {
        switch (h) {
            case 8: mlp<8>(n, B, tx.data(), means.data(), ologit.data(), latent.data(), w, attr.data(), dattr.data(), dm.data(), dol.data(), dlat.data(), mg, backward); break;
            case 16: mlp<16>(n, B, tx.data(), means.data(), ologit.data(), latent.data(), w, attr.data(), dattr.data(), dm.data(), dol.data(), dlat.data(), mg, backward); break;
            case 32: mlp<32>(n, B, tx.data(), means.data(), ologit.data(), latent.data(), w, attr.data(), dattr.data(), dm.data(), dol.data(), dlat.data(), mg, backward); break;
            default: mlp<64>(n, B, tx.data(), means.data(), ologit.data(), latent.data(), w, attr.data(), dattr.data(), dm.data(), dol.data(), dlat.data(), mg, backward); break;
        }
    };
    run_mlp(false);
    // compositing
    std::vector<float2> spec(count);
    std::vector<float> logT((size_t)B * P);
    std::vector<uint32_t> nc((size_t)B * P);
    std::vector<float> dproj(8 * (size_t)n, 0.f);
    RenderArgs a{};
    fill_args(&view, &band, B, n, reinterpret_cast<const float*>(proj.data()),
              reinterpret_cast<const uint32_t*>(ranges.data()), ids.data(), reinterpret_cast<const float*>(attr.data()),
              a);
    a.spectrum = spec.data();
    a.final_logT = logT.data();
    a.n_contrib = nc.data();
    const int S = pick_strip(K, (int64_t)T * B);
    auto fwd = [&]() {
        switch (S) {
            case 1: render_fwd<1>(a, T); break;
            case 2: render_fwd<2>(a, T); break;
            case 4: render_fwd<4>(a, T); break;
            case 8: render_fwd<8>(a, T); break;
            case 16: render_fwd<16>(a, T); break;
            default: render_fwd<32>(a, T); break;
        }
    };
    fwd();
    // loss
    float loss = 0.f;
    std::vector<float2> dz(count);
    emu_launch(emu_dim3{(unsigned)std::min<int64_t>((count + 255) / 256, 152 * 8), 1, 1}, 256, k_l2_loss,
               (int64_t)count, (const float2*)spec.data(), (const float2*)target.data(), (float)(1.0 / (double)count),
               &loss, dz.data());
    // backward
    a.d_spectrum = dz.data();
    a.d_attr = dattr.data();
    a.d_proj = dproj.data();
    switch (S) {
        case 1: render_bwd<1>(a, T); break;
        case 2: render_bwd<2>(a, T); break;
        case 4: render_bwd<4>(a, T); break;
        case 8: render_bwd<8>(a, T); break;
        case 16: render_bwd<16>(a, T); break;
        default: render_bwd<32>(a, T); break;
    }
    run_mlp(true);
    emu_launch(emu_dim3{pblk, 1, 1}, 256, k_project_bwd, vd, n, (const float*)means.data(), (const float*)ls.data(),
               (const float4*)quats.data(), (const float4*)dproj.data(), dm.data(), dl.data(), dq.data());

    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(&loss, 4, 1, o);
    fwrite(spec.data(), 8, spec.size(), o);
    for (auto* v : {&dm, &dl, &dq, &dol, &dlat, &gW1, &gb1, &gW2, &gb2, &gW3, &gb3}) fwrite(v->data(), 4, v->size(), o);
    fwrite(&n_pairs, 4, 1, o);
    int32_t viol = g_emu_violations.load() + (status != 0 ? 1000 : 0);
    fwrite(&viol, 4, 1, o);
    fclose(o);
    return 0;
}
