// Runs the library's FP32 compositing kernels (csrc/render_common.cuh) under the host shim with
// the arguments and launch shape of gsparc_render_fwd / gsparc_render_bwd: fill_args, the strip
// width of pick_strip, a (strips, tiles, transmitters) grid of kThreads threads.
// Input: int32 H, W, K, N, B, n_ids; double f_c, df; float proj[8N]; uint32 ranges[2T],
// ids[n_ids]; float attr[4BN], d_spectrum[2BKHW].  Output: float spectrum[2BKHW], final_logT[BHW];
// uint32 n_contrib[BHW], n_used[BHW]; float d_attr[4BN], d_proj[8N]; int32 shim violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "render_common.cuh"

template <typename T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

template <int S>
static void run(const gsparc::RenderArgs& a, int T) {
    const emu_dim3 grid{(unsigned)((a.K + S - 1) / S), (unsigned)T, (unsigned)a.B};
    emu_launch_smem(grid, gsparc::kThreads, gsparc::F32Smem<S>::kTotal, gsparc::k_render_fwd<S>, a);
    emu_launch_smem(grid, gsparc::kThreads, gsparc::F32BwdSmem<S>::kTotal, gsparc::k_render_bwd<S>, a);
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    auto hdr = rd<int32_t>(f, 6);
    const int H = hdr[0], W = hdr[1], K = hdr[2], N = hdr[3], B = hdr[4], n_ids = hdr[5];
    auto fr = rd<double>(f, 2);
    gsparc_view view{};
    view.H = H;
    view.W = W;
    gsparc_band band{};
    band.K = K;
    band.f_c = fr[0];
    band.df = fr[1];
    const int T = gsparc::tiles_x(view) * gsparc::tiles_y(view);
    auto proj = rd<float4>(f, 2 * (size_t)N);
    auto ranges = rd<uint32_t>(f, 2 * (size_t)T);
    auto ids = rd<uint32_t>(f, n_ids);
    auto attr = rd<float4>(f, (size_t)B * N);
    const size_t P = (size_t)H * W;
    auto dspec = rd<float2>(f, (size_t)B * K * P);
    fclose(f);
    std::vector<float2> spec((size_t)B * K * P, float2{nanf(""), nanf("")});
    std::vector<float> logT((size_t)B * P, nanf(""));
    std::vector<uint32_t> nc((size_t)B * P, 0xffffffffu), nu((size_t)B * P, 0xffffffffu);
    std::vector<float4> dattr((size_t)B * N, float4{0, 0, 0, 0});
    std::vector<float> dproj(8 * (size_t)N, 0.0f);

    gsparc::RenderArgs a{};
    gsparc::fill_args(&view, &band, B, N, reinterpret_cast<const float*>(proj.data()), ranges.data(), ids.data(),
                      reinterpret_cast<const float*>(attr.data()), a);
    a.spectrum = spec.data();
    a.final_logT = logT.data();
    a.n_contrib = nc.data();
    a.n_used = nu.data();
    a.d_spectrum = dspec.data();
    a.d_attr = dattr.data();
    a.d_proj = dproj.data();
    switch (gsparc::pick_strip(K, (int64_t)T * B)) {
        case 1: run<1>(a, T); break;
        case 2: run<2>(a, T); break;
        case 4: run<4>(a, T); break;
        case 8: run<8>(a, T); break;
        case 16: run<16>(a, T); break;
        default: run<32>(a, T); break;
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(spec.data(), 8, spec.size(), o);
    fwrite(logT.data(), 4, logT.size(), o);
    fwrite(nc.data(), 4, nc.size(), o);
    fwrite(nu.data(), 4, nu.size(), o);
    fwrite(dattr.data(), 16, dattr.size(), o);
    fwrite(dproj.data(), 4, dproj.size(), o);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
