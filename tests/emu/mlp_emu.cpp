// Runs the library's FP32 attribute-network kernels (csrc/mlp_fp32.cuh) under the host shim with
// the launch shapes of gsparc_attr_mlp (128-row blocks) and gsparc_attr_mlp_bwd (persistent
// 128-thread CTAs; here two of them, so that each takes several passes).
// Input: int32 N, B, hidden, keep; float tx[3B], rx[3], means[3N], ologit[N], latent[16N], W1[20h],
// b1[h], W2[h h], b2[h], W3[3h], b3[3], d_attr[4BN].  Output: float attr[4BN], d_means[3N],
// d_ologit[N], d_latent[16N], dW1, db1, dW2, db2, dW3, db3; int32 shim violations.  keep = 1: the
// forward stores its activations (buffer and padding rows first set to NaN) and the backward
// reads them instead of recomputing.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "mlp_fp32.cuh"

template <typename T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

struct Grads {
    std::vector<float> W1, b1, W2, b2, W3, b3;
};

template <int HD>
static void run(int N, int B, const std::vector<float>& tx, const std::vector<float>& rx,
                const std::vector<float>& means, const std::vector<float>& ologit, const std::vector<float>& latent,
                const gsparc::W& w, const std::vector<float4>& dattr, std::vector<float4>& attr,
                std::vector<float>& dm, std::vector<float>& dol, std::vector<float>& dlat, Grads& g, bool keep) {
    const int64_t rows = (int64_t)N * B;
    const int64_t ld = (rows + 3) / 4 * 4;
    std::vector<float> hid(keep ? (size_t)(2 * HD) * ld : 0, nanf(""));
    float* hp = keep ? hid.data() : nullptr;
    if (keep)
        emu_launch(emu_dim3{(unsigned)((rows + 127) / 128), 1, 1}, 128, gsparc::k_mlp_fwd<HD, true>, N, B,
                   (const float*)tx.data(), rx[0], rx[1], rx[2], (const float*)means.data(),
                   (const float*)ologit.data(), (const float*)latent.data(), w, attr.data(), hp, ld);
    else
        emu_launch(emu_dim3{(unsigned)((rows + 127) / 128), 1, 1}, 128, gsparc::k_mlp_fwd<HD, false>, N, B,
                   (const float*)tx.data(), rx[0], rx[1], rx[2], (const float*)means.data(),
                   (const float*)ologit.data(), (const float*)latent.data(), w, attr.data(), hp, ld);
    const int64_t tiles = (rows + gsparc::kBwdRows - 1) / gsparc::kBwdRows;
    const unsigned blocks = (unsigned)std::min<int64_t>(tiles, 2);
    gsparc_mlp_grad mg{g.W1.data(), g.b1.data(), g.W2.data(), g.b2.data(), g.W3.data(), g.b3.data()};
    emu_launch_smem(emu_dim3{blocks, 1, 1}, gsparc::kBwdThreads, (size_t)gsparc::BwdSmem<HD>::kTotal * sizeof(float),
                    gsparc::k_mlp_bwd<HD>, N, B, (const float*)tx.data(), rx[0], rx[1], rx[2],
                    (const float*)means.data(), (const float*)ologit.data(), (const float*)latent.data(), w,
                    (const float4*)dattr.data(), dm.data(), dol.data(), dlat.data(), mg, (const float*)hp, ld);
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    auto hdr = rd<int32_t>(f, 4);
    const int N = hdr[0], B = hdr[1], h = hdr[2];
    const bool keep = hdr[3] != 0;
    auto tx = rd<float>(f, 3 * (size_t)B), rx = rd<float>(f, 3), means = rd<float>(f, 3 * (size_t)N);
    auto ologit = rd<float>(f, N);
    auto latent = rd<float>(f, 16 * (size_t)N);
    auto W1 = rd<float>(f, 20 * (size_t)h), b1 = rd<float>(f, h), W2 = rd<float>(f, (size_t)h * h),
         b2 = rd<float>(f, h), W3 = rd<float>(f, 3 * (size_t)h), b3 = rd<float>(f, 3);
    auto dattr = rd<float4>(f, (size_t)B * N);
    fclose(f);
    std::vector<float4> attr((size_t)B * N, float4{nanf(""), nanf(""), nanf(""), nanf("")});
    std::vector<float> dm(3 * (size_t)N, 0.0f), dol(N, 0.0f), dlat(16 * (size_t)N, 0.0f);
    Grads g{std::vector<float>(W1.size(), 0.0f), std::vector<float>(b1.size(), 0.0f),
            std::vector<float>(W2.size(), 0.0f), std::vector<float>(b2.size(), 0.0f),
            std::vector<float>(W3.size(), 0.0f), std::vector<float>(b3.size(), 0.0f)};
    gsparc::W w{W1.data(), b1.data(), W2.data(), b2.data(), W3.data(), b3.data()};
    switch (h) {
        case 8: run<8>(N, B, tx, rx, means, ologit, latent, w, dattr, attr, dm, dol, dlat, g, keep); break;
        case 16: run<16>(N, B, tx, rx, means, ologit, latent, w, dattr, attr, dm, dol, dlat, g, keep); break;
        case 32: run<32>(N, B, tx, rx, means, ologit, latent, w, dattr, attr, dm, dol, dlat, g, keep); break;
        default: run<64>(N, B, tx, rx, means, ologit, latent, w, dattr, attr, dm, dol, dlat, g, keep); break;
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(attr.data(), 16, attr.size(), o);
    for (auto* v : {&dm, &dol, &dlat, &g.W1, &g.b1, &g.W2, &g.b2, &g.W3, &g.b3}) fwrite(v->data(), 4, v->size(), o);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
