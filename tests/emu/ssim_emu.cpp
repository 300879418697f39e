// Runs the library's magnitude-spectrum loss kernels (csrc/ssim.cuh) under the host shim with the
// launch sequence of gsparc_spectrum_loss (the two double accumulators zeroed first).
// Input: int32 B, K, H, W, grad; float lambda; float spectrum[2n], target[n] (n = B K H W).
// Output: float loss, d_spectrum[2n]; int32 shim violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "ssim.cuh"

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
    auto hdr = rd<int32_t>(f, 5);
    const int B = hdr[0], K = hdr[1], H = hdr[2], W = hdr[3], grad = hdr[4];
    const float lambda = rd<float>(f, 1)[0];
    const int64_t n = (int64_t)B * K * H * W;
    auto z = rd<float2>(f, n);
    auto y = rd<float>(f, n);
    fclose(f);
    const SsLayout SL = ss_layout(n);
    std::vector<uint64_t> ws(SL.total / 8 + 2, 0);
    char* w = reinterpret_cast<char*>(ws.data());
    double* acc = reinterpret_cast<double*>(w + SL.acc);
    float* t5 = reinterpret_cast<float*>(w + SL.t5);
    float* abc = reinterpret_cast<float*>(w + SL.abc);
    float* t3 = reinterpret_cast<float*>(w + SL.t3);
    acc[0] = acc[1] = 0.0;
    const Window win = ss_window();
    float loss = nanf("");
    std::vector<float2> dz(n, float2{nanf(""), nanf("")});
    const emu_dim3 grid{(unsigned)((n + kSsThreads - 1) / kSsThreads), 1, 1};
    emu_launch(grid, kSsThreads, k_ssim_h, n, H, W, win, (const float2*)z.data(), (const float*)y.data(), t5);
    emu_launch(grid, kSsThreads, k_ssim_v, n, H, W, win, (const float2*)z.data(), (const float*)y.data(),
               (const float*)t5, abc, acc);
    emu_launch(emu_dim3{1, 1, 1}, 1, k_ssim_finish, (const double*)acc, (double)n, (double)lambda, &loss);
    if (grad) {
        emu_launch(grid, kSsThreads, k_ssim_bh, n, W, win, (const float*)abc, t3);
        emu_launch(grid, kSsThreads, k_ssim_bv, n, H, W, win, (const float2*)z.data(), (const float*)y.data(),
                   (const float*)t3, (float)((1.0 - lambda) / (double)n), (float)(-(double)lambda / (double)n),
                   dz.data());
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(&loss, 4, 1, o);
    fwrite(dz.data(), 8, n, o);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
