// Runs the library's per-Gaussian emission kernels (csrc/emission.cuh) under the host shim with
// the launch shape of gsparc_emission_fwd / _bwd: groups of G = em_group(h) lanes per Gaussian,
// blocks of kEmThreads threads.
// Input: int32 N, B, h, inv_d; float tx[3B], rx[3], means[3N], ologit[N], weights[N stride],
// d_attr[4BN].  Output: float attr[4BN], d_means[3N], d_ologit[N], d_weights[N stride]; int32 shim
// violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "emission.cuh"

template <typename T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

template <int G>
static void run(int N, int B, int h, int stride, const std::vector<float>& tx, const std::vector<float>& rx,
                const std::vector<float>& means, const std::vector<float>& ologit, const std::vector<float>& w,
                int inv_d, const std::vector<float4>& dattr, std::vector<float4>& attr, std::vector<float>& dm,
                std::vector<float>& dol, std::vector<float>& dw) {
    const int64_t threads = (int64_t)N * G;
    const emu_dim3 grid{(unsigned)((threads + gsparc::kEmThreads - 1) / gsparc::kEmThreads), 1, 1};
    emu_launch(grid, gsparc::kEmThreads, gsparc::k_emission_fwd<G>, N, B, h, stride, (const float*)tx.data(), rx[0],
               rx[1], rx[2], (const float*)means.data(), (const float*)ologit.data(), (const float*)w.data(), inv_d,
               attr.data());
    emu_launch(grid, gsparc::kEmThreads, gsparc::k_emission_bwd<G>, N, B, h, stride, (const float*)tx.data(), rx[0],
               rx[1], rx[2], (const float*)means.data(), (const float*)ologit.data(), (const float*)w.data(), inv_d,
               (const float4*)dattr.data(), dm.data(), dol.data(), dw.data());
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    auto hdr = rd<int32_t>(f, 4);
    const int N = hdr[0], B = hdr[1], h = hdr[2], inv_d = hdr[3];
    const int stride = gsparc::em_stride(h);
    auto tx = rd<float>(f, 3 * (size_t)B), rx = rd<float>(f, 3), means = rd<float>(f, 3 * (size_t)N);
    auto ologit = rd<float>(f, N), w = rd<float>(f, (size_t)N * stride);
    auto dattr = rd<float4>(f, (size_t)B * N);
    fclose(f);
    std::vector<float4> attr((size_t)B * N, float4{nanf(""), nanf(""), nanf(""), nanf("")});
    std::vector<float> dm(3 * (size_t)N, 0.0f), dol(N, 0.0f), dw((size_t)N * stride, 0.0f);
    switch (gsparc::em_group(h)) {
        case 1: run<1>(N, B, h, stride, tx, rx, means, ologit, w, inv_d, dattr, attr, dm, dol, dw); break;
        case 2: run<2>(N, B, h, stride, tx, rx, means, ologit, w, inv_d, dattr, attr, dm, dol, dw); break;
        case 4: run<4>(N, B, h, stride, tx, rx, means, ologit, w, inv_d, dattr, attr, dm, dol, dw); break;
        case 8: run<8>(N, B, h, stride, tx, rx, means, ologit, w, inv_d, dattr, attr, dm, dol, dw); break;
        case 16: run<16>(N, B, h, stride, tx, rx, means, ologit, w, inv_d, dattr, attr, dm, dol, dw); break;
        default: run<32>(N, B, h, stride, tx, rx, means, ologit, w, inv_d, dattr, attr, dm, dol, dw); break;
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(attr.data(), 16, attr.size(), o);
    fwrite(dm.data(), 4, dm.size(), o);
    fwrite(dol.data(), 4, dol.size(), o);
    fwrite(dw.data(), 4, dw.size(), o);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
