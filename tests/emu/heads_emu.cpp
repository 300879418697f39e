// Runs the library's CSI head / channel loss / head backward kernels (csrc/csi.cuh) and the
// training step's L2 loss and Adam kernels (csrc/train.cuh) under the host shim, with the launch
// shapes of their entry points on a 152-SM device.
// Input: int32 B, K, P, count, n, step; float scale, lr, b1, b2, eps; float spectrum[2 B K P],
// target_csi[2 B K], z[2 count], target[2 count], p[n], g[n], m[n], v[n].
// Output: float csi[2BK], csi_loss, d_csi[2BK], d_spectrum[2BKP], l2_loss, d_z[2 count], p[n],
// m[n], v[n]; int32 shim violations.
#include <stdio.h>
#include <stdlib.h>

#include <cmath>

#include "cuda_emu.h"
#include "csi.cuh"
#include "train.cuh"

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
    auto hdr = rd<int32_t>(f, 6);
    const int B = hdr[0], K = hdr[1];
    const int64_t P = hdr[2], count = hdr[3], n = hdr[4];
    const int step = hdr[5];
    auto par = rd<float>(f, 5);
    const float scale = par[0], lr = par[1], b1 = par[2], b2 = par[3], eps = par[4];
    const int rows = B * K;
    auto spec = rd<float2>(f, (size_t)rows * P);
    auto tcsi = rd<float2>(f, rows);
    auto z = rd<float2>(f, count), tz = rd<float2>(f, count);
    auto p = rd<float>(f, n), g = rd<float>(f, n), m = rd<float>(f, n), v = rd<float>(f, n);
    fclose(f);
    const int sms = 152;

    // gsparc_csi_head: about four blocks per SM, chunks a multiple of the block size
    std::vector<float2> csi(rows, float2{0.f, 0.f});
    const int64_t want = std::max<int64_t>(1, ((int64_t)sms * 4 + rows - 1) / rows);
    int64_t chunk = (P + want - 1) / want;
    chunk = (chunk + kCsiThreads - 1) / kCsiThreads * kCsiThreads;
    const int64_t nchunk = (P + chunk - 1) / chunk;
    emu_launch(emu_dim3{(unsigned)nchunk, (unsigned)rows, 1}, kCsiThreads, k_csi_head, P, chunk,
               (const float2*)spec.data(), scale, csi.data());
    // gsparc_csi_loss
    float csi_loss = nanf("");
    std::vector<float2> dcsi(rows, float2{nanf(""), nanf("")});
    emu_launch(emu_dim3{1, 1, 1}, kCsiThreads, k_csi_loss, rows, (const float2*)csi.data(),
               (const float2*)tcsi.data(), &csi_loss, dcsi.data());
    // gsparc_csi_head_bwd
    std::vector<float2> dspec((size_t)rows * P, float2{nanf(""), nanf("")});
    const int64_t total = (int64_t)rows * P;
    const int64_t bblocks = std::min<int64_t>((total + kCsiThreads - 1) / kCsiThreads, (int64_t)sms * 8);
    emu_launch(emu_dim3{(unsigned)bblocks, 1, 1}, kCsiThreads, k_csi_bcast, P, total, (const float2*)dcsi.data(),
               scale, dspec.data());
    // gsparc_l2_loss
    float l2 = 0.f;
    std::vector<float2> dz(count, float2{nanf(""), nanf("")});
    const int lblocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)sms * 8);
    emu_launch(emu_dim3{(unsigned)lblocks, 1, 1}, 256, k_l2_loss, count, (const float2*)z.data(),
               (const float2*)tz.data(), (float)(1.0 / (double)count), &l2, dz.data());
    // gsparc_adam
    const float bc1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float bc2 = (float)(1.0 - std::pow((double)b2, (double)step));
    const int ablocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    emu_launch(emu_dim3{(unsigned)ablocks, 1, 1}, 256, k_adam, n, p.data(), (const float*)g.data(), m.data(),
               v.data(), lr, b1, b2, eps, bc1, bc2);

    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(csi.data(), 8, csi.size(), o);
    fwrite(&csi_loss, 4, 1, o);
    fwrite(dcsi.data(), 8, dcsi.size(), o);
    fwrite(dspec.data(), 8, dspec.size(), o);
    fwrite(&l2, 4, 1, o);
    fwrite(dz.data(), 8, dz.size(), o);
    fwrite(p.data(), 4, p.size(), o);
    fwrite(m.data(), 4, m.size(), o);
    fwrite(v.data(), 4, v.size(), o);
    int32_t viol = g_emu_violations.load();
    fwrite(&viol, 4, 1, o);
    fclose(o);
    return 0;
}
