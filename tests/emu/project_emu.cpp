// Runs the library's projection kernels (csrc/project.cuh) under the host shim with the launch
// shape of gsparc_project / gsparc_project_bwd (256 threads, one Gaussian each).
// Input: int32 N, H, W; float rx[3], V[9], near; float means[3N], log_scales[3N], quats[4N],
// d_proj[8N].  Output: float proj[8N], d_means[3N], d_log_scales[3N], d_quats[4N]; int32 shim
// violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "project.cuh"

template <typename T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    auto hdr = rd<int32_t>(f, 3);
    const int N = hdr[0];
    auto vf = rd<float>(f, 13);
    gsparc::ViewDev v;
    v.H = hdr[1];
    v.W = hdr[2];
    v.rx0 = vf[0];
    v.rx1 = vf[1];
    v.rx2 = vf[2];
    for (int i = 0; i < 9; ++i) v.V[i] = vf[3 + i];
    v.near_dist = vf[12];
    auto means = rd<float>(f, 3 * (size_t)N), ls = rd<float>(f, 3 * (size_t)N);
    std::vector<float4> quats(N), dproj(2 * (size_t)N), proj(2 * (size_t)N);
    if (N && fread(quats.data(), 16, N, f) != (size_t)N) return 2;
    if (N && fread(dproj.data(), 16, 2 * (size_t)N, f) != 2 * (size_t)N) return 2;
    fclose(f);
    std::vector<float> dm(3 * (size_t)N, 0.0f), dl(3 * (size_t)N, 0.0f), dq(4 * (size_t)N, 0.0f);
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (N > 0) {
        emu_launch(emu_dim3{blocks, 1, 1}, 256, gsparc::k_project, v, N, (const float*)means.data(),
                   (const float*)ls.data(), (const float4*)quats.data(), proj.data(), static_cast<int32_t*>(nullptr));
        emu_launch(emu_dim3{blocks, 1, 1}, 256, gsparc::k_project_bwd, v, N, (const float*)means.data(),
                   (const float*)ls.data(), (const float4*)quats.data(), (const float4*)dproj.data(), dm.data(),
                   dl.data(), dq.data());
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(proj.data(), 16, 2 * (size_t)N, o);
    fwrite(dm.data(), 4, dm.size(), o);
    fwrite(dl.data(), 4, dl.size(), o);
    fwrite(dq.data(), 4, dq.size(), o);
    int32_t viol = g_emu_violations.load();
    fwrite(&viol, 4, 1, o);
    fclose(o);
    return 0;
}
