// Runs the library's densification kernels (csrc/densify.cuh) under the host shim with the launch
// shapes of gsparc_densify, gsparc_densify_accumulate (a two-block grid, so that its grid-stride
// loop wraps) and gsparc_opacity_reset.
// Input: int32 N, P, capacity, n_split; float tau_grad, clone_scale, sigma_min, r_max, log_shrink,
// logit_cap; float means[3N], log_scales[3N], quats[4N], opacity_logit[N], payload[N P], proj[8N],
// norm_sum[N]; uint32 count[N]; float xi[N n_split 3], d_means[3N].
// Output: uint32 n_out; int32 status; float out_means[3c], out_log_scales[3c], out_quats[4c],
// out_opacity_logit[c], out_payload[c P]; uint32 out_parent[c]; float acc_norm[N]; uint32
// acc_count[N]; float reset_logit[N]; int32 shim violations.  Unwritten rows keep NaN / 0xffffffff.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "cuda_emu.h"
#include "densify.cuh"

template <typename T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

template <typename T>
static void wr(FILE* f, const std::vector<T>& v) {
    if (!v.empty()) fwrite(v.data(), sizeof(T), v.size(), f);
}

// With a third argument "scan": input int32 nb, capacity; uint32 block_rows[nb]; output uint32
// n_out; int32 status; uint32 block_rows[nb] (exclusive scan); int32 shim violations.
static int scan_only(const char* in, const char* out) {
    FILE* f = fopen(in, "rb");
    if (!f) return 2;
    auto hdr = rd<int32_t>(f, 2);
    auto rows = rd<uint32_t>(f, hdr[0]);
    fclose(f);
    uint32_t n_out = 0xffffffffu;
    int32_t status = 0;
    emu_launch(emu_dim3{1, 1, 1}, gsparc::kDensScanThreads, gsparc::k_dens_scan, hdr[0], (uint32_t)hdr[1],
               rows.data(), &n_out, &status);
    FILE* o = fopen(out, "wb");
    if (!o) return 2;
    fwrite(&n_out, 4, 1, o);
    fwrite(&status, 4, 1, o);
    wr(o, rows);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}

int main(int argc, char** argv) {
    if (argc == 4 && strcmp(argv[3], "scan") == 0) return scan_only(argv[1], argv[2]);
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    auto hdr = rd<int32_t>(f, 4);
    const int N = hdr[0], P = hdr[1], cap = hdr[2], n_split = hdr[3];
    auto par = rd<float>(f, 6);
    auto means = rd<float>(f, 3 * (size_t)N), ls = rd<float>(f, 3 * (size_t)N), quats = rd<float>(f, 4 * (size_t)N);
    auto ologit = rd<float>(f, N), payload = rd<float>(f, (size_t)N * P), proj = rd<float>(f, 8 * (size_t)N);
    auto norm_sum = rd<float>(f, N);
    auto count = rd<uint32_t>(f, N);
    auto xi = rd<float>(f, (size_t)N * n_split * 3), d_means = rd<float>(f, 3 * (size_t)N);
    fclose(f);

    gsparc::DensParams p;
    p.tau_grad = par[0];
    p.clone_scale = par[1];
    p.sigma_min = par[2];
    p.r_max = par[3];
    p.log_shrink = par[4];
    p.n_split = n_split;
    const float logit_cap = par[5];

    const int nb = gsparc::dens_blocks(N);
    std::vector<uint32_t> block_rows(nb > 0 ? nb : 1, 0u);
    uint32_t n_out = 0xffffffffu;
    int32_t status = 0;
    const float nan = nanf("");
    std::vector<float> o_means(3 * (size_t)cap, nan), o_ls(3 * (size_t)cap, nan), o_q(4 * (size_t)cap, nan),
        o_ol(cap, nan), o_pl((size_t)cap * P, nan);
    std::vector<uint32_t> o_parent(cap, 0xffffffffu);
    if (N > 0) {
        emu_launch(emu_dim3{(unsigned)nb, 1, 1}, gsparc::kDensThreads, gsparc::k_dens_count, N, p,
                   (const float*)ls.data(), (const float*)ologit.data(), (const float*)proj.data(),
                   (const float*)norm_sum.data(), (const uint32_t*)count.data(), block_rows.data());
        emu_launch(emu_dim3{1, 1, 1}, gsparc::kDensScanThreads, gsparc::k_dens_scan, nb, (uint32_t)cap,
                   block_rows.data(), &n_out, &status);
        gsparc::DensOut o{o_means.data(), o_ls.data(), o_q.data(), o_ol.data(), P > 0 ? o_pl.data() : nullptr,
                          o_parent.data()};
        emu_launch(emu_dim3{(unsigned)nb, 1, 1}, gsparc::kDensThreads, gsparc::k_dens_scatter, N, P, p,
                   (const float*)means.data(), (const float*)ls.data(), (const float*)quats.data(),
                   (const float*)ologit.data(), (const float*)(P > 0 ? payload.data() : nullptr),
                   (const float*)proj.data(), (const float*)norm_sum.data(), (const uint32_t*)count.data(),
                   (const float*)xi.data(), (const uint32_t*)block_rows.data(), (uint32_t)cap, o);
    } else {
        n_out = 0;
    }
    std::vector<float> acc_norm = norm_sum, reset = ologit;
    std::vector<uint32_t> acc_count = count;
    if (N > 0) {
        const unsigned g = nb < 2 ? 1u : 2u;
        emu_launch(emu_dim3{g, 1, 1}, gsparc::kDensThreads, gsparc::k_dens_accumulate, N, (const float*)proj.data(),
                   (const float*)d_means.data(), acc_norm.data(), acc_count.data());
        emu_launch(emu_dim3{g, 1, 1}, gsparc::kDensThreads, gsparc::k_opacity_reset, N, logit_cap, reset.data());
    }

    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(&n_out, 4, 1, o);
    fwrite(&status, 4, 1, o);
    wr(o, o_means);
    wr(o, o_ls);
    wr(o, o_q);
    wr(o, o_ol);
    wr(o, o_pl);
    wr(o, o_parent);
    wr(o, acc_norm);
    wr(o, acc_count);
    wr(o, reset);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
