// Adaptive density control (Algorithm 1, densification branch; Sec. 4.2 "Densification,
// Pruning, and Implementation"): device code only, so that the same source builds into the
// library and, under a host shim, into the test suite's CPU check of the kernels' logic.
//
// Per Gaussian i, from the mean positional-gradient norm since the last densification
// (norm_sum / count), its largest per-axis scale, its opacity and the footprint radius of its
// last projection record:
//   grow  = count > 0 and norm_sum / count >= tau_grad
//   clone = grow and exp(max log-scale) <= clone_scale (eps r_scene); split = grow otherwise
//   faint = sigmoid(opacity logit) < sigma_min;  wide = max(ext_x, ext_y) > r_max
// and it emits, in place and in index order: itself unless faint or wide (kept or cloned
// Gaussians), its clone unless faint, or n_split children unless faint (a split parent goes).
// A child of Gaussian i sits at mu_i + R_i diag(exp(l_i)) xi[i, c] with log-scales
// l_i - ln(0.8 n_split) and copies the rest.  Output positions come from a scan of the
// per-Gaussian output counts: block sums, one block scanning them, then each block scanning
// its own counts and writing its rows.
#pragma once

#include <stdint.h>

#include "gsparc.h"

namespace gsparc {

constexpr int kDensThreads = 256;          // Gaussians per block in the count and scatter passes
constexpr int kDensScanThreads = 1024;     // the one block that scans the block sums
constexpr int kDensMaxSplit = 8;

struct DensParams {
    float tau_grad;      // mean ||dL/dmu|| at or above which a Gaussian grows
    float clone_scale;   // largest per-axis scale (m) of a growing Gaussian that is cloned
    float sigma_min;     // opacity below which a Gaussian is pruned
    float r_max;         // footprint radius (px) above which an existing Gaussian is pruned
    float log_shrink;    // ln(0.8 n_split), subtracted from a child's log-scales
    int n_split;         // children of a split
};

struct DensDecision {
    int action;          // 0 keep, 1 clone, 2 split
    uint32_t n_out;      // rows this Gaussian emits
    bool self_kept;      // keep / clone: the Gaussian itself survives pruning
    bool clone_kept;     // clone: its copy survives pruning
};

inline int dens_blocks(int N) { return (N + kDensThreads - 1) / kDensThreads; }

__device__ __forceinline__ DensDecision dens_decide(int i, const DensParams& p, const float* log_scales,
                                                    const float* opacity_logit, const float* proj,
                                                    const float* norm_sum, const uint32_t* count) {
    const uint32_t c = count[i];
    const bool grow = c > 0 && norm_sum[i] / (float)c >= p.tau_grad;
    const float lmax = fmaxf(log_scales[3 * i], fmaxf(log_scales[3 * i + 1], log_scales[3 * i + 2]));
    const bool small = expf(lmax) <= p.clone_scale;
    const bool faint = 1.0f / (1.0f + expf(-opacity_logit[i])) < p.sigma_min;
    const bool wide = fmaxf(proj[8 * (int64_t)i + 2], proj[8 * (int64_t)i + 3]) > p.r_max;
    DensDecision d;
    d.action = grow ? (small ? 1 : 2) : 0;
    d.self_kept = d.action != 2 && !faint && !wide;
    d.clone_kept = d.action == 1 && !faint;
    d.n_out = d.action == 2 ? (faint ? 0u : (uint32_t)p.n_split) : (uint32_t)d.self_kept + (uint32_t)d.clone_kept;
    return d;
}

// Exclusive scan of one value per thread over a block of NW full warps; *total gets the block's
// sum.  Ends with a barrier, so it can be called again at once.
template <int NW>
__device__ __forceinline__ uint32_t dens_block_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sum[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < NW ? warp_sum[lane] : 0u;
        for (int o = 1; o < NW; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NW) warp_sum[lane] = t;        // inclusive over warps
    }
    __syncthreads();
    const uint32_t base = warp > 0 ? warp_sum[warp - 1] : 0u;
    *total = warp_sum[NW - 1];
    __syncthreads();
    return base + x - v;
}

// Accumulates the statistic: every Gaussian whose last projection was not culled (radius > 0)
// adds ||dL/dmu_i|| to norm_sum and 1 to count.
__global__ void __launch_bounds__(kDensThreads)
k_dens_accumulate(int N, const float* __restrict__ proj, const float* __restrict__ d_means,
                  float* __restrict__ norm_sum, uint32_t* __restrict__ count) {
    for (int i = blockIdx.x * kDensThreads + threadIdx.x; i < N; i += gridDim.x * kDensThreads) {
        if (!(fmaxf(proj[8 * (int64_t)i + 2], proj[8 * (int64_t)i + 3]) > 0.0f)) continue;
        const float gx = d_means[3 * i], gy = d_means[3 * i + 1], gz = d_means[3 * i + 2];
        norm_sum[i] += sqrtf(gx * gx + gy * gy + gz * gz);
        count[i] += 1u;
    }
}

// Pass 1: rows emitted by each block of kDensThreads Gaussians.
__global__ void __launch_bounds__(kDensThreads)
k_dens_count(int N, DensParams p, const float* __restrict__ log_scales, const float* __restrict__ opacity_logit,
             const float* __restrict__ proj, const float* __restrict__ norm_sum,
             const uint32_t* __restrict__ count, uint32_t* __restrict__ block_rows) {
    const int i = blockIdx.x * kDensThreads + threadIdx.x;
    const uint32_t n = i < N ? dens_decide(i, p, log_scales, opacity_logit, proj, norm_sum, count).n_out : 0u;
    uint32_t total = 0;
    dens_block_scan<kDensThreads / 32>(n, &total);
    if (threadIdx.x == 0) block_rows[blockIdx.x] = total;
}

// Pass 2 (one block): exclusive scan of the block row counts in place; the total to *n_out,
// GSPARC_ERR_CAPACITY to the status word when it exceeds the capacity.
__global__ void __launch_bounds__(kDensScanThreads)
k_dens_scan(int nb, uint32_t capacity, uint32_t* __restrict__ block_rows, uint32_t* __restrict__ n_out,
            int32_t* __restrict__ status) {
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += kDensScanThreads) {
        const int j = base + (int)threadIdx.x;
        const uint32_t v = j < nb ? block_rows[j] : 0u;
        uint32_t chunk = 0;
        const uint32_t ex = dens_block_scan<kDensScanThreads / 32>(v, &chunk);
        if (j < nb) block_rows[j] = carry + ex;
        carry += chunk;
    }
    if (threadIdx.x == 0) {
        *n_out = carry;
        if (carry > capacity && status) atomicCAS(reinterpret_cast<int*>(status), 0, GSPARC_ERR_CAPACITY);
    }
}

// Rotation of the unit quaternion q / |q|, q = (w, x, y, z): the matrix of v -> q v q*.
__device__ __forceinline__ void dens_rotation(const float* q, float R[3][3]) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    const float inv = 1.0f / sqrtf(w * w + x * x + y * y + z * z);
    w *= inv;
    x *= inv;
    y *= inv;
    z *= inv;
    R[0][0] = 1.0f - 2.0f * (y * y + z * z);
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = 1.0f - 2.0f * (x * x + z * z);
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = 1.0f - 2.0f * (x * x + y * y);
}

struct DensOut {
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_logit;
    float* payload;      // may be null when P = 0
    uint32_t* parent;
};

// Pass 3: every block scans its Gaussians' row counts, adds its block offset and writes the
// rows that fall below the capacity.
__global__ void __launch_bounds__(kDensThreads)
k_dens_scatter(int N, int P, DensParams p, const float* __restrict__ means, const float* __restrict__ log_scales,
               const float* __restrict__ quats, const float* __restrict__ opacity_logit,
               const float* __restrict__ payload, const float* __restrict__ proj,
               const float* __restrict__ norm_sum, const uint32_t* __restrict__ count,
               const float* __restrict__ xi, const uint32_t* __restrict__ block_rows, uint32_t capacity,
               DensOut out) {
    const int i = blockIdx.x * kDensThreads + threadIdx.x;
    DensDecision d{0, 0u, false, false};
    if (i < N) d = dens_decide(i, p, log_scales, opacity_logit, proj, norm_sum, count);
    uint32_t total = 0;
    const uint32_t first = block_rows[blockIdx.x] + dens_block_scan<kDensThreads / 32>(d.n_out, &total);
    if (i >= N || d.n_out == 0) return;

    auto copy_row = [&](uint32_t row) {
        for (int k = 0; k < 3; ++k) {
            out.means[3 * (size_t)row + k] = means[3 * (size_t)i + k];
            out.log_scales[3 * (size_t)row + k] = log_scales[3 * (size_t)i + k];
        }
        for (int k = 0; k < 4; ++k) out.quats[4 * (size_t)row + k] = quats[4 * (size_t)i + k];
        out.opacity_logit[row] = opacity_logit[i];
        for (int k = 0; k < P; ++k) out.payload[(size_t)P * row + k] = payload[(size_t)P * i + k];
        out.parent[row] = (uint32_t)i;
    };

    if (d.action == 2) {
        float R[3][3];
        dens_rotation(quats + 4 * (size_t)i, R);
        float s[3], l[3], mu[3];
        for (int k = 0; k < 3; ++k) {
            l[k] = log_scales[3 * (size_t)i + k];
            s[k] = expf(l[k]);
            mu[k] = means[3 * (size_t)i + k];
        }
        for (int c = 0; c < p.n_split; ++c) {
            const uint32_t row = first + (uint32_t)c;
            if (row >= capacity) break;
            copy_row(row);
            const float* e = xi + 3 * ((size_t)i * p.n_split + c);
            const float v0 = s[0] * e[0], v1 = s[1] * e[1], v2 = s[2] * e[2];
            for (int k = 0; k < 3; ++k) {
                out.means[3 * (size_t)row + k] = mu[k] + (R[k][0] * v0 + R[k][1] * v1 + R[k][2] * v2);
                out.log_scales[3 * (size_t)row + k] = l[k] - p.log_shrink;
            }
        }
        return;
    }
    uint32_t row = first;
    if (d.self_kept) {
        if (row < capacity) copy_row(row);
        ++row;
    }
    if (d.clone_kept && row < capacity) copy_row(row);
}

// sigma <- min(sigma, cap), on the logits: logit <- min(logit, logit_cap).
__global__ void __launch_bounds__(kDensThreads)
k_opacity_reset(int N, float logit_cap, float* __restrict__ opacity_logit) {
    for (int i = blockIdx.x * kDensThreads + threadIdx.x; i < N; i += gridDim.x * kDensThreads)
        opacity_logit[i] = fminf(opacity_logit[i], logit_cap);
}

}  // namespace gsparc
