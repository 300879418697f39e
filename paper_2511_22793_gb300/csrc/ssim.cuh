// Magnitude-spectrum loss (Eq. 4): L = (1 - lam) L1(x, y) + lam (1 - SSIM(x, y)) with x = |z|
// the magnitude of the rendered spectrum and y a magnitude target, and its gradient dL/dz.
//
// SSIM per (transmitter, subcarrier) plane: an 11 x 11 Gaussian window (sigma 1.5, normalised),
// zero padding with the output the size of the plane, C1 = 0.01^2, C2 = 0.03^2; the loss takes
// the mean of the SSIM map over the plane and over planes; L1 is the mean |x - y|.
// The window is separable, so every filtering is a horizontal and a vertical 11-tap pass:
//   1. horizontal sums of x, y, x^2, y^2, x y                          (5 maps)
//   2. vertical sums -> mu_x, mu_y, E[x^2], E[y^2], E[xy] -> the SSIM map S, its partials
//      A = dS/dmu_x, Bm = dS/dE[x^2], Cm = dS/dE[xy] per pixel; sums of S and |x - y|
//   3. horizontal, 4. vertical sums of A, Bm, Cm (the window is symmetric and the padding zero,
//      so the transpose of the filter is the filter) -> dSSIM/dx_q = (wA)_q + 2 x_q (wBm)_q +
//      y_q (wCm)_q, then dL/dz = dL/dx z / |z| (0 where z = 0).
// Every pass reads and writes whole maps (HBM-bound); sums go to two double accumulators.
//
// Device code and workspace layout only (the entry points are in ssim.cu), so that the same
// source also builds for the host under the test suite's shim.

#pragma once

#include <math.h>
#include <stdint.h>

#include <cmath>

#include "device_common.cuh"

namespace gsparc {
namespace {

constexpr int kSsW = 11;            // window taps
constexpr int kSsR = kSsW / 2;
constexpr int kSsThreads = 256;
constexpr float kSsC1 = 0.01f * 0.01f;
constexpr float kSsC2 = 0.03f * 0.03f;

struct Window {
    float w[kSsW];
};

__device__ __forceinline__ float mag_of(float2 z) { return sqrtf(z.x * z.x + z.y * z.y); }

// 1. horizontal sums of x, y, x^2, y^2, xy: t5[m][e], e = plane * HW + pixel
__global__ void __launch_bounds__(kSsThreads) k_ssim_h(int64_t total, int H, int W, Window win,
                                                       const float2* __restrict__ z, const float* __restrict__ y,
                                                       float* __restrict__ t5) {
    const int64_t e = (int64_t)blockIdx.x * kSsThreads + threadIdx.x;
    if (e >= total) return;
    const int col = (int)(e % W);
    const int64_t rowbase = e - col;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
    for (int t = -kSsR; t <= kSsR; ++t) {
        const int c = col + t;
        if (c >= 0 && c < W) {
            const float xv = mag_of(z[rowbase + c]), yv = y[rowbase + c], wv = win.w[t + kSsR];
            s0 = fmaf(wv, xv, s0);
            s1 = fmaf(wv, yv, s1);
            s2 = fmaf(wv, xv * xv, s2);
            s3 = fmaf(wv, yv * yv, s3);
            s4 = fmaf(wv, xv * yv, s4);
        }
    }
    t5[e] = s0;
    t5[total + e] = s1;
    t5[2 * total + e] = s2;
    t5[3 * total + e] = s3;
    t5[4 * total + e] = s4;
}

__device__ __forceinline__ void block_add2(double a, double b, double* acc) {
    __shared__ double s_a[kSsThreads / 32], s_b[kSsThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        s_a[warp] = a;
        s_b[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w2 = 0; w2 < kSsThreads / 32; ++w2) {
            ta += s_a[w2];
            tb += s_b[w2];
        }
        atomicAdd(&acc[0], ta);
        atomicAdd(&acc[1], tb);
    }
}

// 2. vertical sums -> S and its partials (abc[3][e]); acc[0] += |x - y|, acc[1] += S
__global__ void __launch_bounds__(kSsThreads) k_ssim_v(int64_t total, int H, int W, Window win,
                                                       const float2* __restrict__ z, const float* __restrict__ y,
                                                       const float* __restrict__ t5, float* __restrict__ abc,
                                                       double* __restrict__ acc) {
    const int64_t e = (int64_t)blockIdx.x * kSsThreads + threadIdx.x;
    double l1 = 0.0, ssum = 0.0;
    if (e < total) {
        const int HW = H * W;
        const int p = (int)(e % HW);
        const int row = p / W;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = -kSsR; t <= kSsR; ++t) {
            const int r = row + t;
            if (r >= 0 && r < H) {
                const int64_t q = e + (int64_t)t * W;
                const float wv = win.w[t + kSsR];
#pragma unroll
                for (int k = 0; k < 5; ++k) m[k] = fmaf(wv, t5[k * total + q], m[k]);
            }
        }
        const float mx = m[0], my = m[1];
        const float n1 = 2.f * mx * my + kSsC1, n2 = 2.f * (m[4] - mx * my) + kSsC2;
        const float d1 = mx * mx + my * my + kSsC1, d2 = (m[2] - mx * mx) + (m[3] - my * my) + kSsC2;
        const float inv = 1.0f / (d1 * d2);
        const float S = n1 * n2 * inv;
        // partials written without dividing by n2, which may vanish
        abc[e] = 2.f * my * (n2 - n1) * inv - 2.f * mx * S / d1 + 2.f * mx * S / d2;   // dS/dmu_x
        abc[total + e] = -S / d2;                                                   // dS/dE[x^2]
        abc[2 * total + e] = 2.f * n1 * inv;                                        // dS/dE[xy]
        l1 = fabs((double)mag_of(z[e]) - (double)y[e]);
        ssum = S;
    }
    block_add2(l1, ssum, acc);
}

// 3. horizontal sums of the three partial maps
__global__ void __launch_bounds__(kSsThreads) k_ssim_bh(int64_t total, int W, Window win,
                                                        const float* __restrict__ abc, float* __restrict__ t3) {
    const int64_t e = (int64_t)blockIdx.x * kSsThreads + threadIdx.x;
    if (e >= total) return;
    const int col = (int)(e % W);
    const int64_t rowbase = e - col;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int t = -kSsR; t <= kSsR; ++t) {
        const int c = col + t;
        if (c >= 0 && c < W) {
            const float wv = win.w[t + kSsR];
            s0 = fmaf(wv, abc[rowbase + c], s0);
            s1 = fmaf(wv, abc[total + rowbase + c], s1);
            s2 = fmaf(wv, abc[2 * total + rowbase + c], s2);
        }
    }
    t3[e] = s0;
    t3[total + e] = s1;
    t3[2 * total + e] = s2;
}

// 4. vertical sums, then dL/dx and dL/dz
__global__ void __launch_bounds__(kSsThreads) k_ssim_bv(int64_t total, int H, int W, Window win,
                                                        const float2* __restrict__ z, const float* __restrict__ y,
                                                        const float* __restrict__ t3, float g_l1, float g_ss,
                                                        float2* __restrict__ dz) {
    const int64_t e = (int64_t)blockIdx.x * kSsThreads + threadIdx.x;
    if (e >= total) return;
    const int HW = H * W;
    const int row = (int)(e % HW) / W;
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
#pragma unroll
    for (int t = -kSsR; t <= kSsR; ++t) {
        const int r = row + t;
        if (r >= 0 && r < H) {
            const int64_t q = e + (int64_t)t * W;
            const float wv = win.w[t + kSsR];
            f0 = fmaf(wv, t3[q], f0);
            f1 = fmaf(wv, t3[total + q], f1);
            f2 = fmaf(wv, t3[2 * total + q], f2);
        }
    }
    const float2 zv = z[e];
    const float xv = mag_of(zv), yv = y[e];
    const float sgn = xv > yv ? 1.f : (xv < yv ? -1.f : 0.f);
    // g_l1 = (1 - lam) / M, g_ss = -lam / (planes * HW)
    const float gx = g_l1 * sgn + g_ss * (f0 + 2.f * xv * f1 + yv * f2);
    dz[e] = xv > 0.f ? make_float2(gx * zv.x / xv, gx * zv.y / xv) : make_float2(0.f, 0.f);
}

__global__ void k_ssim_finish(const double* __restrict__ acc, double m, double lam, float* __restrict__ loss) {
    loss[0] = (float)((1.0 - lam) * acc[0] / m + lam * (1.0 - acc[1] / m));
}

struct SsLayout {
    size_t acc, t5, abc, t3, total;
};

inline SsLayout ss_layout(int64_t n) {
    SsLayout L;
    size_t o = 0;
    L.acc = o;  o += 256;
    L.t5 = o;   o += ((size_t)5 * n * 4 + 255) & ~size_t(255);
    L.abc = o;  o += ((size_t)3 * n * 4 + 255) & ~size_t(255);
    L.t3 = o;   o += ((size_t)3 * n * 4 + 255) & ~size_t(255);
    L.total = o;
    return L;
}

// The normalised 11-tap Gaussian window (sigma 1.5), formed in double on the host.
inline Window ss_window() {
    Window win;
    double g[kSsW], sum = 0.0;
    for (int t = 0; t < kSsW; ++t) {
        const double d = t - kSsR;
        g[t] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[t];
    }
    for (int t = 0; t < kSsW; ++t) win.w[t] = (float)(g[t] / sum);
    return win;
}

}  // namespace
}  // namespace gsparc
