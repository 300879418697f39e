// Per-Gaussian emission network (Eq. 1 in the paper's own form, Sec. 4.1; one per Gaussian as
// the Sec. 4.2 implementation notes give it): every Gaussian i carries a network
// f_i: R^3 -> R^2 with one hidden ReLU layer of width h, evaluated at the
// query (transmitter) position x, and emits s_i = sigmoid(o_0 - ln d_i) + j sigmoid(o_1 - ln d_i)
// (the sigmoid element-wise on Re and Im), d_i = max(|x - mu_i|, 0.01).  The renderer's
// attributes follow: a = |s| / d (|s| with the 1/d term of the compositing rule switched off),
// phi0 = arg s, sigma = sigmoid(opacity logit), L = d + |mu - x_rx|.
//
// Flat buffer: row i holds W1 [3, h] (input-major), b1 [h], W2 [h, 2] (input-major), b2 [2]
// (6h + 2 floats), padded to a multiple of 4 floats (gsparc_emission_stride).  Every Gaussian
// has its own weights, so the work is a stream over the buffer (HBM-bound).  A group of G
// threads (G = h rounded up to a power of two, at most 32) takes one Gaussian, one hidden unit
// per thread (two or more when h > 32): a thread loads only its unit's six weights, which are
// consecutive across the group (coalesced), keeps them in registers for every transmitter, and
// the two outputs are summed over the group with shuffles.  Transmitters go in chunks of G: the
// group forms the chunk's outputs together, then each lane finishes one transmitter (distance,
// sigmoids, angle; in the backward the chain to dL/do, which it hands to the group by shuffle).
// The backward accumulates each unit's weight gradients over the transmitters in its thread's
// registers and adds them to the buffer's columns once.
//
// Device code only (launches and entry points are in emission.cu), so that the same source also
// builds for the host under the test suite's shim.

#pragma once

#include <math.h>
#include <stdint.h>

#include "device_common.cuh"

namespace gsparc {
namespace {

constexpr int kEmMaxHidden = 64;
constexpr int kEmThreads = 128;
constexpr int kEmMaxUnits = 2;   // hidden units per thread: h <= 32 G

inline int em_stride(int h) { return (6 * h + 2 + 3) / 4 * 4; }
inline int em_group(int h) {
    int g = 1;
    while (g < h && g < 32) g <<= 1;
    return g;
}

__device__ __forceinline__ float em_sigmoid(float x) { return 1.0f / (1.0f + expf(-x)); }

// Sum over the aligned group of G lanes (G a power of two dividing 32); every lane gets it.
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One hidden unit's weights: W1[0..2][j], b1[j], W2[j][0..1].
struct Unit {
    float w0, w1, w2, b, v0, v1;
    bool on;   // j < h
};

__device__ __forceinline__ Unit load_unit(const float* __restrict__ row, int h, int j) {
    Unit u;
    u.on = j < h;
    if (u.on) {
        u.w0 = __ldg(row + j);
        u.w1 = __ldg(row + h + j);
        u.w2 = __ldg(row + 2 * h + j);
        u.b = __ldg(row + 3 * h + j);
        u.v0 = __ldg(row + 4 * h + 2 * j);
        u.v1 = __ldg(row + 4 * h + 2 * j + 1);
    } else {
        u.w0 = u.w1 = u.w2 = u.b = u.v0 = u.v1 = 0.f;
    }
    return u;
}

__device__ __forceinline__ float unit_pre(const Unit& u, float t0, float t1, float t2) {
    return fmaf(t2, u.w2, fmaf(t1, u.w1, fmaf(t0, u.w0, u.b)));
}

template <int G>
__global__ void __launch_bounds__(kEmThreads) k_emission_fwd(int N, int B, int h, int stride,
                                                             const float* __restrict__ tx, float rx0, float rx1,
                                                             float rx2, const float* __restrict__ means,
                                                             const float* __restrict__ ologit,
                                                             const float* __restrict__ weights, int inv_d,
                                                             float4* __restrict__ attr) {
    const int t = blockIdx.x * kEmThreads + threadIdx.x;
    const int lg = t % G;
    // every lane stays for the group sums (full-warp shuffles); a group past the end reads the
    // last row and writes nothing
    const bool valid = t / G < N;
    const int i = valid ? t / G : N - 1;
    const float* row = weights + (size_t)i * stride;
    constexpr int U = kEmMaxUnits;
    Unit un[U];
#pragma unroll
    for (int q = 0; q < U; ++q) un[q] = load_unit(row, h, lg + G * q);
    const float m0 = __ldg(means + 3 * i), m1 = __ldg(means + 3 * i + 1), m2 = __ldg(means + 3 * i + 2);
    const float sig = em_sigmoid(__ldg(ologit + i));
    const float f0 = m0 - rx0, f1 = m1 - rx1, f2 = m2 - rx2;
    const float r = sqrtf(f0 * f0 + f1 * f1 + f2 * f2);
    const float b20 = __ldg(row + 6 * h), b21 = __ldg(row + 6 * h + 1);
    // transmitters in chunks of G: every lane forms the chunk's outputs (group sums), then lane
    // bb finishes transmitter b0 + bb (the per-Gaussian tail: distance, sigmoids, angle)
    for (int b0 = 0; b0 < B; b0 += G) {
        const int nb = min(G, B - b0);
        float my0 = 0.f, my1 = 0.f;
        for (int bb = 0; bb < nb; ++bb) {
            const int b = b0 + bb;
            const float t0 = __ldg(tx + 3 * b), t1 = __ldg(tx + 3 * b + 1), t2 = __ldg(tx + 3 * b + 2);
            float p0 = 0.f, p1 = 0.f;
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const float p = fmaxf(unit_pre(un[q], t0, t1, t2), 0.0f);
                p0 = fmaf(p, un[q].v0, p0);
                p1 = fmaf(p, un[q].v1, p1);
            }
            const float o0 = group_sum<G>(p0) + b20, o1 = group_sum<G>(p1) + b21;
            if (lg == bb) {
                my0 = o0;
                my1 = o1;
            }
        }
        if (lg < nb && valid) {
            const int b = b0 + lg;
            const float e0 = m0 - __ldg(tx + 3 * b), e1 = m1 - __ldg(tx + 3 * b + 1), e2 = m2 - __ldg(tx + 3 * b + 2);
            const float d = fmaxf(sqrtf(e0 * e0 + e1 * e1 + e2 * e2), kDMin);
            const float logd = logf(d);
            const float re = em_sigmoid(my0 - logd), im = em_sigmoid(my1 - logd);
            const float mag = sqrtf(re * re + im * im);
            attr[(size_t)b * N + i] = make_float4(inv_d ? mag / d : mag, atan2f(im, re), sig, d + r);
        }
    }
}

template <int G>
__global__ void __launch_bounds__(kEmThreads) k_emission_bwd(int N, int B, int h, int stride,
                                                             const float* __restrict__ tx, float rx0, float rx1,
                                                             float rx2, const float* __restrict__ means,
                                                             const float* __restrict__ ologit,
                                                             const float* __restrict__ weights, int inv_d,
                                                             const float4* __restrict__ d_attr,
                                                             float* __restrict__ d_means, float* __restrict__ d_ologit,
                                                             float* __restrict__ d_weights) {
    const int t = blockIdx.x * kEmThreads + threadIdx.x;
    const int lg = t % G;
    const bool valid = t / G < N;   // as in the forward: all lanes take part in the group sums
    const int i = valid ? t / G : N - 1;
    const float* row = weights + (size_t)i * stride;
    constexpr int U = kEmMaxUnits;
    Unit un[U];
    float gw0[U], gw1[U], gw2[U], gb[U], gv0[U], gv1[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
        un[q] = load_unit(row, h, lg + G * q);
        gw0[q] = gw1[q] = gw2[q] = gb[q] = gv0[q] = gv1[q] = 0.f;
    }
    const float m0 = __ldg(means + 3 * i), m1 = __ldg(means + 3 * i + 1), m2 = __ldg(means + 3 * i + 2);
    const float sig = em_sigmoid(__ldg(ologit + i));
    const float f0 = m0 - rx0, f1 = m1 - rx1, f2 = m2 - rx2;
    const float r = sqrtf(f0 * f0 + f1 * f1 + f2 * f2);
    const float b20 = __ldg(row + 6 * h), b21 = __ldg(row + 6 * h + 1);
    float gm0 = 0.f, gm1 = 0.f, gm2 = 0.f, gol = 0.f, gb20 = 0.f, gb21 = 0.f;
    const int base = (int)(threadIdx.x & 31) & ~(G - 1);   // the group's first lane in the warp
    // transmitters in chunks of G as in the forward: the chunk's outputs (group sums), lane bb's
    // tail for transmitter b0 + bb (its per-Gaussian gradient terms accumulate in that lane),
    // then dL/do of each transmitter from its lane to the whole group for the units' gradients
    for (int b0 = 0; b0 < B; b0 += G) {
        const int nb = min(G, B - b0);
        float my0 = 0.f, my1 = 0.f;
        for (int bb = 0; bb < nb; ++bb) {
            const int b = b0 + bb;
            const float t0 = __ldg(tx + 3 * b), t1 = __ldg(tx + 3 * b + 1), t2 = __ldg(tx + 3 * b + 2);
            float p0 = 0.f, p1 = 0.f;
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const float p = fmaxf(unit_pre(un[q], t0, t1, t2), 0.0f);
                p0 = fmaf(p, un[q].v0, p0);
                p1 = fmaf(p, un[q].v1, p1);
            }
            const float o0 = group_sum<G>(p0) + b20, o1 = group_sum<G>(p1) + b21;
            if (lg == bb) {
                my0 = o0;
                my1 = o1;
            }
        }
        float g_o0 = 0.f, g_o1 = 0.f;
        if (lg < nb) {
            const int b = b0 + lg;
            const float4 da = __ldg(d_attr + (size_t)b * N + i);   // (a, phi0, sigma, L)
            const float e0 = m0 - __ldg(tx + 3 * b), e1 = m1 - __ldg(tx + 3 * b + 1), e2 = m2 - __ldg(tx + 3 * b + 2);
            const float dist = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
            const float d = fmaxf(dist, kDMin);
            const float logd = logf(d);
            const float re = em_sigmoid(my0 - logd), im = em_sigmoid(my1 - logd);
            const float mag2 = re * re + im * im, mag = sqrtf(mag2);
            const float ka = inv_d ? 1.0f / d : 1.0f;
            // a = |s| ka, phi0 = atan2(im, re): chain to Re and Im of s
            const float g_re = da.x * ka * re / mag - da.y * im / mag2;
            const float g_im = da.x * ka * im / mag + da.y * re / mag2;
            g_o0 = g_re * re * (1.0f - re);
            g_o1 = g_im * im * (1.0f - im);
            gb20 += g_o0;
            gb21 += g_o1;
            // d enters through ln d (both sigmoids), the 1/d factor and L = d + r
            float g_d = -(g_o0 + g_o1) / d + da.w;
            if (inv_d) g_d -= da.x * mag / (d * d);
            if (dist > kDMin) {
                const float k = g_d / dist;
                gm0 += k * e0;
                gm1 += k * e1;
                gm2 += k * e2;
            }
            if (r > 0.f) {
                const float k = da.w / r;
                gm0 += k * f0;
                gm1 += k * f1;
                gm2 += k * f2;
            }
            gol += da.z * sig * (1.0f - sig);
        }
        // the network: W2, then through the ReLU to W1, b1 (each lane its units)
        for (int bb = 0; bb < nb; ++bb) {
            const int b = b0 + bb;
            const float go0 = __shfl_sync(0xffffffffu, g_o0, base + bb);
            const float go1 = __shfl_sync(0xffffffffu, g_o1, base + bb);
            const float t0 = __ldg(tx + 3 * b), t1 = __ldg(tx + 3 * b + 1), t2 = __ldg(tx + 3 * b + 2);
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const float pre = unit_pre(un[q], t0, t1, t2);
                if (pre > 0.f) {
                    gv0[q] = fmaf(pre, go0, gv0[q]);
                    gv1[q] = fmaf(pre, go1, gv1[q]);
                    const float gh = un[q].v0 * go0 + un[q].v1 * go1;
                    gb[q] += gh;
                    gw0[q] = fmaf(t0, gh, gw0[q]);
                    gw1[q] = fmaf(t1, gh, gw1[q]);
                    gw2[q] = fmaf(t2, gh, gw2[q]);
                }
            }
        }
    }
    // the per-Gaussian terms, spread over the lanes that took transmitters, to the group
    gm0 = group_sum<G>(gm0);
    gm1 = group_sum<G>(gm1);
    gm2 = group_sum<G>(gm2);
    gol = group_sum<G>(gol);
    gb20 = group_sum<G>(gb20);
    gb21 = group_sum<G>(gb21);
    if (!valid) return;   // after the last group sum
    float* grow = d_weights + (size_t)i * stride;
#pragma unroll
    for (int q = 0; q < U; ++q) {
        const int j = lg + G * q;
        if (j < h) {
            grow[j] += gw0[q];
            grow[h + j] += gw1[q];
            grow[2 * h + j] += gw2[q];
            grow[3 * h + j] += gb[q];
            grow[4 * h + 2 * j] += gv0[q];
            grow[4 * h + 2 * j + 1] += gv1[q];
        }
    }
    if (lg == 0) {
        grow[6 * h] += gb20;
        grow[6 * h + 1] += gb21;
        atomicAdd(&d_means[3 * i], gm0);
        atomicAdd(&d_means[3 * i + 1], gm1);
        atomicAdd(&d_means[3 * i + 2], gm2);
        atomicAdd(&d_ologit[i], gol);
    }
}

}  // namespace
}  // namespace gsparc
