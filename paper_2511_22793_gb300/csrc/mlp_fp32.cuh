// Attribute network: per-(transmitter, Gaussian) emission and opacity.
//
// Eq. 1: s_i = sigmoid(f(x) - log d_i), d_i = |x_tx - mu_i|, with the 1/d_i
// free-space factor of the Sec. 4.2 compositing rule.  One network is shared
// by all Gaussians; its input is h0 = [tx (3), latent_i (16), ln d_i] and its
// three outputs give a = sigmoid(o_0 - ln d)/d, phi0 = o_1 and
// sigma = sigmoid(opacity_logit + o_2); L = d + |mu - rx| is the path length
// whose delay phases the subcarriers.
//
// FP32 path: one thread per (b, i) row, weights in shared memory (broadcast
// reads), the second hidden layer folded straight into the output layer so
// only one hidden vector lives in registers.
//
// Backward: persistent CTAs; one thread per row recomputes the activations in
// registers, the per-row vectors the weight gradients need are staged in
// shared memory (row-minor, padded against bank conflicts), and every CTA keeps
// its weight-gradient partials in registers until one atomic per entry at the
// end.
//
// Device code only (the entry points are in mlp.cu), so that the same source also builds for the
// host under the test suite's shim.

#pragma once

#include <math.h>
#include <stdint.h>

#include "device_common.cuh"

namespace gsparc {
namespace {

struct W {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};

template <int HD>
struct WSmem {
    static constexpr int kW1 = 0;
    static constexpr int kB1 = kW1 + GSPARC_MLP_IN * HD;
    static constexpr int kW2 = kB1 + HD;
    static constexpr int kB2 = kW2 + HD * HD;
    static constexpr int kW3 = kB2 + HD;
    static constexpr int kB3 = kW3 + HD * 3;
    static constexpr int kTotal = kB3 + 4;
};

template <int HD>
__device__ __forceinline__ void load_weights(const W& w, float* sw) {
    using L = WSmem<HD>;
    for (int t = threadIdx.x; t < GSPARC_MLP_IN * HD; t += blockDim.x) sw[L::kW1 + t] = w.W1[t];
    for (int t = threadIdx.x; t < HD * HD; t += blockDim.x) sw[L::kW2 + t] = w.W2[t];
    for (int t = threadIdx.x; t < HD * 3; t += blockDim.x) sw[L::kW3 + t] = w.W3[t];
    for (int t = threadIdx.x; t < HD; t += blockDim.x) {
        sw[L::kB1 + t] = w.b1[t];
        sw[L::kB2 + t] = w.b2[t];
    }
    if (threadIdx.x < 3) sw[L::kB3 + threadIdx.x] = w.b3[threadIdx.x];
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

struct RowIn {
    float t0, t1, t2;      // transmitter
    float m0, m1, m2;      // mean
    float dist, d, logd;   // raw and clamped distance to the transmitter, ln d
    float r;               // |mu - rx|
};

__device__ __forceinline__ RowIn row_inputs(const float* __restrict__ tx, const float* __restrict__ means,
                                            int b, int i, float rx0, float rx1, float rx2) {
    RowIn in;
    in.t0 = tx[3 * b + 0];
    in.t1 = tx[3 * b + 1];
    in.t2 = tx[3 * b + 2];
    in.m0 = means[3 * i + 0];
    in.m1 = means[3 * i + 1];
    in.m2 = means[3 * i + 2];
    const float e0 = in.m0 - in.t0, e1 = in.m1 - in.t1, e2 = in.m2 - in.t2;
    in.dist = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
    in.d = fmaxf(in.dist, kDMin);
    in.logd = logf(in.d);
    const float f0 = in.m0 - rx0, f1 = in.m1 - rx1, f2 = in.m2 - rx2;
    in.r = sqrtf(f0 * f0 + f1 * f1 + f2 * f2);
    return in;
}

__device__ __forceinline__ void load_h0(const RowIn& in, const float* __restrict__ latent, int i,
                                        float h0[GSPARC_MLP_IN]) {
    h0[0] = in.t0;
    h0[1] = in.t1;
    h0[2] = in.t2;
    const float4* l4 = reinterpret_cast<const float4*>(latent + (size_t)i * GSPARC_LATENT);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = l4[q];
        h0[3 + 4 * q + 0] = v.x;
        h0[3 + 4 * q + 1] = v.y;
        h0[3 + 4 * q + 2] = v.z;
        h0[3 + 4 * q + 3] = v.w;
    }
    h0[19] = in.logd;
}

template <int HD>
__global__ void __launch_bounds__(128) k_mlp_fwd(int N, int B, const float* __restrict__ tx, float rx0,
                                                 float rx1, float rx2, const float* __restrict__ means,
                                                 const float* __restrict__ ologit,
                                                 const float* __restrict__ latent, W w,
                                                 float4* __restrict__ attr) {
    using L = WSmem<HD>;
    __shared__ float sw[L::kTotal];
    load_weights<HD>(w, sw);
    __syncthreads();
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (int64_t)N * B) return;
    const int b = (int)(row / N), i = (int)(row - (int64_t)b * N);
    const RowIn in = row_inputs(tx, means, b, i, rx0, rx1, rx2);
    float h0[GSPARC_MLP_IN];
    load_h0(in, latent, i, h0);
    float h1[HD];
#pragma unroll
    for (int j = 0; j < HD; ++j) {
        float acc = sw[L::kB1 + j];
#pragma unroll
        for (int f = 0; f < GSPARC_MLP_IN; ++f) acc = fmaf(h0[f], sw[L::kW1 + f * HD + j], acc);
        h1[j] = fmaxf(acc, 0.f);
    }
    float o0 = sw[L::kB3 + 0], o1 = sw[L::kB3 + 1], o2 = sw[L::kB3 + 2];
#pragma unroll 4
    for (int j2 = 0; j2 < HD; ++j2) {
        float acc = sw[L::kB2 + j2];
#pragma unroll
        for (int j = 0; j < HD; ++j) acc = fmaf(h1[j], sw[L::kW2 + j * HD + j2], acc);
        const float h2 = fmaxf(acc, 0.f);
        o0 = fmaf(h2, sw[L::kW3 + j2 * 3 + 0], o0);
        o1 = fmaf(h2, sw[L::kW3 + j2 * 3 + 1], o1);
        o2 = fmaf(h2, sw[L::kW3 + j2 * 3 + 2], o2);
    }
    const float a = sigmoidf_(o0 - in.logd) / in.d;
    const float sig = sigmoidf_(ologit[i] + o2);
    attr[row] = make_float4(a, o1, sig, in.d + in.r);
}

constexpr int kBwdRows = 128;

// Shared memory of the backward (floats).  Weights as the forward reads them plus transposed
// copies (W1T [HD][20], W2T [HD][HD]) so that every product reads four consecutive weights per
// load; W3 padded to [HD][4].  Per pass, the rows' vectors the weight gradients need, row-major
// with a stride of n + 4 (so that 8 consecutive threads storing 16 bytes each hit distinct banks):
// the factors h0 | 1, h1 | 1, h2 | 1 (a column of ones gives the bias gradients) and the
// gradients du1, du2, dL/do.
template <int HD>
struct BwdSmem {
    static constexpr int kW1 = 0;                          // [20][HD]
    static constexpr int kW1T = kW1 + GSPARC_MLP_IN * HD;  // [HD][20]
    static constexpr int kW2 = kW1T + HD * GSPARC_MLP_IN;  // [HD][HD]
    static constexpr int kW2T = kW2 + HD * HD;             // [HD][HD]
    static constexpr int kW3 = kW2T + HD * HD;             // [HD][4]
    static constexpr int kB1 = kW3 + HD * 4;
    static constexpr int kB2 = kB1 + HD;
    static constexpr int kB3 = kB2 + HD;                   // [4]
    static constexpr int kN0 = 24, kN1 = HD + 4, kN3 = 4;  // columns of h0 | 1, h1 | 1 (h2 | 1), do
    static constexpr int kS0 = kN0 + 4, kS1 = kN1 + 4, kSG = HD + 4, kS3 = kN3 + 4;   // row strides
    static constexpr int kA0 = kB3 + 4;                    // [rows][kS0]  h0 | 1
    static constexpr int kA1 = kA0 + kBwdRows * kS0;       // [rows][kS1]  h1 | 1
    static constexpr int kA2 = kA1 + kBwdRows * kS1;       // [rows][kS1]  h2 | 1
    static constexpr int kG1 = kA2 + kBwdRows * kS1;       // [rows][kSG]  du1
    static constexpr int kG2 = kG1 + kBwdRows * kSG;       // [rows][kSG]  du2
    static constexpr int kG3 = kG2 + kBwdRows * kSG;       // [rows][kS3]  dL/do
    static constexpr int kTotal = kG3 + kBwdRows * kS3;
    // 4x4 blocks of the three weight-gradient outer products (bias gradients in the ones column)
    static constexpr int kBlk1 = (kN0 / 4) * (HD / 4);
    static constexpr int kBlk2 = (kN1 / 4) * (HD / 4);
    static constexpr int kBlk3 = kN1 / 4;
    static constexpr int kBlocks = kBlk1 + kBlk2 + kBlk3;
    static constexpr int kPer = (kBlocks + kBwdRows - 1) / kBwdRows;   // blocks per thread
    static_assert(HD % 4 == 0, "hidden width a multiple of 4");
    static_assert(kA0 % 4 == 0 && kA1 % 4 == 0 && kG1 % 4 == 0 && kG3 % 4 == 0 && kW3 % 4 == 0, "16-byte rows");
};

// One 4x4 block of a weight-gradient outer product sum_r a[r][p0..p0+3] (x) g[r][q0..q0+3].
struct GBlk {
    int a_off, a_stride, g_off, g_stride;   // staging arrays (floats) and their row strides
    int p0, q0;                             // first column of each factor
};

template <int HD>
__device__ __forceinline__ GBlk grad_block(int blk) {
    using S = BwdSmem<HD>;
    GBlk g;
    if (blk < S::kBlk1) {
        g.a_off = S::kA0; g.a_stride = S::kS0; g.g_off = S::kG1; g.g_stride = S::kSG;
        g.p0 = 4 * (blk / (HD / 4)); g.q0 = 4 * (blk % (HD / 4));
    } else if (blk < S::kBlk1 + S::kBlk2) {
        const int e = blk - S::kBlk1;
        g.a_off = S::kA1; g.a_stride = S::kS1; g.g_off = S::kG2; g.g_stride = S::kSG;
        g.p0 = 4 * (e / (HD / 4)); g.q0 = 4 * (e % (HD / 4));
    } else {
        const int e = blk - S::kBlk1 - S::kBlk2;
        g.a_off = S::kA2; g.a_stride = S::kS1; g.g_off = S::kG3; g.g_stride = S::kS3;
        g.p0 = 4 * e; g.q0 = 0;
    }
    return g;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// Persistent CTAs of 128 threads; each pass takes 128 rows (one per thread).  A thread
// recomputes its row's activations in registers (weights read four at a time), stages the
// per-row vectors the weight gradients need in shared memory, and after a barrier adds the pass's
// 128 rows into the 4x4 weight-gradient blocks it owns, kept in registers across passes (16
// FMAs per two 16-byte loads).  One atomic per weight entry per CTA at the end.
template <int HD>
__global__ void __launch_bounds__(kBwdRows) k_mlp_bwd(int N, int B, const float* __restrict__ tx,
                                                      float rx0, float rx1, float rx2,
                                                      const float* __restrict__ means,
                                                      const float* __restrict__ ologit,
                                                      const float* __restrict__ latent, W w,
                                                      const float4* __restrict__ d_attr,
                                                      float* __restrict__ d_means,
                                                      float* __restrict__ d_ologit,
                                                      float* __restrict__ d_latent, gsparc_mlp_grad g) {
    using S = BwdSmem<HD>;
    constexpr int IN = GSPARC_MLP_IN;
    GSPARC_DYNAMIC_SMEM(sm_raw);
    float* sm = reinterpret_cast<float*>(sm_raw);
    const int t = threadIdx.x;
    for (int e = t; e < IN * HD; e += kBwdRows) {
        const float v = w.W1[e];
        sm[S::kW1 + e] = v;
        sm[S::kW1T + (e % HD) * IN + e / HD] = v;
    }
    for (int e = t; e < HD * HD; e += kBwdRows) {
        const float v = w.W2[e];
        sm[S::kW2 + e] = v;
        sm[S::kW2T + (e % HD) * HD + e / HD] = v;
    }
    for (int e = t; e < HD * 4; e += kBwdRows) sm[S::kW3 + e] = (e & 3) < 3 ? w.W3[(e >> 2) * 3 + (e & 3)] : 0.f;
    for (int e = t; e < HD; e += kBwdRows) {
        sm[S::kB1 + e] = w.b1[e];
        sm[S::kB2 + e] = w.b2[e];
    }
    if (t < 4) sm[S::kB3 + t] = t < 3 ? w.b3[t] : 0.f;
    float acc[S::kPer][16];
#pragma unroll
    for (int m = 0; m < S::kPer; ++m)
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[m][q] = 0.f;
    const int64_t rows = (int64_t)N * B;
    const int64_t tiles = (rows + kBwdRows - 1) / kBwdRows;
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row = tile * kBwdRows + t;
        float* a0 = sm + S::kA0 + t * S::kS0;
        float* a1 = sm + S::kA1 + t * S::kS1;
        float* a2 = sm + S::kA2 + t * S::kS1;
        float* g1 = sm + S::kG1 + t * S::kSG;
        float* g2 = sm + S::kG2 + t * S::kSG;
        float* g3 = sm + S::kG3 + t * S::kS3;
        if (row < rows) {
            const int b = (int)(row / N), i = (int)(row - (int64_t)b * N);
            const RowIn in = row_inputs(tx, means, b, i, rx0, rx1, rx2);
            float h0[IN];
            load_h0(in, latent, i, h0);
#pragma unroll
            for (int f = 0; f < IN; f += 4) st4(a0 + f, h0[f], h0[f + 1], h0[f + 2], h0[f + 3]);
            st4(a0 + IN, 1.f, 0.f, 0.f, 0.f);
            // h1 = relu(h0 W1 + b1)
            float h1[HD];
#pragma unroll
            for (int j = 0; j < HD; j += 4) {
                const float4 bb = ld4(sm + S::kB1 + j);
                h1[j] = bb.x; h1[j + 1] = bb.y; h1[j + 2] = bb.z; h1[j + 3] = bb.w;
            }
#pragma unroll
            for (int f = 0; f < IN; ++f) {
#pragma unroll
                for (int j = 0; j < HD; j += 4) {
                    const float4 wv = ld4(sm + S::kW1 + f * HD + j);
                    h1[j] = fmaf(h0[f], wv.x, h1[j]);
                    h1[j + 1] = fmaf(h0[f], wv.y, h1[j + 1]);
                    h1[j + 2] = fmaf(h0[f], wv.z, h1[j + 2]);
                    h1[j + 3] = fmaf(h0[f], wv.w, h1[j + 3]);
                }
            }
#pragma unroll
            for (int j = 0; j < HD; ++j) h1[j] = fmaxf(h1[j], 0.f);
#pragma unroll
            for (int j = 0; j < HD; j += 4) st4(a1 + j, h1[j], h1[j + 1], h1[j + 2], h1[j + 3]);
            st4(a1 + HD, 1.f, 0.f, 0.f, 0.f);
            // h2 = relu(h1 W2 + b2), then the outputs
            float v[HD];
#pragma unroll
            for (int j = 0; j < HD; j += 4) {
                const float4 bb = ld4(sm + S::kB2 + j);
                v[j] = bb.x; v[j + 1] = bb.y; v[j + 2] = bb.z; v[j + 3] = bb.w;
            }
#pragma unroll
            for (int j = 0; j < HD; ++j) {
#pragma unroll
                for (int j2 = 0; j2 < HD; j2 += 4) {
                    const float4 wv = ld4(sm + S::kW2 + j * HD + j2);
                    v[j2] = fmaf(h1[j], wv.x, v[j2]);
                    v[j2 + 1] = fmaf(h1[j], wv.y, v[j2 + 1]);
                    v[j2 + 2] = fmaf(h1[j], wv.z, v[j2 + 2]);
                    v[j2 + 3] = fmaf(h1[j], wv.w, v[j2 + 3]);
                }
            }
            float o0 = sm[S::kB3 + 0], o2 = sm[S::kB3 + 2];
#pragma unroll
            for (int j2 = 0; j2 < HD; ++j2) {
                v[j2] = fmaxf(v[j2], 0.f);
                const float4 w3 = ld4(sm + S::kW3 + j2 * 4);
                o0 = fmaf(v[j2], w3.x, o0);
                o2 = fmaf(v[j2], w3.z, o2);
            }
#pragma unroll
            for (int j = 0; j < HD; j += 4) st4(a2 + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
            st4(a2 + HD, 1.f, 0.f, 0.f, 0.f);
            const float s0 = sigmoidf_(o0 - in.logd);
            const float sig = sigmoidf_(ologit[i] + o2);
            const float4 da = d_attr[row];   // d a, d phi0, d sigma, d L
            const float do0 = da.x * s0 * (1.f - s0) / in.d;
            const float do1 = da.y;
            const float do2 = da.z * sig * (1.f - sig);
            st4(g3, do0, do1, do2, 0.f);
            atomicAdd(&d_ologit[i], do2);
            // du2 = (W3 do) masked by the second ReLU
#pragma unroll
            for (int j2 = 0; j2 < HD; ++j2) {
                const float4 w3 = ld4(sm + S::kW3 + j2 * 4);
                const float dh2 = w3.x * do0 + w3.y * do1 + w3.z * do2;
                v[j2] = v[j2] > 0.f ? dh2 : 0.f;
            }
#pragma unroll
            for (int j = 0; j < HD; j += 4) st4(g2 + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
            // du1 = (W2 du2) masked by the first ReLU (W2T rows: four consecutive j per load)
            float dh1[HD];
#pragma unroll
            for (int j = 0; j < HD; ++j) dh1[j] = 0.f;
#pragma unroll
            for (int j2 = 0; j2 < HD; ++j2) {
#pragma unroll
                for (int j = 0; j < HD; j += 4) {
                    const float4 wv = ld4(sm + S::kW2T + j2 * HD + j);
                    dh1[j] = fmaf(wv.x, v[j2], dh1[j]);
                    dh1[j + 1] = fmaf(wv.y, v[j2], dh1[j + 1]);
                    dh1[j + 2] = fmaf(wv.z, v[j2], dh1[j + 2]);
                    dh1[j + 3] = fmaf(wv.w, v[j2], dh1[j + 3]);
                }
            }
#pragma unroll
            for (int j = 0; j < HD; ++j) dh1[j] = h1[j] > 0.f ? dh1[j] : 0.f;
#pragma unroll
            for (int j = 0; j < HD; j += 4) st4(g1 + j, dh1[j], dh1[j + 1], dh1[j + 2], dh1[j + 3]);
            // dL/dh0 for the latents and ln d (W1T rows: the 20 inputs of hidden unit j)
            float dh0[IN];
#pragma unroll
            for (int f = 0; f < IN; ++f) dh0[f] = 0.f;
#pragma unroll
            for (int j = 0; j < HD; ++j) {
#pragma unroll
                for (int f = 0; f < IN; f += 4) {
                    const float4 wv = ld4(sm + S::kW1T + j * IN + f);
                    dh0[f] = fmaf(wv.x, dh1[j], dh0[f]);
                    dh0[f + 1] = fmaf(wv.y, dh1[j], dh0[f + 1]);
                    dh0[f + 2] = fmaf(wv.z, dh1[j], dh0[f + 2]);
                    dh0[f + 3] = fmaf(wv.w, dh1[j], dh0[f + 3]);
                }
            }
#pragma unroll
            for (int f = 0; f < GSPARC_LATENT; ++f) atomicAdd(&d_latent[(size_t)i * GSPARC_LATENT + f], dh0[3 + f]);
            // a = sigmoid(o0 - ln d)/d: explicit ln d (-do0), network input ln d, L = d + r
            const float dlogd = -do0 + dh0[IN - 1];
            const float dd = da.x * (-s0 / (in.d * in.d)) + da.w + dlogd / in.d;
            float gm0 = 0.f, gm1 = 0.f, gm2 = 0.f;
            if (in.dist > kDMin) {
                const float f = dd / in.dist;
                gm0 += f * (in.m0 - in.t0);
                gm1 += f * (in.m1 - in.t1);
                gm2 += f * (in.m2 - in.t2);
            }
            if (in.r > 0.f) {
                const float f = da.w / in.r;
                gm0 += f * (in.m0 - rx0);
                gm1 += f * (in.m1 - rx1);
                gm2 += f * (in.m2 - rx2);
            }
            atomicAdd(&d_means[3 * i + 0], gm0);
            atomicAdd(&d_means[3 * i + 1], gm1);
            atomicAdd(&d_means[3 * i + 2], gm2);
        } else {
            // a row past the end contributes nothing (its ones column is 0 too)
#pragma unroll
            for (int f = 0; f < S::kN0; f += 4) st4(a0 + f, 0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < S::kN1; j += 4) {
                st4(a1 + j, 0.f, 0.f, 0.f, 0.f);
                st4(a2 + j, 0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < HD; j += 4) {
                st4(g1 + j, 0.f, 0.f, 0.f, 0.f);
                st4(g2 + j, 0.f, 0.f, 0.f, 0.f);
            }
            st4(g3, 0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        // this pass's 128 rows into the thread's 4x4 blocks
#pragma unroll
        for (int m = 0; m < S::kPer; ++m) {
            const int blk = t + kBwdRows * m;
            if (blk < S::kBlocks) {
                const GBlk gb = grad_block<HD>(blk);
                const float* pa = sm + gb.a_off + gb.p0;
                const float* pg = sm + gb.g_off + gb.q0;
#pragma unroll 4
                for (int r = 0; r < kBwdRows; ++r) {
                    const float4 x = ld4(pa + r * gb.a_stride);
                    const float4 y = ld4(pg + r * gb.g_stride);
                    const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[m][4 * p + q] = fmaf(xs[p], ys[q], acc[m][4 * p + q]);
                }
            }
        }
        __syncthreads();
    }
    // one atomic per entry: rows of the first factor are weight rows, its ones column the bias
#pragma unroll
    for (int m = 0; m < S::kPer; ++m) {
        const int blk = t + kBwdRows * m;
        if (blk >= S::kBlocks) continue;
        const GBlk gb = grad_block<HD>(blk);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int fr = gb.p0 + p, c = gb.q0 + q;
                const float v = acc[m][4 * p + q];
                if (blk < S::kBlk1) {
                    if (fr < IN) atomicAdd(&g.W1[fr * HD + c], v);
                    else if (fr == IN) atomicAdd(&g.b1[c], v);
                } else if (blk < S::kBlk1 + S::kBlk2) {
                    if (fr < HD) atomicAdd(&g.W2[fr * HD + c], v);
                    else if (fr == HD) atomicAdd(&g.b2[c], v);
                } else if (c < 3) {
                    if (fr < HD) atomicAdd(&g.W3[fr * 3 + c], v);
                    else if (fr == HD) atomicAdd(&g.b3[c], v);
                }
            }
        }
    }
}

}  // namespace
}  // namespace gsparc
