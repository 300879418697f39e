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
constexpr int kRS = kBwdRows + 1;   // padded stride of the row-minor staging arrays

template <int HD>
struct BwdSmem {
    static constexpr int kH0 = WSmem<HD>::kTotal;
    static constexpr int kH1 = kH0 + GSPARC_MLP_IN * kRS;
    static constexpr int kDU1 = kH1 + HD * kRS;
    static constexpr int kH2 = kDU1 + HD * kRS;
    static constexpr int kDU2 = kH2 + HD * kRS;
    static constexpr int kDO = kDU2 + HD * kRS;
    static constexpr int kTotal = kDO + 3 * kRS;
};

// Weight-gradient entries owned by one thread: entry e = t + kBwdRows * m.
template <int COUNT>
struct Owned {
    static constexpr int kPer = (COUNT + kBwdRows - 1) / kBwdRows;
};

// Persistent CTAs of 128 threads; each pass takes 128 rows (one per thread).  A thread
// recomputes its row's activations in registers (independent accumulators, fully
// unrolled), stages the per-row vectors needed by the weight gradients in shared memory,
// and after a barrier adds the CTA's 128 rows into weight-gradient partials it keeps in
// registers across passes.  One atomic per weight entry per CTA at the end.
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
    using L = WSmem<HD>;
    using S = BwdSmem<HD>;
    constexpr int kP1 = Owned<GSPARC_MLP_IN * HD>::kPer;
    constexpr int kP2 = Owned<HD * HD>::kPer;
    constexpr int kP3 = Owned<HD * 3>::kPer;
    GSPARC_DYNAMIC_SMEM(sm_raw);
    float* sm = reinterpret_cast<float*>(sm_raw);
    float* sw = sm;
    load_weights<HD>(w, sw);
    const int t = threadIdx.x;
    float aW1[kP1], aW2[kP2], aW3[kP3], ab1 = 0.f, ab2 = 0.f, ab3 = 0.f;
#pragma unroll
    for (int m = 0; m < kP1; ++m) aW1[m] = 0.f;
#pragma unroll
    for (int m = 0; m < kP2; ++m) aW2[m] = 0.f;
#pragma unroll
    for (int m = 0; m < kP3; ++m) aW3[m] = 0.f;
    const int64_t rows = (int64_t)N * B;
    const int64_t tiles = (rows + kBwdRows - 1) / kBwdRows;
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row = tile * kBwdRows + t;
        if (row < rows) {
            const int b = (int)(row / N), i = (int)(row - (int64_t)b * N);
            const RowIn in = row_inputs(tx, means, b, i, rx0, rx1, rx2);
            float h0[GSPARC_MLP_IN];
            load_h0(in, latent, i, h0);
#pragma unroll
            for (int f = 0; f < GSPARC_MLP_IN; ++f) sm[S::kH0 + f * kRS + t] = h0[f];
            float h1[HD];
#pragma unroll
            for (int j = 0; j < HD; ++j) {
                float acc = sw[L::kB1 + j];
#pragma unroll
                for (int f = 0; f < GSPARC_MLP_IN; ++f) acc = fmaf(h0[f], sw[L::kW1 + f * HD + j], acc);
                h1[j] = fmaxf(acc, 0.f);
                sm[S::kH1 + j * kRS + t] = h1[j];
            }
            float v[HD];   // h2, then du2
#pragma unroll
            for (int j2 = 0; j2 < HD; ++j2) v[j2] = sw[L::kB2 + j2];
#pragma unroll
            for (int j = 0; j < HD; ++j) {
#pragma unroll
                for (int j2 = 0; j2 < HD; ++j2) v[j2] = fmaf(h1[j], sw[L::kW2 + j * HD + j2], v[j2]);
            }
            float o0 = sw[L::kB3 + 0], o2 = sw[L::kB3 + 2];
#pragma unroll
            for (int j2 = 0; j2 < HD; ++j2) {
                v[j2] = fmaxf(v[j2], 0.f);
                sm[S::kH2 + j2 * kRS + t] = v[j2];
                o0 = fmaf(v[j2], sw[L::kW3 + j2 * 3 + 0], o0);
                o2 = fmaf(v[j2], sw[L::kW3 + j2 * 3 + 2], o2);
            }
            const float s0 = sigmoidf_(o0 - in.logd);
            const float sig = sigmoidf_(ologit[i] + o2);
            const float4 da = d_attr[row];   // d a, d phi0, d sigma, d L
            const float do0 = da.x * s0 * (1.f - s0) / in.d;
            const float do1 = da.y;
            const float do2 = da.z * sig * (1.f - sig);
            sm[S::kDO + 0 * kRS + t] = do0;
            sm[S::kDO + 1 * kRS + t] = do1;
            sm[S::kDO + 2 * kRS + t] = do2;
            atomicAdd(&d_ologit[i], do2);
#pragma unroll
            for (int j2 = 0; j2 < HD; ++j2) {
                const float dh2 = sw[L::kW3 + j2 * 3 + 0] * do0 + sw[L::kW3 + j2 * 3 + 1] * do1 +
                                  sw[L::kW3 + j2 * 3 + 2] * do2;
                v[j2] = v[j2] > 0.f ? dh2 : 0.f;
                sm[S::kDU2 + j2 * kRS + t] = v[j2];
            }
            float dh1[HD];
#pragma unroll
            for (int j = 0; j < HD; ++j) dh1[j] = 0.f;
#pragma unroll
            for (int j2 = 0; j2 < HD; ++j2) {
#pragma unroll
                for (int j = 0; j < HD; ++j) dh1[j] = fmaf(sw[L::kW2 + j * HD + j2], v[j2], dh1[j]);
            }
#pragma unroll
            for (int j = 0; j < HD; ++j) {
                dh1[j] = h1[j] > 0.f ? dh1[j] : 0.f;
                sm[S::kDU1 + j * kRS + t] = dh1[j];
            }
            float dh0[GSPARC_MLP_IN - 3];
#pragma unroll
            for (int f = 0; f < GSPARC_MLP_IN - 3; ++f) dh0[f] = 0.f;
#pragma unroll
            for (int j = 0; j < HD; ++j) {
#pragma unroll
                for (int f = 0; f < GSPARC_MLP_IN - 3; ++f)
                    dh0[f] = fmaf(sw[L::kW1 + (f + 3) * HD + j], dh1[j], dh0[f]);
            }
#pragma unroll
            for (int f = 0; f < GSPARC_LATENT; ++f) atomicAdd(&d_latent[(size_t)i * GSPARC_LATENT + f], dh0[f]);
            // a = sigmoid(o0 - ln d)/d: explicit ln d (-do0), network input ln d, L = d + r
            const float dlogd = -do0 + dh0[GSPARC_MLP_IN - 4];
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
#pragma unroll
            for (int f = 0; f < GSPARC_MLP_IN; ++f) sm[S::kH0 + f * kRS + t] = 0.f;
#pragma unroll
            for (int j = 0; j < HD; ++j) {
                sm[S::kH1 + j * kRS + t] = 0.f;
                sm[S::kH2 + j * kRS + t] = 0.f;
                sm[S::kDU1 + j * kRS + t] = 0.f;
                sm[S::kDU2 + j * kRS + t] = 0.f;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) sm[S::kDO + c * kRS + t] = 0.f;
        }
        __syncthreads();
        // this pass's 128 rows into the register partials
#pragma unroll
        for (int m = 0; m < kP1; ++m) {
            const int e = t + kBwdRows * m;
            if (e < GSPARC_MLP_IN * HD) {
                const int f = e / HD, j = e - f * HD;
                float acc = aW1[m];
                for (int r = 0; r < kBwdRows; ++r) acc = fmaf(sm[S::kH0 + f * kRS + r], sm[S::kDU1 + j * kRS + r], acc);
                aW1[m] = acc;
            }
        }
#pragma unroll
        for (int m = 0; m < kP2; ++m) {
            const int e = t + kBwdRows * m;
            if (e < HD * HD) {
                const int j = e / HD, j2 = e - j * HD;
                float acc = aW2[m];
                for (int r = 0; r < kBwdRows; ++r) acc = fmaf(sm[S::kH1 + j * kRS + r], sm[S::kDU2 + j2 * kRS + r], acc);
                aW2[m] = acc;
            }
        }
#pragma unroll
        for (int m = 0; m < kP3; ++m) {
            const int e = t + kBwdRows * m;
            if (e < HD * 3) {
                const int j2 = e / 3, c = e - j2 * 3;
                float acc = aW3[m];
                for (int r = 0; r < kBwdRows; ++r) acc = fmaf(sm[S::kH2 + j2 * kRS + r], sm[S::kDO + c * kRS + r], acc);
                aW3[m] = acc;
            }
        }
        if (t < HD) {
            for (int r = 0; r < kBwdRows; ++r) {
                ab1 += sm[S::kDU1 + t * kRS + r];
                ab2 += sm[S::kDU2 + t * kRS + r];
            }
        }
        if (t < 3) {
            for (int r = 0; r < kBwdRows; ++r) ab3 += sm[S::kDO + t * kRS + r];
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < kP1; ++m) {
        const int e = t + kBwdRows * m;
        if (e < GSPARC_MLP_IN * HD) atomicAdd(&g.W1[e], aW1[m]);
    }
#pragma unroll
    for (int m = 0; m < kP2; ++m) {
        const int e = t + kBwdRows * m;
        if (e < HD * HD) atomicAdd(&g.W2[e], aW2[m]);
    }
#pragma unroll
    for (int m = 0; m < kP3; ++m) {
        const int e = t + kBwdRows * m;
        if (e < HD * 3) atomicAdd(&g.W3[e], aW3[m]);
    }
    if (t < HD) {
        atomicAdd(&g.b1[t], ab1);
        atomicAdd(&g.b2[t], ab2);
    }
    if (t < 3) atomicAdd(&g.b3[t], ab3);
}

}  // namespace
}  // namespace gsparc
