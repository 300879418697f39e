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
// Backward: persistent CTAs over tiles of 64 rows; the forward is recomputed and
// the gradients formed as tile products over shared-memory operands stored
// feature-major (bank-permuted), and every CTA keeps its weight-gradient
// partials in registers until one atomic per entry at the end.
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

// One thread per (transmitter, Gaussian) row.  KEEP: the row's post-ReLU activations h1 and h2
// stored feature-major, hidden[j * ld + row] = h1_j and hidden[(HD + j) * ld + row] = h2_j, for
// the backward to read instead of recomputing them (a separate instantiation, so that the form
// without them compiles to the plain loops).
template <int HD, bool KEEP = false>
__global__ void __launch_bounds__(128) k_mlp_fwd(int N, int B, const float* __restrict__ tx, float rx0,
                                                 float rx1, float rx2, const float* __restrict__ means,
                                                 const float* __restrict__ ologit,
                                                 const float* __restrict__ latent, W w,
                                                 float4* __restrict__ attr, float* __restrict__ hidden,
                                                 int64_t ld) {
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
        if constexpr (KEEP) hidden[(size_t)j * ld + row] = h1[j];
    }
    float o0 = sw[L::kB3 + 0], o1 = sw[L::kB3 + 1], o2 = sw[L::kB3 + 2];
#pragma unroll 4
    for (int j2 = 0; j2 < HD; ++j2) {
        float acc = sw[L::kB2 + j2];
#pragma unroll
        for (int j = 0; j < HD; ++j) acc = fmaf(h1[j], sw[L::kW2 + j * HD + j2], acc);
        const float h2 = fmaxf(acc, 0.f);
        if constexpr (KEEP) hidden[(size_t)(HD + j2) * ld + row] = h2;
        o0 = fmaf(h2, sw[L::kW3 + j2 * 3 + 0], o0);
        o1 = fmaf(h2, sw[L::kW3 + j2 * 3 + 1], o1);
        o2 = fmaf(h2, sw[L::kW3 + j2 * 3 + 2], o2);
    }
    const float a = sigmoidf_(o0 - in.logd) / in.d;
    const float sig = sigmoidf_(ologit[i] + o2);
    attr[row] = make_float4(a, o1, sig, in.d + in.r);
}

constexpr int kBwdRows = 64;       // rows (Gaussian, transmitter) per tile of the backward
constexpr int kBwdThreads = 128;   // threads per CTA of the backward

// Shared memory of the backward (floats).  Weights as the forward reads them plus transposed
// copies (W1T [HD][20], W2T [HD][HD]), W3 padded to [HD][4].  Per tile, every per-row vector is
// stored feature-major, one row of kBwdRows floats per feature, with the 4-row groups of a
// feature row permuted by an XOR of the feature index (fm4 below): a warp reading 8 consecutive
// row groups of one feature, or one row group of features 4 apart, touches 8 distinct bank
// quads.  A0 = h0 | 1 | 0 0 0, A1 = h1 | 1 | 0 0 0, A2 = h2 | 1 | 0 0 0 (a row of ones gives the
// bias gradients), G1 = du1, G2 = du2, G3 = dL/do | 0, D0 = dL/dh0.
template <int HD>
struct BwdSmem {
    static constexpr int IN = GSPARC_MLP_IN;
    static constexpr int kW1 = 0;                      // [20][HD]
    static constexpr int kW1T = kW1 + IN * HD;         // [HD][20]
    static constexpr int kW2 = kW1T + HD * IN;         // [HD][HD]
    static constexpr int kW2T = kW2 + HD * HD;         // [HD][HD]
    static constexpr int kW3 = kW2T + HD * HD;         // [HD][4]
    static constexpr int kB1 = kW3 + HD * 4;
    static constexpr int kB2 = kB1 + HD;
    static constexpr int kB3 = kB2 + HD;               // [4]
    static constexpr int kF0 = IN + 4, kF1 = HD + 4;   // feature rows of A0 and of A1, A2
    static constexpr int kA0 = kB3 + 4;
    static constexpr int kA1 = kA0 + kF0 * kBwdRows;
    static constexpr int kA2 = kA1 + kF1 * kBwdRows;
    static constexpr int kG1 = kA2 + kF1 * kBwdRows;
    static constexpr int kG2 = kG1 + HD * kBwdRows;
    static constexpr int kG3 = kG2 + HD * kBwdRows;
    static constexpr int kD0 = kG3 + 4 * kBwdRows;
    static constexpr int kTotal = kD0 + IN * kBwdRows;
    // 4x4 blocks of the weight-gradient products: (h0 | 1)^T du1, (h1 | 1)^T du2, h2^T dL/do (the
    // bias of the last layer is the column sum of dL/do, reduced over the warps of the rows)
    static constexpr int kBlk1 = (kF0 / 4) * (HD / 4);
    static constexpr int kBlk2 = (kF1 / 4) * (HD / 4);
    static constexpr int kBlk3 = HD / 4;
    static constexpr int kBlocks = kBlk1 + kBlk2 + kBlk3;
    static constexpr int kPer = (kBlocks + kBwdThreads - 1) / kBwdThreads;
    static_assert(HD % 8 == 0 && HD <= 64, "hidden width 8, 16, 32 or 64");
    static_assert(kW1T % 4 == 0 && kW3 % 4 == 0 && kA0 % 4 == 0 && kA1 % 4 == 0 && kG1 % 4 == 0, "16-byte rows");
};
static_assert(kBwdRows == 64 && kBwdThreads == 128, "tile products: 16 row groups x 8 column groups");
#ifdef GSPARC_HOST_SHIM
constexpr bool kHostShim = true;    // the test suite's host shim has no bulk copies: atomics
#else
constexpr bool kHostShim = false;
#endif

// Offset of rows r..r+3 (r a multiple of 4) of feature x in a feature-major array.
__device__ __forceinline__ int fm4(int x, int r) { return x * kBwdRows + (((r >> 2) ^ ((x >> 2) & 7)) << 2); }
__device__ __forceinline__ int fm(int x, int r) { return fm4(x, r & ~3) + (r & 3); }

// A tile's stored activations (features 0..HD-1 of A1 and A2, from k_mlp_fwd's `hidden`) into
// shared memory: a 16-byte asynchronous copy (cp.async: no registers held while it is in flight)
// per 4-row group inside the rows, zeros past them (the padding rows' dL/do is zero, and these
// values multiply it in the weight-gradient sums, so they must be finite).  Sixteen consecutive
// threads read 256 contiguous bytes of one feature.  hidden and ld: 16-byte aligned, ld % 4 == 0.
template <int HD>
__device__ __forceinline__ void fetch_hidden(float* sm, const float* __restrict__ hidden, int64_t ld,
                                             int64_t row0, int64_t rows, int t) {
    using S = BwdSmem<HD>;
    constexpr int G4 = kBwdRows / 4;
    for (int e = t; e < 2 * HD * G4; e += kBwdThreads) {
        const int f = e / G4, gi = e - f * G4;
        const int64_t r = row0 + 4 * gi;
        float* dst = sm + (f < HD ? S::kA1 + fm4(f, 4 * gi) : S::kA2 + fm4(f - HD, 4 * gi));
        const float* src = hidden + (size_t)f * ld + r;
#ifndef GSPARC_HOST_SHIM
        if (r + 4 <= rows) {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                         "l"(src)
                         : "memory");
            continue;
        }
#endif
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = r + q < rows ? src[q] : 0.f;
    }
#ifndef GSPARC_HOST_SHIM
    asm volatile("cp.async.commit_group;" ::: "memory");
#endif
}

// Completion of this thread's fetch_hidden copies (a block barrier then shows them to all).
__device__ __forceinline__ void fetch_hidden_wait() {
#ifndef GSPARC_HOST_SHIM
    asm volatile("cp.async.wait_all;" ::: "memory");
#endif
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// C[r][n] = sum_k A[k][r] Bm[k][n] for the tile's 64 rows and NC = 8 CW columns: the thread
// (rg, cg) accumulates rows 4rg..4rg+3 and columns CW cg..CW cg + CW - 1 (16 FMAs per two 16-byte
// loads at CW = 4).  A is feature-major (fm4), Bm row-major [K][NC].
template <int K, int CW>
__device__ __forceinline__ void tile_mm(const float* __restrict__ A, const float* __restrict__ Bm, int rg, int cg,
                                        float acc[4][CW]) {
    constexpr int NC = 8 * CW;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 a = ld4(A + fm4(k, 4 * rg));
        float b[CW];
        if constexpr (CW % 4 == 0) {
#pragma unroll
            for (int q = 0; q < CW; q += 4) {
                const float4 v = ld4(Bm + k * NC + CW * cg + q);
                b[q] = v.x; b[q + 1] = v.y; b[q + 2] = v.z; b[q + 3] = v.w;
            }
        } else if constexpr (CW == 2) {
            const float2 v = *reinterpret_cast<const float2*>(Bm + k * NC + CW * cg);
            b[0] = v.x; b[1] = v.y;
        } else {
            b[0] = Bm[k * NC + cg];
        }
        const float as[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < CW; ++q) acc[p][q] = fmaf(as[p], b[q], acc[p][q]);
    }
}

// The thread's block of a tile product stored feature-major (one 16-byte store per column).
template <int CW>
__device__ __forceinline__ void tile_store(float* __restrict__ C, int rg, int cg, const float acc[4][CW]) {
#pragma unroll
    for (int q = 0; q < CW; ++q) st4(C + fm4(CW * cg + q, 4 * rg), acc[0][q], acc[1][q], acc[2][q], acc[3][q]);
}

// One 4x4 block of a weight-gradient product sum_r a[p0 + p][r] g[q0 + q][r].
struct GBlk {
    int a_off, g_off, p0, q0;
};

template <int HD>
__device__ __forceinline__ GBlk grad_block(int blk) {
    using S = BwdSmem<HD>;
    GBlk g;
    if (blk < S::kBlk1) {
        g.a_off = S::kA0; g.g_off = S::kG1;
        g.p0 = 4 * (blk / (HD / 4)); g.q0 = 4 * (blk % (HD / 4));
    } else if (blk < S::kBlk1 + S::kBlk2) {
        const int e = blk - S::kBlk1;
        g.a_off = S::kA1; g.g_off = S::kG2;
        g.p0 = 4 * (e / (HD / 4)); g.q0 = 4 * (e % (HD / 4));
    } else {
        g.a_off = S::kA2; g.g_off = S::kG3;
        g.p0 = 4 * (blk - S::kBlk1 - S::kBlk2); g.q0 = 0;
    }
    return g;
}

// A row's raw inputs, loaded one tile ahead of their use.
struct RowRaw {
    float t0, t1, t2, m0, m1, m2;
    float4 lat[GSPARC_LATENT / 4];
    float4 da;   // d a, d phi0, d sigma, d L
    float ol;
};

__device__ __forceinline__ void load_raw(const float* __restrict__ tx, const float* __restrict__ means,
                                         const float* __restrict__ ologit, const float* __restrict__ latent,
                                         const float4* __restrict__ d_attr, int64_t row, int N, RowRaw& x) {
    const int b = (int)(row / N), i = (int)(row - (int64_t)b * N);
    x.t0 = tx[3 * b + 0];
    x.t1 = tx[3 * b + 1];
    x.t2 = tx[3 * b + 2];
    x.m0 = means[3 * i + 0];
    x.m1 = means[3 * i + 1];
    x.m2 = means[3 * i + 2];
    const float4* l4 = reinterpret_cast<const float4*>(latent + (size_t)i * GSPARC_LATENT);
#pragma unroll
    for (int q = 0; q < GSPARC_LATENT / 4; ++q) x.lat[q] = l4[q];
    x.da = d_attr[row];
    x.ol = ologit[i];
}

// Persistent CTAs of 128 threads over tiles of 64 rows.  Per tile: the rows' inputs (one thread
// per row), the forward's activations, recomputed as tile products (h1 = relu(h0 W1 + b1),
// h2 = relu(h1 W2 + b2)) or, with `hidden` (k_mlp_fwd's stored h1 and h2, leading dimension ld),
// copied in asynchronously while the previous tile finishes,
// the outputs and dL/do per row, du2 per row, du1 = (du2 W2^T) . [h1 > 0] and dL/dh0 = du1 W1^T as
// tile products, the weight gradients added into the 4x4 blocks each thread keeps in registers
// across tiles (one atomic per weight entry per CTA at the end), and the per-row input gradients
// (latents, ln d, means) by the row threads.
template <int HD>
__global__ void __launch_bounds__(kBwdThreads, HD <= 32 ? 3 : 1)
    k_mlp_bwd(int N, int B, const float* __restrict__ tx, float rx0, float rx1, float rx2,
              const float* __restrict__ means, const float* __restrict__ ologit, const float* __restrict__ latent,
              W w, const float4* __restrict__ d_attr, float* __restrict__ d_means, float* __restrict__ d_ologit,
              float* __restrict__ d_latent, gsparc_mlp_grad g, const float* __restrict__ hidden, int64_t ld) {
    using S = BwdSmem<HD>;
    constexpr int IN = GSPARC_MLP_IN, R = kBwdRows, CW = HD / 8;
    GSPARC_DYNAMIC_SMEM(sm_raw);
    float* sm = reinterpret_cast<float*>(sm_raw);
    grid_dep_wait();     // the attribute gradients of the compositing backward
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int e = t; e < IN * HD; e += kBwdThreads) {
        const float v = w.W1[e];
        sm[S::kW1 + e] = v;
        sm[S::kW1T + (e % HD) * IN + e / HD] = v;
    }
    for (int e = t; e < HD * HD; e += kBwdThreads) {
        const float v = w.W2[e];
        sm[S::kW2 + e] = v;
        sm[S::kW2T + (e % HD) * HD + e / HD] = v;
    }
    for (int e = t; e < HD * 4; e += kBwdThreads) sm[S::kW3 + e] = (e & 3) < 3 ? w.W3[(e >> 2) * 3 + (e & 3)] : 0.f;
    for (int e = t; e < HD; e += kBwdThreads) {
        sm[S::kB1 + e] = w.b1[e];
        sm[S::kB2 + e] = w.b2[e];
    }
    if (t < 4) sm[S::kB3 + t] = t < 3 ? w.b3[t] : 0.f;
    // the constant feature rows: ones (bias gradients), zeros (padding to 4), dL/do's fourth row
    for (int r = t; r < R; r += kBwdThreads) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sm[S::kA0 + fm(IN + q, r)] = q == 0 ? 1.f : 0.f;
            sm[S::kA1 + fm(HD + q, r)] = q == 0 ? 1.f : 0.f;
            sm[S::kA2 + fm(HD + q, r)] = q == 0 ? 1.f : 0.f;
        }
        sm[S::kG3 + fm(3, r)] = 0.f;
    }
    // tile-product thread layout: a warp covers 8 row groups x 4 column groups
    const int rg = (warp & 1) * 8 + (lane & 7), cg = (warp >> 1) * 4 + (lane >> 3);
    float acc[S::kPer][16];
#pragma unroll
    for (int m = 0; m < S::kPer; ++m)
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[m][q] = 0.f;
    float db3[3] = {0.f, 0.f, 0.f};   // lane 0 of the two row warps
    const int64_t rows = (int64_t)N * B;
    const int64_t tiles = (rows + R - 1) / R;
    const bool rowt = t < R;
    RowRaw nxt{};
    if (rowt && (int64_t)blockIdx.x * R + t < rows)
        load_raw(tx, means, ologit, latent, d_attr, (int64_t)blockIdx.x * R + t, N, nxt);
    if (hidden && (int64_t)blockIdx.x < tiles) fetch_hidden<HD>(sm, hidden, ld, (int64_t)blockIdx.x * R, rows, t);
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        // rows' inputs (threads 0..63, one row each), then the next tile's raw inputs requested
        const int64_t row = tile * R + t;
        const bool valid = rowt && row < rows;
        const RowRaw cur = nxt;
        const int64_t row_next = row + (int64_t)gridDim.x * R;
        if (rowt && row_next < rows) load_raw(tx, means, ologit, latent, d_attr, row_next, N, nxt);
        int i = 0;
        RowIn in{};
        const float4 da = cur.da;
        const float ol = cur.ol;
        if (valid) {
            i = (int)(row % N);
            in.t0 = cur.t0; in.t1 = cur.t1; in.t2 = cur.t2;
            in.m0 = cur.m0; in.m1 = cur.m1; in.m2 = cur.m2;
            const float e0 = in.m0 - in.t0, e1 = in.m1 - in.t1, e2 = in.m2 - in.t2;
            in.dist = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
            in.d = fmaxf(in.dist, kDMin);
            in.logd = logf(in.d);
            const float f0 = in.m0 - rx0, f1 = in.m1 - rx1, f2 = in.m2 - rx2;
            in.r = sqrtf(f0 * f0 + f1 * f1 + f2 * f2);
            sm[S::kA0 + fm(0, t)] = in.t0;
            sm[S::kA0 + fm(1, t)] = in.t1;
            sm[S::kA0 + fm(2, t)] = in.t2;
#pragma unroll
            for (int q = 0; q < GSPARC_LATENT / 4; ++q) {
                sm[S::kA0 + fm(3 + 4 * q, t)] = cur.lat[q].x;
                sm[S::kA0 + fm(4 + 4 * q, t)] = cur.lat[q].y;
                sm[S::kA0 + fm(5 + 4 * q, t)] = cur.lat[q].z;
                sm[S::kA0 + fm(6 + 4 * q, t)] = cur.lat[q].w;
            }
            sm[S::kA0 + fm(IN - 1, t)] = in.logd;
        } else if (rowt) {
#pragma unroll
            for (int f = 0; f < IN; ++f) sm[S::kA0 + fm(f, t)] = 0.f;
        }
        if (hidden) fetch_hidden_wait();   // this tile's h1, h2, requested a phase ahead
        __syncthreads();
        if (!hidden) {
        {   // h1 = relu(h0 W1 + b1)
            float c[4][CW];
#pragma unroll
            for (int q = 0; q < CW; ++q) {
                const float bb = sm[S::kB1 + CW * cg + q];
#pragma unroll
                for (int p = 0; p < 4; ++p) c[p][q] = bb;
            }
            tile_mm<IN, CW>(sm + S::kA0, sm + S::kW1, rg, cg, c);
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < CW; ++q) c[p][q] = fmaxf(c[p][q], 0.f);
            tile_store<CW>(sm + S::kA1, rg, cg, c);
        }
        __syncthreads();
        {   // h2 = relu(h1 W2 + b2)
            float c[4][CW];
#pragma unroll
            for (int q = 0; q < CW; ++q) {
                const float bb = sm[S::kB2 + CW * cg + q];
#pragma unroll
                for (int p = 0; p < 4; ++p) c[p][q] = bb;
            }
            tile_mm<HD, CW>(sm + S::kA1, sm + S::kW2, rg, cg, c);
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < CW; ++q) c[p][q] = fmaxf(c[p][q], 0.f);
            tile_store<CW>(sm + S::kA2, rg, cg, c);
        }
        __syncthreads();
        }
        // outputs, dL/do and du2 = (W3 do) . [h2 > 0], per row
        float do0 = 0.f, do1 = 0.f, do2 = 0.f, s0 = 0.f;
        if (rowt) {
            float o0 = sm[S::kB3 + 0], o2 = sm[S::kB3 + 2];
#pragma unroll 8
            for (int j = 0; j < HD; ++j) {
                const float h = sm[S::kA2 + fm(j, t)];
                const float4 w3 = ld4(sm + S::kW3 + 4 * j);
                o0 = fmaf(h, w3.x, o0);
                o2 = fmaf(h, w3.z, o2);
            }
            if (valid) {
                s0 = sigmoidf_(o0 - in.logd);
                const float sig = sigmoidf_(ol + o2);
                do0 = da.x * s0 * (1.f - s0) / in.d;
                do1 = da.y;
                do2 = da.z * sig * (1.f - sig);
                atomicAdd(&d_ologit[i], do2);
            }
            sm[S::kG3 + fm(0, t)] = do0;
            sm[S::kG3 + fm(1, t)] = do1;
            sm[S::kG3 + fm(2, t)] = do2;
#pragma unroll 8
            for (int j = 0; j < HD; ++j) {
                const float4 w3 = ld4(sm + S::kW3 + 4 * j);
                const float dh2 = w3.x * do0 + w3.y * do1 + w3.z * do2;
                sm[S::kG2 + fm(j, t)] = sm[S::kA2 + fm(j, t)] > 0.f ? dh2 : 0.f;
            }
            // the last layer's bias gradient: the rows' dL/do summed over the warp
            float v0 = do0, v1 = do1, v2 = do2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                v2 += __shfl_xor_sync(0xffffffffu, v2, o);
            }
            db3[0] += v0;
            db3[1] += v1;
            db3[2] += v2;
        }
        __syncthreads();
        {   // du1 = (du2 W2^T) . [h1 > 0]
            float c[4][CW];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < CW; ++q) c[p][q] = 0.f;
            tile_mm<HD, CW>(sm + S::kG2, sm + S::kW2T, rg, cg, c);
#pragma unroll
            for (int q = 0; q < CW; ++q) {
                const float4 hm = ld4(sm + S::kA1 + fm4(CW * cg + q, 4 * rg));
                c[0][q] = hm.x > 0.f ? c[0][q] : 0.f;
                c[1][q] = hm.y > 0.f ? c[1][q] : 0.f;
                c[2][q] = hm.z > 0.f ? c[2][q] : 0.f;
                c[3][q] = hm.w > 0.f ? c[3][q] : 0.f;
            }
            tile_store<CW>(sm + S::kG1, rg, cg, c);
        }
        __syncthreads();
        // dL/dh0 = du1 W1^T (80 threads: 16 row groups x 5 groups of 4 inputs)
        if (t < 80) {
            const int rg2 = t & 15, cg2 = t >> 4;
            float c[4][4];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) c[p][q] = 0.f;
#pragma unroll 4
            for (int k = 0; k < HD; ++k) {
                const float4 a = ld4(sm + S::kG1 + fm4(k, 4 * rg2));
                const float4 bv = ld4(sm + S::kW1T + k * IN + 4 * cg2);
                const float as[4] = {a.x, a.y, a.z, a.w}, bs[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) c[p][q] = fmaf(as[p], bs[q], c[p][q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                st4(sm + S::kD0 + fm4(4 * cg2 + q, 4 * rg2), c[0][q], c[1][q], c[2][q], c[3][q]);
        }
        // this tile's rows into the thread's 4x4 weight-gradient blocks
#pragma unroll
        for (int m = 0; m < S::kPer; ++m) {
            const int blk = t + kBwdThreads * m;
            if (blk < S::kBlocks) {
                const GBlk gb = grad_block<HD>(blk);
                const float* pa = sm + gb.a_off;
                const float* pg = sm + gb.g_off;
#pragma unroll 2
                for (int r = 0; r < R; r += 4) {
                    float4 x[4], y[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) x[p] = ld4(pa + fm4(gb.p0 + p, r));
#pragma unroll
                    for (int q = 0; q < 4; ++q) y[q] = ld4(pg + fm4(gb.q0 + q, r));
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float s = acc[m][4 * p + q];
                            s = fmaf(x[p].x, y[q].x, s);
                            s = fmaf(x[p].y, y[q].y, s);
                            s = fmaf(x[p].z, y[q].z, s);
                            s = fmaf(x[p].w, y[q].w, s);
                            acc[m][4 * p + q] = s;
                        }
                }
            }
        }
        __syncthreads();
        // A1 and A2 are free until the next tile's products: its stored activations on their way
        if (hidden && tile + gridDim.x < tiles) fetch_hidden<HD>(sm, hidden, ld, (tile + gridDim.x) * R, rows, t);
        // the rows' input gradients: latents, ln d (network input and explicit term), means
        if (valid) {
            float* dl = d_latent + (size_t)i * GSPARC_LATENT;
            if ((reinterpret_cast<uintptr_t>(d_latent) & 15) == 0) {   // four 16-byte vector atomics
#pragma unroll
                for (int q = 0; q < GSPARC_LATENT / 4; ++q)
                    atomicAdd(reinterpret_cast<float4*>(dl) + q,
                              make_float4(sm[S::kD0 + fm(3 + 4 * q, t)], sm[S::kD0 + fm(4 + 4 * q, t)],
                                          sm[S::kD0 + fm(5 + 4 * q, t)], sm[S::kD0 + fm(6 + 4 * q, t)]));
            } else {
#pragma unroll
                for (int f = 0; f < GSPARC_LATENT; ++f) atomicAdd(dl + f, sm[S::kD0 + fm(3 + f, t)]);
            }
            // a = sigmoid(o0 - ln d)/d: explicit ln d (-do0), network input ln d, L = d + r
            const float dlogd = -do0 + sm[S::kD0 + fm(IN - 1, t)];
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
        }
    }
    // The weight gradients: rows of the first factor are weight rows, its ones row the bias.
    // Every CTA adds into the same entries at about the same time, so that the additions queue
    // at the L2.  With 16-byte aligned gradients the CTA's sums are laid out in shared memory as
    // the gradient arrays (W1, b1, W2, b2, W3; every entry written by one thread) and added to
    // global memory by bulk reductions (cp.reduce.async.bulk .add.f32, a few per CTA);
    // otherwise each entry by an atomic.
    const bool aligned = ((reinterpret_cast<uintptr_t>(g.W1) | reinterpret_cast<uintptr_t>(g.b1) |
                           reinterpret_cast<uintptr_t>(g.W2) | reinterpret_cast<uintptr_t>(g.b2) |
                           reinterpret_cast<uintptr_t>(g.W3)) & 15) == 0;
#ifndef GSPARC_HOST_SHIM
    if (aligned) {
        constexpr int oW1 = 0, ob1 = oW1 + IN * HD, oW2 = ob1 + HD, ob2 = oW2 + HD * HD, oW3 = ob2 + HD;
        static_assert(ob1 % 4 == 0 && oW2 % 4 == 0 && ob2 % 4 == 0 && oW3 % 4 == 0 && (3 * HD) % 4 == 0,
                      "16-byte segments");
        static_assert(oW3 + 3 * HD <= S::kTotal - S::kA0, "staging within the tile buffers");
        float* st = sm + S::kA0;   // the tile buffers are free after the last tile
        __syncthreads();           // every thread is past its last tile
#pragma unroll
        for (int m = 0; m < S::kPer; ++m) {
            const int blk = t + kBwdThreads * m;
            if (blk >= S::kBlocks) continue;
            const GBlk gb = grad_block<HD>(blk);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int fr = gb.p0 + p;
                float* row = nullptr;
                if (blk < S::kBlk1) row = fr < IN ? st + oW1 + fr * HD + gb.q0 : (fr == IN ? st + ob1 + gb.q0 : nullptr);
                else if (blk < S::kBlk1 + S::kBlk2)
                    row = fr < HD ? st + oW2 + fr * HD + gb.q0 : (fr == HD ? st + ob2 + gb.q0 : nullptr);
                if (row) {
                    st4(row, acc[m][4 * p], acc[m][4 * p + 1], acc[m][4 * p + 2], acc[m][4 * p + 3]);
                } else if (blk >= S::kBlk1 + S::kBlk2) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) st[oW3 + fr * 3 + q] = acc[m][4 * p + q];
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the stores, to the bulk copies
        __syncthreads();
        if (t == 0) {
            auto bulk_add = [&](float* dst, const float* src, int n) {
                asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(dst),
                             "r"(static_cast<uint32_t>(__cvta_generic_to_shared(src))), "r"(4 * n)
                             : "memory");
            };
            bulk_add(g.W1, st + oW1, IN * HD);
            bulk_add(g.b1, st + ob1, HD);
            bulk_add(g.W2, st + oW2, HD * HD);
            bulk_add(g.b2, st + ob2, HD);
            bulk_add(g.W3, st + oW3, 3 * HD);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // shared memory read before exit
        }
    }
#endif
    if (!aligned || kHostShim) {
#pragma unroll
        for (int m = 0; m < S::kPer; ++m) {
            const int blk = t + kBwdThreads * m;
            if (blk >= S::kBlocks) continue;
            const GBlk gb = grad_block<HD>(blk);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int fr = gb.p0 + p;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = gb.q0 + q;
                    const float v = acc[m][4 * p + q];
                    if (blk < S::kBlk1) {
                        if (fr < IN) atomicAdd(&g.W1[fr * HD + c], v);
                        else if (fr == IN) atomicAdd(&g.b1[c], v);
                    } else if (blk < S::kBlk1 + S::kBlk2) {
                        if (fr < HD) atomicAdd(&g.W2[fr * HD + c], v);
                        else if (fr == HD) atomicAdd(&g.b2[c], v);
                    } else if (c < 3) {
                        atomicAdd(&g.W3[fr * 3 + c], v);
                    }
                }
            }
        }
    }
    if (t < R && lane == 0) {
        atomicAdd(&g.b3[0], db3[0]);
        atomicAdd(&g.b3[1], db3[1]);
        atomicAdd(&g.b3[2], db3[2]);
    }
}

}  // namespace
}  // namespace gsparc
