// Backward of the attribute network on the 5th-generation tensor cores (tcgen05, BF16 operands
// split into hi/lo terms, FP32 accumulation in tensor memory).
//
// Eq. 1 network as in gsparc_attr_mlp: h1 = relu(h0 W1 + b1), h2 = relu(h1 W2 + b2),
// o = h2 W3 + b3.  Per tile of 128 (transmitter, Gaussian) rows, one row per thread and one
// TMEM lane per row, four M=128 products run on the tensor cores:
//     D1 = h0 W1        (forward recompute)        D2 = h1 W2        (forward recompute)
//     D3 = du2 W2^T     (dL/dh1 before the ReLU)   D4 = du1 W1^T     (dL/dh0)
// with the CUDA cores doing the epilogues (ReLU masks, the output layer and its sigmoids,
// the chain rule through d = |mu - tx| and L).  The weight gradients are contractions over
// rows: with the row index as the K dimension,
//     Dg = [h0 | h1 | h2 | 1]^T [du1 | du2 | do]
// holds dW1, dW2, dW3 and the three bias gradients as blocks of one 128 x (2 HD + 16)
// product, accumulated in TMEM over every tile the CTA takes and added to memory once at the
// end.  Each thread writes its row's values into those row-contracted operands transposed
// (one column per thread); their K-direction core-matrix stride is 144 bytes instead of 128
// so that the 32 columns a warp writes fall in distinct shared-memory banks.
//
// Every product uses three terms, x_hi y_hi + x_lo y_hi + x_hi y_lo (x_hi = bf16(x),
// x_lo = bf16(x - x_hi)), as GSPARC_BF16X2 in the forward.  Hidden widths 16 and 32 (the
// feature rows h0 | h1 | h2 | 1 must fit M = 128).

#include <algorithm>

#include "internal.cuh"
#include "tc.cuh"

namespace gsparc {
namespace {

constexpr int kRowsB = 128;
constexpr int kK0 = 32;            // 20 network inputs padded to a multiple of 16
constexpr int kGL = 144;           // K-direction core stride of the row-contracted operands
constexpr int kGS = 16 * kGL;      // 8-row group stride: 128 rows of K = 16 core matrices

template <int HD>
struct BtSmem {
    static constexpr int kKr = (kK0 > HD ? kK0 : HD) * 3;   // K of a per-row operand (3 terms)
    static constexpr int kARow = kRowsB * kKr * 2;
    static constexpr int kNG = 2 * HD + 16;                  // gradient columns: du1 | du2 | do
    static constexpr int kFH1 = 32, kFH2 = 32 + HD, kFOne = 32 + 2 * HD;   // feature rows (h0: 0..19)
    static constexpr int kGA = 16 * kGS;                     // [128 features x 128 rows], one term
    static constexpr int kGB = (kNG / 8) * kGS;              // [kNG gradients x 128 rows], one term
    static constexpr int kA0 = 0;
    static constexpr int kA1 = kA0 + kARow;
    static constexpr int kW1T = kA1 + kARow;                 // B of h0 W1:   [HD x 3*32]
    static constexpr int kW2T = kW1T + HD * kK0 * 3 * 2;     // B of h1 W2:   [HD x 3*HD]
    static constexpr int kW2R = kW2T + HD * HD * 3 * 2;      // B of du2 W2^T: [HD x 3*HD]
    static constexpr int kW1R = kW2R + HD * HD * 3 * 2;      // B of du1 W1^T: [32 x 3*HD]
    static constexpr int kGAhi = kW1R + kK0 * HD * 3 * 2;
    static constexpr int kGAlo = kGAhi + kGA;
    static constexpr int kGBhi = kGAlo + kGA;
    static constexpr int kGBlo = kGBhi + kGB;
    static constexpr int kF = kGBlo + kGB;                   // fp32: b1, b2, W3, b3
    static constexpr int kMisc = kF + (5 * HD + 4) * 4;      // mbarrier, TMEM slot, drain mbarrier
    static constexpr int kTotal = kMisc + 32;
    // TMEM columns: D1 | D2 | D3 (HD each) | D4 (32) | Dg (kNG)
    static constexpr uint32_t kD1 = 0, kD2 = HD, kD3 = 2 * HD, kD4 = 3 * HD, kDg = 3 * HD + 32;
    static constexpr uint32_t kCols = 256;
    static_assert(kDg + kNG <= kCols, "accumulators fit the TMEM allocation");
    static_assert(kFOne < 128, "feature rows fit M = 128");
    static_assert(kTotal <= 232448, "shared memory per block");
    static_assert(kMisc % 8 == 0, "mbarriers 8-byte aligned");
};

// x split into hi / lo terms laid out [hi | lo | hi] along K (Kb columns each) in row r of a
// K-major canonical tile (the A side of the three-term product).
__device__ __forceinline__ void put_row3(uint8_t* tile, int r, const float* x, int n, int Kb) {
    const int Kt = 3 * Kb;
    for (int k0 = 0; k0 < Kb; k0 += 8) {
        float v8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v8[q] = (k0 + q) < n ? x[k0 + q] : 0.f;
        uint4 H, Lo;
        split8(v8, H, Lo);
        *reinterpret_cast<uint4*>(tile + canon_off(r, k0, Kt)) = H;
        *reinterpret_cast<uint4*>(tile + canon_off(r, Kb + k0, Kt)) = Lo;
        *reinterpret_cast<uint4*>(tile + canon_off(r, 2 * Kb + k0, Kt)) = H;
    }
}

// B side of the three-term product, blocks [hi | hi | lo] along K: B[n][k] = W(n, k) for
// n < Nr, k < Kr (zero elsewhere in [Nt x Kb]); W(n, k) = W[k * ld + n] when `cols`
// (the weight stored input-major and used as W), W[n * ld + k] otherwise (used as W^T).
// The thread's elements are loaded together (global-space loads, one round trip) before
// the shared-memory stores.
template <int Nt, int Kb>
__device__ __forceinline__ void put_weights3(uint8_t* tile, const float* __restrict__ W, bool cols, int ld,
                                             int Nr, int Kr) {
    constexpr int Kt = 3 * Kb;
    constexpr int kPer = (Nt * Kb + kRowsB - 1) / kRowsB;
    float v[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int e = (int)threadIdx.x + q * kRowsB;
        const int n = e / Kb, k = e - n * Kb;
        v[q] = (e < Nt * Kb && n < Nr && k < Kr) ? __ldg(cols ? W + k * ld + n : W + n * ld + k) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int e = (int)threadIdx.x + q * kRowsB;
        if (e < Nt * Kb) {
            const int n = e / Kb, k = e - n * Kb;
            const __nv_bfloat16 hi = __float2bfloat16_rn(v[q]);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v[q] - __bfloat162float(hi));
            *reinterpret_cast<__nv_bfloat16*>(tile + canon_off(n, k, Kt)) = hi;
            *reinterpret_cast<__nv_bfloat16*>(tile + canon_off(n, Kb + k, Kt)) = hi;
            *reinterpret_cast<__nv_bfloat16*>(tile + canon_off(n, 2 * Kb + k, Kt)) = lo;
        }
    }
}

// One row's inputs: transmitter, mean, latent code, upstream gradient, opacity logit.
struct RowIn {
    float t0, t1, t2, m0, m1, m2, olog;
    float4 lat[GSPARC_LATENT / 4];
    float4 da;
};

// Element (m, k) of a row-contracted operand (K = the tile's 128 rows), hi and lo terms.
__device__ __forceinline__ void put_col(uint8_t* hi, uint8_t* lo, int m, int k, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    const uint32_t off = (uint32_t)((m >> 3) * kGS + (k >> 3) * kGL + (m & 7) * 16 + (k & 7) * 2);
    *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
}

// Issue the three-term product of a per-row operand (Kt = 3 Kb columns) with a weight tile.
__device__ __forceinline__ void mma_rows(uint32_t d, uint32_t a, uint32_t b, int Kb, uint32_t idesc) {
    const int Kt = 3 * Kb;
    for (int s = 0; s < Kt / 16; ++s)
        mma_bf16(d, make_desc(a + s * 256, 128, Kt * 16), make_desc(b + s * 256, 128, Kt * 16), idesc, s > 0);
}

// Commit, then a bounded wait in every thread; false (CTA-uniform) when any wait expired.
__device__ __forceinline__ bool round_trip(uint32_t mb, uint32_t& phase, bool ok) {
    if (threadIdx.x == 0 && ok) mma_commit(mb);
    const bool w = ok && mbar_wait(mb, phase);
    phase ^= 1;
    const bool all = __syncthreads_and(w) != 0;
    tc_fence_after();
    return all;
}

__device__ __forceinline__ void operands_ready() {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

template <int HD>
__global__ void __launch_bounds__(kRowsB, 1) k_mlp_bwd_tc(
    int N, int B, const float* __restrict__ tx, float rx0, float rx1, float rx2, const float* __restrict__ means,
    const float* __restrict__ ologit, const float* __restrict__ latent, const float* __restrict__ W1,
    const float* __restrict__ b1, const float* __restrict__ W2, const float* __restrict__ b2,
    const float* __restrict__ W3, const float* __restrict__ b3, const float4* __restrict__ d_attr,
    float* __restrict__ d_means, float* __restrict__ d_ologit, float* __restrict__ d_latent, gsparc_mlp_grad g) {
    using L = BtSmem<HD>;
    extern __shared__ __align__(1024) uint8_t sm[];
    const int t = threadIdx.x, warp = t >> 5;
    float* sb1 = reinterpret_cast<float*>(sm + L::kF);
    float* sb2 = sb1 + HD;
    float* sW3 = sb1 + 2 * HD;
    float* sb3 = sb1 + 5 * HD;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + L::kMisc);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::kMisc + 8);
    uint8_t* GAhi = sm + L::kGAhi;
    uint8_t* GAlo = sm + L::kGAlo;
    uint8_t* GBhi = sm + L::kGBhi;
    uint8_t* GBlo = sm + L::kGBlo;
    grid_dep_wait();     // the attribute gradients of the compositing backward

    put_weights3<HD, kK0>(sm + L::kW1T, W1, true, HD, HD, GSPARC_MLP_IN);
    put_weights3<HD, HD>(sm + L::kW2T, W2, true, HD, HD, HD);
    put_weights3<HD, HD>(sm + L::kW2R, W2, false, HD, HD, HD);
    put_weights3<kK0, HD>(sm + L::kW1R, W1, false, HD, GSPARC_MLP_IN, HD);
    {
        // the row-contracted operands start at zero (padding rows stay zero)
        uint4* z = reinterpret_cast<uint4*>(sm + L::kGAhi);
        const int n16 = (2 * L::kGA + 2 * L::kGB) / 16;
        for (int e = t; e < n16; e += kRowsB) z[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int e = t; e < HD; e += kRowsB) {
        sb1[e] = b1[e];
        sb2[e] = b2[e];
    }
    for (int e = t; e < 3 * HD; e += kRowsB) sW3[e] = W3[e];
    if (t < 3) sb3[t] = b3[t];
    const uint32_t mb = smem_u32(mbar);
    if (t == 0) {
        mbar_init(mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(L::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    put_col(GAhi, GAlo, L::kFOne, t, 1.0f);   // the constant feature behind the bias gradients
    operands_ready();
    const uint32_t tbase = *tslot;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    constexpr uint32_t id_h = make_idesc(kRowsB, HD);
    constexpr uint32_t id_0 = make_idesc(kRowsB, kK0);
    constexpr uint32_t id_g = make_idesc(kRowsB, L::kNG);
    const uint32_t a0 = smem_u32(sm + L::kA0), a1 = smem_u32(sm + L::kA1);
    const uint32_t gahi = smem_u32(GAhi), galo = smem_u32(GAlo), gbhi = smem_u32(GBhi), gblo = smem_u32(GBlo);
    uint32_t phase = 0;
    bool ok = true, any = false;

    const int64_t rows = (int64_t)N * B;
    const int64_t tiles = (rows + kRowsB - 1) / kRowsB;
    // the next tile's row inputs are loaded while this tile computes (global-space loads, so
    // no shared-memory store orders them)
    auto load_row = [&](int64_t tl) {
        RowIn in{};
        const int64_t row = tl * kRowsB + t;
        if (tl < tiles && row < rows) {
            const int bb = (int)(row / N);
            const int i = (int)(row - (int64_t)bb * N);
            in.t0 = __ldg(tx + 3 * bb);
            in.t1 = __ldg(tx + 3 * bb + 1);
            in.t2 = __ldg(tx + 3 * bb + 2);
            in.m0 = __ldg(means + 3 * i);
            in.m1 = __ldg(means + 3 * i + 1);
            in.m2 = __ldg(means + 3 * i + 2);
            in.olog = __ldg(ologit + i);
            const float4* l4 = reinterpret_cast<const float4*>(latent + (size_t)i * GSPARC_LATENT);
#pragma unroll
            for (int q = 0; q < GSPARC_LATENT / 4; ++q) in.lat[q] = __ldg(l4 + q);
            in.da = __ldg(d_attr + row);
        }
        return in;
    };
    RowIn next = load_row(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const RowIn cur = next;
        next = load_row(tile + gridDim.x);
        const int64_t row = tile * kRowsB + t;
        const bool valid = row < rows;
        int bb = 0, i = 0;
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
        float dist = 1.f, d = 1.f, logd = 0.f, r = 0.f;
        float h0[GSPARC_MLP_IN];
        if (valid) {
            bb = (int)(row / N);
            i = (int)(row - (int64_t)bb * N);
            t0 = cur.t0;
            t1 = cur.t1;
            t2 = cur.t2;
            m0 = cur.m0;
            m1 = cur.m1;
            m2 = cur.m2;
            const float e0 = m0 - t0, e1 = m1 - t1, e2 = m2 - t2;
            dist = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
            d = fmaxf(dist, kDMin);
            logd = logf(d);
            const float f0 = m0 - rx0, f1 = m1 - rx1, f2 = m2 - rx2;
            r = sqrtf(f0 * f0 + f1 * f1 + f2 * f2);
            h0[0] = t0;
            h0[1] = t1;
            h0[2] = t2;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = cur.lat[q];
                h0[3 + 4 * q] = v.x;
                h0[4 + 4 * q] = v.y;
                h0[5 + 4 * q] = v.z;
                h0[6 + 4 * q] = v.w;
            }
            h0[19] = logd;
        } else {
#pragma unroll
            for (int f = 0; f < GSPARC_MLP_IN; ++f) h0[f] = 0.f;
        }
        const float4 da = valid ? cur.da : make_float4(0.f, 0.f, 0.f, 0.f);
        const float olog = valid ? cur.olog : 0.f;
        // ---- D1 = h0 W1
        put_row3(sm + L::kA0, t, h0, GSPARC_MLP_IN, kK0);
#pragma unroll
        for (int f = 0; f < GSPARC_MLP_IN; ++f) put_col(GAhi, GAlo, f, t, h0[f]);
        operands_ready();
        if (t == 0) mma_rows(tbase + L::kD1, a0, smem_u32(sm + L::kW1T), kK0, id_h);
        ok = round_trip(mb, phase, ok);
        if (!ok) break;
        // ---- h1 = relu(D1 + b1); D2 = h1 W2
        float hv[HD];
        uint32_t mask1 = 0;
#pragma unroll
        for (int c = 0; c < HD; c += 16) {
            float v[16];
            tmem_ld16(tbase + L::kD1 + lane + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                hv[c + q] = fmaxf(v[q] + sb1[c + q], 0.f);
                mask1 |= (hv[c + q] > 0.f ? 1u : 0u) << (c + q);
            }
        }
        put_row3(sm + L::kA1, t, hv, HD, HD);
#pragma unroll
        for (int j = 0; j < HD; ++j) put_col(GAhi, GAlo, L::kFH1 + j, t, hv[j]);
        operands_ready();
        if (t == 0) mma_rows(tbase + L::kD2, a1, smem_u32(sm + L::kW2T), HD, id_h);
        ok = round_trip(mb, phase, ok);
        if (!ok) break;
        // ---- h2 = relu(D2 + b2), output layer, dL/do, du2; D3 = du2 W2^T
        uint32_t mask2 = 0;
        float o0 = sb3[0], o2 = sb3[2];
#pragma unroll
        for (int c = 0; c < HD; c += 16) {
            float v[16];
            tmem_ld16(tbase + L::kD2 + lane + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float h2 = fmaxf(v[q] + sb2[c + q], 0.f);
                mask2 |= (h2 > 0.f ? 1u : 0u) << (c + q);
                o0 = fmaf(h2, sW3[(c + q) * 3 + 0], o0);
                o2 = fmaf(h2, sW3[(c + q) * 3 + 2], o2);
                put_col(GAhi, GAlo, L::kFH2 + c + q, t, h2);
            }
        }
        const float s0 = 1.0f / (1.0f + expf(-(o0 - logd)));
        const float sig = 1.0f / (1.0f + expf(-(olog + o2)));
        const float do0 = da.x * s0 * (1.f - s0) / d;
        const float do1 = da.y;
        const float do2 = da.z * sig * (1.f - sig);
#pragma unroll
        for (int j2 = 0; j2 < HD; ++j2) {
            const float dh2 = sW3[j2 * 3 + 0] * do0 + sW3[j2 * 3 + 1] * do1 + sW3[j2 * 3 + 2] * do2;
            hv[j2] = ((mask2 >> j2) & 1u) ? dh2 : 0.f;
            put_col(GBhi, GBlo, HD + j2, t, hv[j2]);
        }
        put_col(GBhi, GBlo, 2 * HD + 0, t, do0);
        put_col(GBhi, GBlo, 2 * HD + 1, t, do1);
        put_col(GBhi, GBlo, 2 * HD + 2, t, do2);
        put_row3(sm + L::kA0, t, hv, HD, HD);
        operands_ready();
        if (t == 0) mma_rows(tbase + L::kD3, a0, smem_u32(sm + L::kW2R), HD, id_h);
        ok = round_trip(mb, phase, ok);
        if (!ok) break;
        // ---- du1 = [h1 > 0] D3; D4 = du1 W1^T and the weight-gradient product
#pragma unroll
        for (int c = 0; c < HD; c += 16) {
            float v[16];
            tmem_ld16(tbase + L::kD3 + lane + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) hv[c + q] = ((mask1 >> (c + q)) & 1u) ? v[q] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < HD; ++j) put_col(GBhi, GBlo, j, t, hv[j]);
        put_row3(sm + L::kA1, t, hv, HD, HD);
        operands_ready();
        if (t == 0) {
            mma_rows(tbase + L::kD4, a1, smem_u32(sm + L::kW1R), HD, id_0);
            // Dg += GA_hi GB_hi + GA_lo GB_hi + GA_hi GB_lo over the tile's 128 rows
            const uint32_t as_[3] = {gahi, galo, gahi};
            const uint32_t bs_[3] = {gbhi, gbhi, gblo};
#pragma unroll
            for (int term = 0; term < 3; ++term)
#pragma unroll
                for (int s = 0; s < kRowsB / 16; ++s)
                    mma_bf16(tbase + L::kDg, make_desc(as_[term] + s * 2 * kGL, kGL, kGS),
                             make_desc(bs_[term] + s * 2 * kGL, kGL, kGS), id_g,
                             (any || term > 0 || s > 0) ? 1u : 0u);
        }
        any = true;
        ok = round_trip(mb, phase, ok);
        if (!ok) break;
        // ---- dL/dh0: latent codes, ln d
        float dh0[kK0];
#pragma unroll
        for (int c = 0; c < kK0; c += 16) {
            float v[16];
            tmem_ld16(tbase + L::kD4 + lane + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) dh0[c + q] = v[q];
        }
        tc_fence_before();
        if (valid) {
            float* dl = d_latent + (size_t)i * GSPARC_LATENT;
            if ((reinterpret_cast<uintptr_t>(d_latent) & 15) == 0) {   // four 16-byte vector atomics
#pragma unroll
                for (int q = 0; q < GSPARC_LATENT / 4; ++q)
                    atomicAdd(reinterpret_cast<float4*>(dl) + q,
                              make_float4(dh0[3 + 4 * q], dh0[4 + 4 * q], dh0[5 + 4 * q], dh0[6 + 4 * q]));
            } else {
#pragma unroll
                for (int f = 0; f < GSPARC_LATENT; ++f) atomicAdd(dl + f, dh0[3 + f]);
            }
            atomicAdd(&d_ologit[i], do2);
            // a = sigmoid(o0 - ln d)/d: explicit ln d (-do0), network input ln d, L = d + r
            const float dlogd = -do0 + dh0[GSPARC_MLP_IN - 1];
            const float dd = da.x * (-s0 / (d * d)) + da.w + dlogd / d;
            float gm0 = 0.f, gm1 = 0.f, gm2 = 0.f;
            if (dist > kDMin) {
                const float f = dd / dist;
                gm0 += f * (m0 - t0);
                gm1 += f * (m1 - t1);
                gm2 += f * (m2 - t2);
            }
            if (r > 0.f) {
                const float f = da.w / r;
                gm0 += f * (m0 - rx0);
                gm1 += f * (m1 - rx1);
                gm2 += f * (m2 - rx2);
            }
            atomicAdd(&d_means[3 * i + 0], gm0);
            atomicAdd(&d_means[3 * i + 1], gm1);
            atomicAdd(&d_means[3 * i + 2], gm2);
        }
    }
    // ---- the CTA's weight gradients: TMEM lane t holds feature row t of Dg
    if (ok && any) {
        float v[L::kNG];
#pragma unroll
        for (int c = 0; c < L::kNG; c += 16) {
            float w16[16];
            tmem_ld16(tbase + L::kDg + lane + c, w16);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[c + q] = w16[q];
        }
        // every CTA adds into the same entries at about the same time, so the additions queue at
        // the L2: with 16-byte aligned gradients the CTA's rows are laid out in shared memory as
        // the gradient arrays (the per-row operand buffer is free after the last tile) and added
        // by bulk reductions (cp.reduce.async.bulk .add.f32), else one atomic per entry
        const bool aligned = ((reinterpret_cast<uintptr_t>(g.W1) | reinterpret_cast<uintptr_t>(g.b1) |
                               reinterpret_cast<uintptr_t>(g.W2) | reinterpret_cast<uintptr_t>(g.b2) |
                               reinterpret_cast<uintptr_t>(g.W3)) & 15) == 0;
        constexpr int IN = GSPARC_MLP_IN;
        constexpr int oW1 = 0, ob1 = oW1 + IN * HD, oW2 = ob1 + HD, ob2 = oW2 + HD * HD, oW3 = ob2 + HD;
        static_assert(ob1 % 4 == 0 && oW2 % 4 == 0 && ob2 % 4 == 0 && oW3 % 4 == 0 && (3 * HD) % 4 == 0,
                      "16-byte segments");
        static_assert((oW3 + 3 * HD) * 4 <= L::kARow, "staging within the per-row operand buffer");
        if (aligned) {
            float* st = reinterpret_cast<float*>(sm + L::kA0);
            auto put = [&](float* dst, const float* src, int n) {
                for (int q = 0; q < n; q += 4) *reinterpret_cast<float4*>(dst + q) = make_float4(src[q], src[q + 1], src[q + 2], src[q + 3]);
            };
            if (t < IN) {
                put(st + oW1 + t * HD, v, HD);
            } else if (t >= L::kFH1 && t < L::kFH1 + HD) {
                put(st + oW2 + (t - L::kFH1) * HD, v + HD, HD);
            } else if (t >= L::kFH2 && t < L::kFH2 + HD) {
#pragma unroll
                for (int c = 0; c < 3; ++c) st[oW3 + (t - L::kFH2) * 3 + c] = v[2 * HD + c];
            } else if (t == L::kFOne) {
                put(st + ob1, v, HD);
                put(st + ob2, v + HD, HD);
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(&g.b3[c], v[2 * HD + c]);
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
        } else {
            if (t < IN) {
#pragma unroll
                for (int n = 0; n < HD; ++n) atomicAdd(&g.W1[t * HD + n], v[n]);
            } else if (t >= L::kFH1 && t < L::kFH1 + HD) {
#pragma unroll
                for (int n = 0; n < HD; ++n) atomicAdd(&g.W2[(t - L::kFH1) * HD + n], v[HD + n]);
            } else if (t >= L::kFH2 && t < L::kFH2 + HD) {
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(&g.W3[(t - L::kFH2) * 3 + c], v[2 * HD + c]);
            } else if (t == L::kFOne) {
#pragma unroll
                for (int n = 0; n < HD; ++n) {
                    atomicAdd(&g.b1[n], v[n]);
                    atomicAdd(&g.b2[n], v[HD + n]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(&g.b3[c], v[2 * HD + c]);
            }
        }
    }
    if (!ok && t == 0) atomicAdd(&g.b3[0], __int_as_float(0x7fc00000));   // an expired wait poisons the result
    // no product still in flight when the TMEM is freed (an expired wait skipped the last ones)
    if (t == 0) tc_drain(smem_u32(sm + L::kMisc + 16));
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(L::kCols) : "memory");
    }
}

template <int HD>
int launch_bwd_tc(int32_t N, int32_t B, const float* tx, const float* rx, const float* means, const float* ologit,
                  const float* latent, const gsparc_mlp* m, const float* d_attr, float* d_means, float* d_ologit,
                  float* d_latent, const gsparc_mlp_grad& g, cudaStream_t s) {
    using L = BtSmem<HD>;
    if (!ensure_smem_attr(k_mlp_bwd_tc<HD>, L::kTotal)) return GSPARC_ERR_CUDA;
    const int64_t tiles = ((int64_t)N * B + kRowsB - 1) / kRowsB;
    // one CTA per SM (the operands take most of its shared memory)
    const int blocks = (int)std::min<int64_t>(tiles, (int64_t)num_sms());
    return launch_after(GSPARC_OVERLAP_NETWORK, k_mlp_bwd_tc<HD>, dim3(blocks), dim3(kRowsB), L::kTotal, s, N, B, tx, rx[0], rx[1], rx[2],
                        means, ologit, latent, m->W1, m->b1, m->W2, m->b2, m->W3, m->b3,
                        reinterpret_cast<const float4*>(d_attr), d_means, d_ologit, d_latent, g);
}

}  // namespace
}  // namespace gsparc

using namespace gsparc;

extern "C" int gsparc_attr_mlp_bwd_tc(int32_t N, int32_t B, const float* tx, const float* rx, const float* means,
                                      const float* opacity_logit, const float* latent, const gsparc_mlp* mlp,
                                      int32_t precision, const float* d_attr, float* d_means,
                                      float* d_opacity_logit, float* d_latent, const gsparc_mlp_grad* grads,
                                      void* stream) {
    if (N < 0 || B <= 0 || !mlp || !rx || !grads) return GSPARC_ERR_INVALID;
    if (precision != GSPARC_BF16X2) return GSPARC_ERR_INVALID;
    if (mlp->hidden != 16 && mlp->hidden != 32) return GSPARC_ERR_INVALID;
    if (!mlp->W1 || !mlp->b1 || !mlp->W2 || !mlp->b2 || !mlp->W3 || !mlp->b3) return GSPARC_ERR_INVALID;
    if ((int64_t)N * B >= (1ll << 31)) return GSPARC_ERR_INVALID;
    if (N == 0) return GSPARC_OK;
    if (!tx || !means || !opacity_logit || !latent || !d_attr || !d_means || !d_opacity_logit || !d_latent)
        return GSPARC_ERR_INVALID;
    if (!grads->W1 || !grads->b1 || !grads->W2 || !grads->b2 || !grads->W3 || !grads->b3) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(latent) | reinterpret_cast<uintptr_t>(d_attr)) & 15) return GSPARC_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    if (mlp->hidden == 16)
        return launch_bwd_tc<16>(N, B, tx, rx, means, opacity_logit, latent, mlp, d_attr, d_means, d_opacity_logit,
                                 d_latent, *grads, s);
    return launch_bwd_tc<32>(N, B, tx, rx, means, opacity_logit, latent, mlp, d_attr, d_means, d_opacity_logit,
                             d_latent, *grads, s);
}
