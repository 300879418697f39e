// Attribute network on the 5th-generation tensor cores (tcgen05, BF16 operands,
// FP32 accumulation in tensor memory).
//
// Eq. 1 network, batched over (transmitter, Gaussian) rows as in
// gsparc_attr_mlp: h1 = relu(h0 W1 + b1), h2 = relu(h1 W2 + b2), o = h2 W3 + b3.
// Layers 1 and 2 are M=128 x N=hidden x K GEMMs issued with tcgen05.mma by one
// thread; the output layer (hidden -> 3) and the activation epilogues run on the
// CUDA cores in FP32.
//
// Precision modes:
//   GSPARC_BF16    each operand rounded to BF16 once (one term).
//   GSPARC_BF16X2  each operand x split as x_hi = bf16(x), x_lo = bf16(x - x_hi);
//                  the products x_hi y_hi + x_lo y_hi + x_hi y_lo (three terms laid
//                  side by side along K) recover ~16 mantissa bits.
//
// Shared-memory operands use the canonical K-major layout without swizzling:
// 8-row x 16-byte core matrices, core matrices adjacent along K 128 bytes apart
// (leading byte offset), 8-row groups Kt*16 bytes apart (stride byte offset).
// One CTA of 128 threads (4 warps) owns TMEM lanes 0..127 = the tile's rows;
// thread t builds row t of the A operand and reads row t of each accumulator.

#include <algorithm>

#include "internal.cuh"
#include "tc.cuh"

namespace gsparc {
namespace {

constexpr int kRows = 128;
constexpr int kK1 = 32;   // 20 inputs padded to a multiple of 16

// Write the `terms` K-blocks of a row: values x[0..n) split into hi/lo; block layout
// [hi | lo | hi] (three terms) or [hi] (one term), each block Kb columns wide.
template <int TERMS>
__device__ __forceinline__ void write_row(uint8_t* tile, int r, const float* x, int n, int Kb) {
    const int Kt = Kb * TERMS;
    for (int k0 = 0; k0 < Kb; k0 += 8) {
        float v8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v8[q] = (k0 + q) < n ? x[k0 + q] : 0.f;
        uint4 H, Lo;
        split8(v8, H, Lo);
        *reinterpret_cast<uint4*>(tile + canon_off(r, k0, Kt)) = H;
        if (TERMS == 3) {
            *reinterpret_cast<uint4*>(tile + canon_off(r, Kb + k0, Kt)) = Lo;
            *reinterpret_cast<uint4*>(tile + canon_off(r, 2 * Kb + k0, Kt)) = H;
        }
    }
}

// Weight operand B[n][k] = W[k][n] (W input-major [kin, N]) in blocks [hi | hi | lo].  The
// thread's elements are loaded together (global-space loads, one round trip) before the
// shared-memory stores.
template <int TERMS, int N, int Kb>
__device__ __forceinline__ void write_weights(uint8_t* tile, const float* __restrict__ W, int kin) {
    constexpr int Kt = Kb * TERMS;
    constexpr int kPer = (N * Kb + kRows - 1) / kRows;
    float v[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int e = (int)threadIdx.x + q * kRows;
        const int n = e / Kb, k = e - n * Kb;
        v[q] = (e < N * Kb && k < kin) ? __ldg(W + k * N + n) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int e = (int)threadIdx.x + q * kRows;
        if (e < N * Kb) {
            const int n = e / Kb, k = e - n * Kb;
            const __nv_bfloat16 hi = __float2bfloat16_rn(v[q]);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v[q] - __bfloat162float(hi));
            *reinterpret_cast<__nv_bfloat16*>(tile + canon_off(n, k, Kt)) = hi;
            if (TERMS == 3) {
                *reinterpret_cast<__nv_bfloat16*>(tile + canon_off(n, Kb + k, Kt)) = hi;
                *reinterpret_cast<__nv_bfloat16*>(tile + canon_off(n, 2 * Kb + k, Kt)) = lo;
            }
        }
    }
}

template <int HD, int TERMS>
struct TcSmem {
    static constexpr int kKt1 = kK1 * TERMS;
    static constexpr int kKt2 = HD * TERMS;
    static constexpr int kA1 = 0;                                  // [128 x Kt1] bf16
    static constexpr int kA2 = kA1 + kRows * kKt1 * 2;             // [128 x Kt2]
    static constexpr int kB1 = kA2 + kRows * kKt2 * 2;             // [HD x Kt1]
    static constexpr int kB2 = kB1 + HD * kKt1 * 2;                // [HD x Kt2]
    static constexpr int kF = kB2 + HD * kKt2 * 2;                 // fp32: b1, b2, W3, b3
    static constexpr int kMisc = kF + (2 * HD + 3 * HD + 4) * 4;   // mbarrier, tmem addr, drain mbarrier
    static constexpr int kTotal = kMisc + 32;
    static_assert(kMisc % 8 == 0, "mbarriers 8-byte aligned");
};

template <int HD, int TERMS>
__global__ void __launch_bounds__(kRows) k_mlp_tc(int N, int B, const float* __restrict__ tx, float rx0,
                                                  float rx1, float rx2, const float* __restrict__ means,
                                                  const float* __restrict__ ologit,
                                                  const float* __restrict__ latent,
                                                  const float* __restrict__ W1, const float* __restrict__ b1,
                                                  const float* __restrict__ W2, const float* __restrict__ b2,
                                                  const float* __restrict__ W3, const float* __restrict__ b3,
                                                  float4* __restrict__ attr) {
    using L = TcSmem<HD, TERMS>;
    extern __shared__ __align__(1024) uint8_t sm[];
    const int t = threadIdx.x, warp = t >> 5;
    float* sf = reinterpret_cast<float*>(sm + L::kF);
    float* sb1 = sf;
    float* sb2 = sf + HD;
    float* sW3 = sf + 2 * HD;
    float* sb3 = sf + 5 * HD;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + L::kMisc);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::kMisc + 8);

    write_weights<TERMS, HD, kK1>(sm + L::kB1, W1, GSPARC_MLP_IN);
    write_weights<TERMS, HD, HD>(sm + L::kB2, W2, HD);
    for (int e = t; e < HD; e += kRows) {
        sb1[e] = b1[e];
        sb2[e] = b2[e];
    }
    for (int e = t; e < 3 * HD; e += kRows) sW3[e] = W3[e];
    if (t < 3) sb3[t] = b3[t];
    const uint32_t mb = smem_u32(mbar);
    if (t == 0) {
        mbar_init(mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        // 2*HD accumulator columns (D1 then D2), rounded up to a power of two >= 32
        constexpr uint32_t ncols = (2 * HD <= 32) ? 32 : (2 * HD <= 64 ? 64 : 128);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t d1 = tbase, d2 = tbase + HD;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    constexpr uint32_t idesc = make_idesc(kRows, HD);
    const uint32_t a1 = smem_u32(sm + L::kA1), a2 = smem_u32(sm + L::kA2);
    const uint32_t bb1 = smem_u32(sm + L::kB1), bb2 = smem_u32(sm + L::kB2);
    uint32_t phase = 0;
    bool ok = true;

    const int64_t rows = (int64_t)N * B;
    const int64_t tiles = (rows + kRows - 1) / kRows;
    // the next tile's row inputs are loaded while this tile computes (global-space loads, so
    // no shared-memory store orders them)
    struct RowIn {
        float t0, t1, t2, m0, m1, m2;
        float4 lat[GSPARC_LATENT / 4];
    };
    auto load_row = [&](int64_t tl) {
        RowIn in{};
        const int64_t rw = tl * kRows + t;
        if (tl < tiles && rw < rows) {
            const int bq = (int)(rw / N);
            const int iq = (int)(rw - (int64_t)bq * N);
            in.t0 = __ldg(tx + 3 * bq);
            in.t1 = __ldg(tx + 3 * bq + 1);
            in.t2 = __ldg(tx + 3 * bq + 2);
            in.m0 = __ldg(means + 3 * iq);
            in.m1 = __ldg(means + 3 * iq + 1);
            in.m2 = __ldg(means + 3 * iq + 2);
            const float4* l4 = reinterpret_cast<const float4*>(latent + (size_t)iq * GSPARC_LATENT);
#pragma unroll
            for (int q = 0; q < GSPARC_LATENT / 4; ++q) in.lat[q] = __ldg(l4 + q);
        }
        return in;
    };
    RowIn next = load_row(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const RowIn cur = next;
        next = load_row(tile + gridDim.x);
        const int64_t row = tile * kRows + t;
        const bool valid = row < rows;
        int b = 0, i = 0;
        float d = 1.f, logd = 0.f, r = 0.f;
        float h0[GSPARC_MLP_IN];
        if (valid) {
            b = (int)(row / N);
            i = (int)(row - (int64_t)b * N);
            const float t0 = cur.t0, t1 = cur.t1, t2 = cur.t2;
            const float m0 = cur.m0, m1 = cur.m1, m2 = cur.m2;
            const float e0 = m0 - t0, e1 = m1 - t1, e2 = m2 - t2;
            d = fmaxf(sqrtf(e0 * e0 + e1 * e1 + e2 * e2), kDMin);
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
        // ---- layer 1 on the tensor cores
        write_row<TERMS>(sm + L::kA1, t, h0, GSPARC_MLP_IN, kK1);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) {
#pragma unroll
            for (int s = 0; s < L::kKt1 / 16; ++s)
                mma_bf16(d1, make_desc(a1 + s * 256, 128, L::kKt1 * 16),
                         make_desc(bb1 + s * 256, 128, L::kKt1 * 16), idesc, s > 0);
            mma_commit(mb);
        }
        ok = __syncthreads_and(mbar_wait(mb, phase)) != 0;   // uniform across the CTA
        phase ^= 1;
        tc_fence_after();
        float h1[HD];
#pragma unroll
        for (int c = 0; c < HD; c += 16) {
            float v[16];
            tmem_ld16(d1 + lane_base + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) h1[c + q] = fmaxf(v[q] + sb1[c + q], 0.f);
        }
        // ---- layer 2 on the tensor cores
        write_row<TERMS>(sm + L::kA2, t, h1, HD, HD);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0 && ok) {
#pragma unroll
            for (int s = 0; s < L::kKt2 / 16; ++s)
                mma_bf16(d2, make_desc(a2 + s * 256, 128, L::kKt2 * 16),
                         make_desc(bb2 + s * 256, 128, L::kKt2 * 16), idesc, s > 0);
            mma_commit(mb);
        }
        ok = __syncthreads_and(ok && mbar_wait(mb, phase)) != 0;
        phase ^= 1;
        tc_fence_after();
        float o0 = sb3[0], o1 = sb3[1], o2 = sb3[2];
#pragma unroll
        for (int c = 0; c < HD; c += 16) {
            float v[16];
            tmem_ld16(d2 + lane_base + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float h2 = fmaxf(v[q] + sb2[c + q], 0.f);
                o0 = fmaf(h2, sW3[(c + q) * 3 + 0], o0);
                o1 = fmaf(h2, sW3[(c + q) * 3 + 1], o1);
                o2 = fmaf(h2, sW3[(c + q) * 3 + 2], o2);
            }
        }
        tc_fence_before();
        if (valid) {
            if (ok) {
                const float a = 1.0f / (1.0f + expf(-(o0 - logd))) / d;
                const float sig = 1.0f / (1.0f + expf(-(ologit[i] + o2)));
                attr[row] = make_float4(a, o1, sig, d + r);
            } else {
                const float nan = __int_as_float(0x7fc00000);
                attr[row] = make_float4(nan, nan, nan, nan);   // an expired wait poisons the rows
            }
        }
    }
    // no product still in flight when the TMEM is freed (an expired wait skipped the last ones)
    if (t == 0) tc_drain(smem_u32(sm + L::kMisc + 16));
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        constexpr uint32_t ncols = (2 * HD <= 32) ? 32 : (2 * HD <= 64 ? 64 : 128);
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols) : "memory");
    }
}

template <int HD, int TERMS>
int launch_tc(int32_t N, int32_t B, const float* tx, const float* rx, const float* means, const float* ologit,
              const float* latent, const gsparc_mlp* m, float* attr, cudaStream_t s) {
    using L = TcSmem<HD, TERMS>;
    const size_t smem = L::kTotal;
    if (!ensure_smem_attr(k_mlp_tc<HD, TERMS>, (int)smem)) return GSPARC_ERR_CUDA;
    const int64_t tiles = ((int64_t)N * B + kRows - 1) / kRows;
    // at most 4 resident CTAs per SM fit the 512 TMEM columns (128 each)
    const int blocks = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * 2);
    k_mlp_tc<HD, TERMS><<<blocks, kRows, smem, s>>>(N, B, tx, rx[0], rx[1], rx[2], means, ologit, latent, m->W1,
                                                    m->b1, m->W2, m->b2, m->W3, m->b3,
                                                    reinterpret_cast<float4*>(attr));
    return launch_status();
}

}  // namespace

int attr_mlp_bf16(int32_t N, int32_t B, const float* tx, const float* rx, const float* means,
                  const float* opacity_logit, const float* latent, const gsparc_mlp* mlp, int32_t precision,
                  float* attr, cudaStream_t s) {
    const bool x2 = precision == GSPARC_BF16X2;
    switch (mlp->hidden) {
        case 16: return x2 ? launch_tc<16, 3>(N, B, tx, rx, means, opacity_logit, latent, mlp, attr, s)
                           : launch_tc<16, 1>(N, B, tx, rx, means, opacity_logit, latent, mlp, attr, s);
        case 32: return x2 ? launch_tc<32, 3>(N, B, tx, rx, means, opacity_logit, latent, mlp, attr, s)
                           : launch_tc<32, 1>(N, B, tx, rx, means, opacity_logit, latent, mlp, attr, s);
        case 64: return x2 ? launch_tc<64, 3>(N, B, tx, rx, means, opacity_logit, latent, mlp, attr, s)
                           : launch_tc<64, 1>(N, B, tx, rx, means, opacity_logit, latent, mlp, attr, s);
        default: return GSPARC_ERR_INVALID;   // the tensor-core form needs N = hidden >= 16
    }
}

}  // namespace gsparc
