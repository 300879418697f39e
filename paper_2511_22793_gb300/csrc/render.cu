// Compositing launches and entry points: the FP32 kernels (render_common.cuh) and the
// tensor-core kernels below.

#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "render_common.cuh"
#include "bwd_schedule.cuh"

namespace gsparc {
namespace {

template <int S>
int launch_fwd(const RenderArgs& a, int T, cudaStream_t s) {
    constexpr int smem = F32Smem<S>::kTotal;
    if (!ensure_smem_attr(k_render_fwd<S>, smem)) return GSPARC_ERR_CUDA;
    dim3 grid((a.K + S - 1) / S, T, a.B);
    return launch_after(GSPARC_OVERLAP_FORWARD, k_render_fwd<S>, grid, dim3(kThreads), smem, s, a);
}

// max_items > 0: a scheduled launch (a.items), one CTA per item
template <int S>
int launch_bwd(const RenderArgs& a, int T, cudaStream_t s, uint32_t max_items = 0) {
    constexpr int smem = F32BwdSmem<S>::kTotal;
    if (!ensure_smem_attr(k_render_bwd<S>, smem)) return GSPARC_ERR_CUDA;
    if (max_items) return launch_after(GSPARC_OVERLAP_BACKWARD, k_render_bwd<S>, dim3(max_items), dim3(kThreads), smem, s, a);
    dim3 grid((a.K + S - 1) / S, T, a.B);
    return launch_after(GSPARC_OVERLAP_BACKWARD, k_render_bwd<S>, grid, dim3(kThreads), smem, s, a);
}

int launch_fwd_any(const RenderArgs& a, int T, cudaStream_t s) {
    switch (pick_strip(a.K, (int64_t)T * a.B)) {
        case 1: return launch_fwd<1>(a, T, s);
        case 2: return launch_fwd<2>(a, T, s);
        case 4: return launch_fwd<4>(a, T, s);
        case 8: return launch_fwd<8>(a, T, s);
        case 16: return launch_fwd<16>(a, T, s);
        default: return launch_fwd<32>(a, T, s);
    }
}

int launch_bwd_any(const RenderArgs& a, int T, cudaStream_t s, uint32_t max_items = 0) {
    switch (pick_strip(a.K, (int64_t)T * a.B)) {
        case 1: return launch_bwd<1>(a, T, s, max_items);
        case 2: return launch_bwd<2>(a, T, s, max_items);
        case 4: return launch_bwd<4>(a, T, s, max_items);
        case 8: return launch_bwd<8>(a, T, s, max_items);
        case 16: return launch_bwd<16>(a, T, s, max_items);
        default: return launch_bwd<32>(a, T, s, max_items);
    }
}

// strips of the FP32 kernels (the s_tot layout of gsparc_render_fwd_l2)
int fp32_strips(int K) {
    const int S = pick_strip(K, 0);
    return (K + S - 1) / S;
}

bool common_ok(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
               const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
               const float* attr) {
    if (!view_ok(view) || !band || band->K <= 0 || band->K > 65535 || B <= 0 || B > 65535 || N < 0)
        return false;
    if (!tile_ranges || !sorted_ids || (N > 0 && (!proj || !attr))) return false;
    if ((reinterpret_cast<uintptr_t>(proj) | reinterpret_cast<uintptr_t>(attr)) & 15) return false;
    if (reinterpret_cast<uintptr_t>(tile_ranges) & 7) return false;
    return true;
}

}  // namespace
}  // namespace gsparc

using namespace gsparc;

extern "C" int gsparc_render_fwd(const gsparc_view* view, const gsparc_band* band, int32_t B,
                                 int32_t N, const float* proj, const uint32_t* tile_ranges,
                                 const uint32_t* sorted_ids, const float* attr, float* spectrum,
                                 float* final_logT, uint32_t* n_contrib, uint32_t* n_used,
                                 int32_t* d_status, void* stream) {
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr) || !spectrum)
        return GSPARC_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(spectrum) & 7) return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.spectrum = reinterpret_cast<float2*>(spectrum);
    a.final_logT = final_logT;
    a.n_contrib = n_contrib;
    a.n_used = n_used;
    a.T = tiles_x(*view) * tiles_y(*view);
    return launch_fwd_any(a, a.T, as_stream(stream));
}

extern "C" int gsparc_render_fwd_l2(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                                    const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                                    const float* attr, const float* target, float* loss, float* d_spectrum,
                                    float* spectrum, float* final_logT, uint32_t* n_contrib, uint32_t* n_used,
                                    float* s_tot, uint32_t* tile_walk, int32_t* d_status, void* stream) {
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr)) return GSPARC_ERR_INVALID;
    if (!target || !loss || !d_spectrum) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(spectrum) | reinterpret_cast<uintptr_t>(target) |
         reinterpret_cast<uintptr_t>(d_spectrum)) & 7)
        return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.spectrum = reinterpret_cast<float2*>(spectrum);
    a.final_logT = final_logT;
    a.n_contrib = n_contrib;
    a.n_used = n_used;
    a.l2_target = reinterpret_cast<const float2*>(target);
    a.l2_loss = loss;
    a.l2_grad = reinterpret_cast<float2*>(d_spectrum);
    a.s_tot = s_tot;
    a.tile_walk = tile_walk;
    const int64_t count = (int64_t)B * band->K * view->H * view->W;
    a.l2_inv = (float)(1.0 / (double)count);
    a.T = tiles_x(*view) * tiles_y(*view);
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return GSPARC_ERR_CUDA;
    return launch_fwd_any(a, a.T, s);
}

extern "C" int gsparc_render_bwd(const gsparc_view* view, const gsparc_band* band, int32_t B,
                                 int32_t N, const float* proj, const uint32_t* tile_ranges,
                                 const uint32_t* sorted_ids, const float* attr,
                                 const float* final_logT, const uint32_t* n_contrib,
                                 const float* d_spectrum, float* d_attr, float* d_proj,
                                 int32_t* d_status, void* stream) {
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr)) return GSPARC_ERR_INVALID;
    if (!final_logT || !n_contrib || !d_spectrum || !d_attr || !d_proj) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_spectrum) & 7) || (reinterpret_cast<uintptr_t>(d_attr) & 15))
        return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.final_logT = const_cast<float*>(final_logT);
    a.n_contrib = const_cast<uint32_t*>(n_contrib);
    a.d_spectrum = reinterpret_cast<const float2*>(d_spectrum);
    a.d_attr = reinterpret_cast<float4*>(d_attr);
    a.d_proj = d_proj;
    a.T = tiles_x(*view) * tiles_y(*view);
    return launch_bwd_any(a, a.T, as_stream(stream));
}

// =============================================================================================
// Tensor-core forward: the subcarrier contraction on tcgen05.
//
// For one (transmitter, tile, strip of S subcarriers) and a batch of E list entries, every
// pixel's compositing weights w_pj = T_pj alpha_pj are computed on the CUDA cores exactly as in
// k_render_fwd (same alpha, same log2 T recursion, same termination), and the strip of the
// spectrum accumulates
//     Z[p][2kk + {re, im}] += sum_j w_pj * Re/Im(a_j e^{j psi_jk})
// as a [128 pixels x E] x [E x 2S] product per half tile on the tensor cores, accumulating in
// TMEM (FP32).  Both operands are split into BF16 hi/lo terms laid side by side along K
// ([w_hi | w_lo | w_hi] . [s_hi | s_hi | s_lo]), so every product carries ~16 mantissa bits
// and the sum is accumulated in FP32.  A and B are double-buffered and the kernel is
// warp-specialised (below): the pixel warps build A, builder warps build B, one warp issues the
// MMAs; tcgen05.commit on a per-stage mbarrier frees a stage.  Every mbarrier wait is bounded;
// an expired wait poisons the strip with NaN.
// =============================================================================================

#include "tc.cuh"

namespace gsparc {
namespace {

// Warp-specialised kernels: builder warps synchronise among themselves by named barrier 1.
constexpr int kWsProd = 96;                    // builder threads (three warps)

__device__ __forceinline__ void producer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kWsProd) : "memory");
}

// Barrier of the producer warps that also ANDs a flag over them: every producer thread takes
// the same branch afterwards (a warp leaving the loop alone would strand the others at the
// next producer_sync).
__device__ __forceinline__ bool producer_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kWsProd)
        : "memory");
    return r != 0;
}

constexpr int kTcE = 32;            // list entries per batch
constexpr int kTcKt = 3 * kTcE;     // three split-BF16 terms along K

template <int S>
struct RTcSmem {
    static constexpr int kN = 2 * S;
    static constexpr int kAHalf = 128 * kTcKt * 2;
    static constexpr int kA = 0;                              // [stage][half] 128 x Kt bf16
    static constexpr int kBStage = kN * kTcKt * 2;
    static constexpr int kB = kA + 4 * kAHalf;                // [stage] 2S x Kt bf16
    // per-entry records, double-buffered: batch i+1 is gathered while batch i computes
    static constexpr int kGeo = kB + 2 * kBStage;             // float4[2][E]
    static constexpr int kGeo2 = kGeo + 2 * kTcE * 16;        // float2[2][E]
    static constexpr int kExt = kGeo2 + 2 * kTcE * 8;         // float2[2][E]
    static constexpr int kAmp = kExt + 2 * kTcE * 8;          // float[2][E]
    static constexpr int kPhi = kAmp + 2 * kTcE * 4;
    static constexpr int kLen = kPhi + 2 * kTcE * 4;
    static constexpr int kCsi = kLen + 2 * kTcE * 4;          // float[8 warps][2S]: CSI partial sums
    static constexpr int kL2 = kCsi + 8 * 2 * S * 4;          // float[8 warps]: loss partial sums
    static constexpr int kBar = kL2 + 8 * 4;                  // start of the mbarriers
    static constexpr uint32_t kCols = (4 * S <= 32) ? 32 : (4 * S <= 64 ? 64 : (4 * S <= 128 ? 128 : 256));
};

// ---------------------------------------------------------------------------------------------
// Warp-specialised form of the tensor-core forward.  Warps 0-7 (one pixel per thread) compute
// the weights w = T alpha of each batch and write their rows of the A operand; warps 8-10
// (builders) publish each batch's records and build the phasor operand B; warp 11 issues the
// MMAs once both operands of a stage are in place.  mbarriers per stage (two stages):
//   rec[s]    (1): the builders released the batch's records            -> pixel warps
//   bready[s] (1): B of the batch is complete                            -> MMA warp
//   aready[s] (8): one arrival per pixel warp after writing its A rows   -> MMA warp
//   mdone[s]  (1): tcgen05.commit of the batch's MMAs (stage free again) -> builders, pixel warps
// The builders end the stream (batch count in shared memory, published with rec/bready) when
// the tile list is exhausted or every pixel warp reports all its pixels terminated; a pixel warp
// that is done keeps writing zero rows until then.  Every wait is bounded; an expired wait
// raises a shared error flag and the outputs are poisoned with NaN.
// ---------------------------------------------------------------------------------------------

constexpr int kFwsThreads = kThreads + kWsProd + 32;

template <int S>
struct RFwsSmem {
    using T = RTcSmem<S>;
    static constexpr int kBars = T::kBar;                     // rec[2], bready[2], aready[2], mdone[2], drain
    static constexpr int kMisc = kBars + 9 * 8;               // TMEM slot, done warps, batch count, error, end, walk
    static constexpr int kTotal = kMisc + 32;
};

template <int S>
__global__ void __launch_bounds__(kFwsThreads, 1) k_render_fwd_ws(RenderArgs a) {
    using L = RTcSmem<S>;
    using F = RFwsSmem<S>;
    extern __shared__ __align__(1024) uint8_t sm[];
    float4* s_geo = reinterpret_cast<float4*>(sm + L::kGeo);
    float2* s_geo2 = reinterpret_cast<float2*>(sm + L::kGeo2);
    float2* s_ext = reinterpret_cast<float2*>(sm + L::kExt);
    float* s_amp = reinterpret_cast<float*>(sm + L::kAmp);
    float* s_phi = reinterpret_cast<float*>(sm + L::kPhi);   // per entry: phase_base at the strip's k0
    float* s_len = reinterpret_cast<float*>(sm + L::kLen);   // per entry: phase step L df / c
    float* s_csi = reinterpret_cast<float*>(sm + L::kCsi);   // [warp][2S], every slot written once
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + F::kBars);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + F::kMisc);
    volatile uint32_t* s_done = tslot + 1;
    volatile uint32_t* s_nbat = tslot + 2;
    volatile uint32_t* s_err = tslot + 3;
    volatile uint32_t* s_end = tslot + 4;
    uint32_t* s_walk = tslot + 5;
    auto rec_bar = [&](int st) { return smem_u32(&bars[st]); };
    auto bready_bar = [&](int st) { return smem_u32(&bars[2 + st]); };
    auto aready_bar = [&](int st) { return smem_u32(&bars[4 + st]); };
    auto mdone_bar = [&](int st) { return smem_u32(&bars[6 + st]); };
    const uint32_t drain_bar = smem_u32(&bars[8]);
    grid_dep_wait();     // the tile lists and attributes of the kernels before

    const int strip = blockIdx.x, tile = blockIdx.y, b = blockIdx.z;
    const int k0 = strip * S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool pixel = tid < kThreads;
    const bool mma_warp = warp == (kThreads + kWsProd) / 32;
    const bool builder = !pixel && !mma_warp;
    const int prod = tid - kThreads;   // builder thread index (0..95)
    const int ptid = pixel ? tid : 0;
    const int half = ptid >> 7, m = ptid & 127;
    const int tx0 = (tile % a.TW) * kTile, ty0 = (tile / a.TW) * kTile;
    const int x = tx0 + (ptid & 15), y = ty0 + (ptid >> 4);
    const bool inside = pixel && x < a.W && y < a.H;
    const float ux = (float)x + 0.5f, uy = (float)y + 0.5f;
    const float wcx = (float)tx0 + 8.0f, wcy = (float)(ty0 + 2 * warp) + 1.0f;
    const uint2 range = a.ranges[tile];

    if (tid == 0) {
        for (int st = 0; st < 2; ++st) {
            mbar_init(rec_bar(st), 1);
            mbar_init(bready_bar(st), 1);
            mbar_init(aready_bar(st), kThreads / 32);
            mbar_init(mdone_bar(st), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_done = 0u;
        *s_nbat = 0xffffffffu;
        *s_err = 0u;
        *s_end = 0u;
        *s_walk = 0u;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(L::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    auto wait_ok = [&](uint32_t bar, uint32_t parity) {
        bool w = (*s_err == 0u) && mbar_wait(bar, parity, a.spin ? a.spin : kSpin);
        w = __all_sync(0xffffffffu, w);
        if (!w && lane == 0) *s_err = 1u;
        return w;
    };

    float logT = 0.f;
    uint32_t last = 0, used = 0;
    if (builder) {
        // ---------------- builder warps: records and the phasor operand
        // records of the batch at pos (its id already in pf_nid), then the id of the next batch:
        // the ids run one batch ahead, so that no record load waits on its id
        const bool gatherer = prod < kTcE;
        uint32_t pf_gid = 0xffffffffu, pf_nid = 0xffffffffu;
        float4 pf_p0 = make_float4(0.f, 0.f, 0.f, 0.f), pf_p1 = pf_p0, pf_at = pf_p0;
        auto load_id = [&](uint32_t pos) -> uint32_t {
            return pos + prod < range.y ? __ldg(a.ids + pos + prod) : 0xffffffffu;
        };
        auto gather = [&](uint32_t pos) {
            if (gatherer) {
                pf_gid = pf_nid;
                if (pf_gid < (uint32_t)a.N) {
                    pf_p0 = __ldg(a.proj + 2 * pf_gid);
                    pf_p1 = __ldg(a.proj + 2 * pf_gid + 1);
                    pf_at = __ldg(a.attr + (size_t)b * a.N + pf_gid);
                } else if (pf_gid != 0xffffffffu) {
                    set_status(a.status, GSPARC_ERR_INPUT);   // a list id outside the scene: skipped
                }
                pf_nid = load_id(pos + kTcE);
            }
        };
        if (gatherer) pf_nid = load_id(range.x);
        gather(range.x);
        for (int i = 0;; ++i) {
            const int st = i & 1;
            if (i >= 2) {
                // the MMAs of batch i-2 are done: the stage's A, B and records are free
                const bool w = wait_ok(mdone_bar(st), (uint32_t)((i >> 1) - 1) & 1u);
                if (!producer_all(w)) break;
            }
            const uint32_t bs = range.x + (uint32_t)i * kTcE;
            if (prod == 0) *s_end = (bs >= range.y || *s_done >= (uint32_t)(kThreads / 32)) ? 1u : 0u;
            producer_sync();
            if (*s_end) {
                if (prod == 0) {
                    *s_nbat = (uint32_t)i;
                    mbar_arrive(rec_bar(st));
                    mbar_arrive(bready_bar(st));
                }
                break;
            }
            if (gatherer) {
                const int e = st * kTcE + prod;
                if (pf_gid < (uint32_t)a.N) {
                    s_geo[e] = make_float4(pf_p0.x, pf_p0.y, pf_p1.x, pf_p1.y);
                    s_geo2[e] = make_float2(pf_p1.z, pf_at.z);
                    s_ext[e] = make_float2(pf_p0.z, pf_p0.w);
                    s_amp[e] = pf_at.x;
                    // the phasor operand's per-entry phase at the strip's first subcarrier and step
                    s_phi[e] = phase_base(a, pf_at.w, pf_at.y, k0);
                    s_len[e] = pf_at.w * a.dlam;
                } else {
                    s_geo[e] = make_float4(0.f, 0.f, __int_as_float(0x7fc00000), 0.f);
                    s_geo2[e] = make_float2(0.f, 0.f);
                    s_ext[e] = make_float2(-1.f, -1.f);
                    s_amp[e] = 0.f;
                    s_phi[e] = 0.f;
                    s_len[e] = 0.f;
                }
            }
            gather(bs + kTcE);
            producer_sync();
            if (prod == 0) mbar_arrive(rec_bar(st));   // the records, released to the pixel warps
            const int nb = (int)min((uint32_t)kTcE, range.y - bs);
            const float* amp = s_amp + st * kTcE;
            const float* phi = s_phi + st * kTcE;
            const float* len = s_len + st * kTcE;
            uint8_t* Bst = sm + L::kB + st * L::kBStage;
            for (int e = prod; e < S * (kTcE / 8); e += kWsProd) {
                const int kk = e % S, j0 = (e / S) * 8;
                const int k = k0 + kk;
                float re[8], im[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = j0 + q;
                    re[q] = 0.f;
                    im[q] = 0.f;
                    if (j < nb && k < a.K) {
                        const float2 ph = phasor_at(phi[j], len[j], kk);
                        re[q] = amp[j] * ph.x;
                        im[q] = amp[j] * ph.y;
                    }
                }
                uint4 RH, RL, IH, IL;
                split8(re, RH, RL);
                split8(im, IH, IL);
                const int nre = 2 * kk, nim = 2 * kk + 1;
                *reinterpret_cast<uint4*>(Bst + canon_off(nre, j0, kTcKt)) = RH;
                *reinterpret_cast<uint4*>(Bst + canon_off(nre, kTcE + j0, kTcKt)) = RH;
                *reinterpret_cast<uint4*>(Bst + canon_off(nre, 2 * kTcE + j0, kTcKt)) = RL;
                *reinterpret_cast<uint4*>(Bst + canon_off(nim, j0, kTcKt)) = IH;
                *reinterpret_cast<uint4*>(Bst + canon_off(nim, kTcE + j0, kTcKt)) = IH;
                *reinterpret_cast<uint4*>(Bst + canon_off(nim, 2 * kTcE + j0, kTcKt)) = IL;
            }
            fence_async_smem();
            producer_sync();
            if (prod == 0) mbar_arrive(bready_bar(st));
        }
    } else if (mma_warp) {
        // ---------------- MMA warp
        constexpr uint32_t idesc = make_idesc(128, 2 * S);
        const uint32_t a_base = smem_u32(sm + L::kA), b_base = smem_u32(sm + L::kB);
        for (int i = 0;; ++i) {
            const int st = i & 1;
            const uint32_t ph = (uint32_t)(i >> 1) & 1u;
            if (!wait_ok(bready_bar(st), ph)) break;
            if ((uint32_t)i >= *s_nbat) break;
            if (!wait_ok(aready_bar(st), ph)) break;
            if (lane == 0) {
                tc_fence_after();
                const uint64_t bd = make_desc(b_base + st * L::kBStage, 128, kTcKt * 16);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint64_t ad = make_desc(a_base + (st * 2 + h) * L::kAHalf, 128, kTcKt * 16);
#pragma unroll
                    for (int q = 0; q < kTcKt / 16; ++q)
                        mma_bf16(tbase + h * 2 * S, ad + (uint64_t)(q * 16), bd + (uint64_t)(q * 16), idesc,
                                 (i > 0 || q > 0) ? 1u : 0u);
                }
                mma_commit(mdone_bar(st));
            }
            __syncwarp();
        }
        // no product may still be in flight when the CTA frees its TMEM (after an expired wait
        // the other warps leave without waiting for the last commit)
        if (lane == 0) tc_drain(drain_bar);
        __syncwarp();
    } else {
        // ---------------- pixel warps: the weights of each batch
        bool done = !inside, counted = false;
        for (int i = 0;; ++i) {
            const int st = i & 1;
            if (!wait_ok(rec_bar(st), (uint32_t)(i >> 1) & 1u)) break;
            if ((uint32_t)i >= *s_nbat) break;
            if (i >= 2 && !wait_ok(mdone_bar(st), (uint32_t)((i >> 1) - 1) & 1u)) break;
            const uint32_t bs = range.x + (uint32_t)i * kTcE;
            const int nb = (int)min((uint32_t)kTcE, range.y - bs);
            const float4* geo = s_geo + st * kTcE;
            const float2* geo2 = s_geo2 + st * kTcE;
            const float2* ext = s_ext + st * kTcE;
            float wv[kTcE];
#pragma unroll
            for (int j = 0; j < kTcE; ++j) wv[j] = 0.f;
            if (__any_sync(0xffffffffu, !done)) {
                const uint64_t mask = warp_entry_mask(geo, geo2, ext, nb, wcx, wcy, a.W);
                if (!done) {
                    // phase 1: alpha and log2(1 - alpha) of every entry, independent of each other.
                    // Groups of 8 entries that miss the warp's rows are skipped (warp-uniform);
                    // inside a group the evaluation is branch-free so that the eight chains
                    // overlap.  The operations are eval_alpha's, in its order (the backward
                    // re-takes the same decisions); q > q_max or alpha < 1/255 gives al = -1.
                    float al[kTcE], nlv[kTcE];
#pragma unroll
                    for (int g0 = 0; g0 < kTcE; g0 += 8) {
#pragma unroll
                        for (int j = g0; j < g0 + 8; ++j) {
                            al[j] = -1.f;
                            nlv[j] = 0.f;
                        }
                        if (((mask >> g0) & 0xffull) == 0ull) continue;   // warp-uniform
#pragma unroll
                        for (int j = g0; j < g0 + 8; ++j) {
                            const float4 gg = geo[j];
                            const float2 g2 = geo2[j];
                            float dx = __fsub_rn(ux, gg.x);
                            const float hw = 0.5f * (float)a.W;
                            dx = dx >= hw ? __fsub_rn(dx, (float)a.W) : (dx < -hw ? __fadd_rn(dx, (float)a.W) : dx);
                            const float dy = __fsub_rn(uy, gg.y);
                            float q = __fmul_rn(__fmul_rn(g2.x, dy), dy);
                            q = __fmaf_rn(__fmul_rn(__fmul_rn(2.0f, gg.w), dx), dy, q);
                            q = __fmaf_rn(__fmul_rn(gg.z, dx), dx, q);
                            const float G = ex2(__fmul_rn(-0.5f * kLog2e, q));
                            const float a0 = __fmul_rn(g2.y, G);
                            const float alpha = a0 > kAlphaMax ? kAlphaMax : a0;
                            const bool ok_j = ((mask >> j) & 1ull) && q <= kQMax && alpha >= kAlphaMin;
                            al[j] = ok_j ? alpha : -1.f;
                            nlv[j] = ok_j ? lg2(__fsub_rn(1.0f, alpha)) : 0.f;
                        }
                    }
                    // phase 2: the transmittance recursion, one FADD per entry on the serial
                    // chain; branch-free, the same decisions as stopping before T < T_min
                    bool stop = false;
#pragma unroll
                    for (int j = 0; j < kTcE; ++j) {
                        const float nt = __fadd_rn(logT, nlv[j]);
                        const bool cand = !stop && al[j] >= 0.f;
                        const bool term = cand && nt < kLog2TMin;
                        stop = stop || term;
                        const bool take = cand && !term;
                        wv[j] = take ? ex2(logT) * al[j] : 0.f;
                        logT = take ? nt : logT;
                        last = take ? bs - range.x + (uint32_t)j + 1u : last;
                        used += take ? 1u : 0u;
                    }
                    done = stop;
                }
            }
            uint8_t* Ast = sm + L::kA + (st * 2 + half) * L::kAHalf;
#pragma unroll
            for (int j0 = 0; j0 < kTcE; j0 += 8) {
                float w8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) w8[q] = wv[j0 + q];
                uint4 H, Lo;
                split8(w8, H, Lo);
                *reinterpret_cast<uint4*>(Ast + canon_off(m, j0, kTcKt)) = H;
                *reinterpret_cast<uint4*>(Ast + canon_off(m, kTcE + j0, kTcKt)) = Lo;
                *reinterpret_cast<uint4*>(Ast + canon_off(m, 2 * kTcE + j0, kTcKt)) = H;
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(aready_bar(st));
            if (!counted && __all_sync(0xffffffffu, done)) {
                counted = true;
                if (lane == 0) atomicAdd(const_cast<uint32_t*>(s_done), 1u);
            }
        }
    }
    // ---------------- epilogue: the accumulated spectrum of the strip
    const size_t plane = (size_t)a.H * a.W;
    const size_t pix = (size_t)y * a.W + x;
    const uint32_t nbat = *s_nbat;
    const bool any_mma = nbat != 0xffffffffu && nbat > 0u;
    // fused loss: the targets of kAhead chunks of 8 subcarriers are in flight ahead of their
    // use, the first ones already during the wait for the last products
    constexpr int kChunks = 2 * S / 16;
    constexpr int kAhead = kChunks < 4 ? kChunks : 4;
    float2 tq[kAhead][8];
    auto load_tg = [&](int c, float2 (&t)[8]) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + c / 2 + q;
            t[q] = (a.l2_grad && inside && k < a.K) ? __ldcs(a.l2_target + ((size_t)b * a.K + k) * plane + pix)
                                                    : make_float2(0.f, 0.f);
        }
    };
    if (pixel) {
#pragma unroll
        for (int q = 0; q < kAhead; ++q) load_tg(16 * q, tq[q]);
    }
    if (pixel && any_mma) {
        const int lb = (int)nbat - 1;
        wait_ok(mdone_bar(lb & 1), (uint32_t)(lb >> 1) & 1u);
    }
    __syncthreads();
    const bool ok = *s_err == 0u && nbat != 0xffffffffu;
    tc_fence_after();
    float l2acc = 0.f, stot = 0.f;
    if (pixel) {
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll
        for (int c = 0; c < 2 * S; c += 16) {
            float2 (&tg)[8] = tq[(c / 16) % kAhead];
            float v[16];
            if (any_mma) {
                tmem_ld16(tbase + half * 2 * S + lane_base + c, v);
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0.f;
            }
            if (inside && a.spectrum) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = k0 + c / 2 + q;
                    if (k < a.K) {
                        const float nan = __int_as_float(0x7fc00000);
                        const float2 z = ok ? make_float2(v[2 * q], v[2 * q + 1]) : make_float2(nan, nan);
                        float2* dst = &a.spectrum[((size_t)b * a.K + k) * plane + pix];
                        if (a.stream_out) __stcs(dst, z);
                        else *dst = z;
                    }
                }
            }
            if (inside && a.l2_grad) {
                // fused loss: the same arithmetic as gsparc_l2_loss on this spectrum
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = k0 + c / 2 + q;
                    if (k < a.K) {
                        const size_t e = ((size_t)b * a.K + k) * plane + pix;
                        const float2 t = tg[q];
                        const float zr = ok ? v[2 * q] : __int_as_float(0x7fc00000);
                        const float dr = zr - t.x, di = v[2 * q + 1] - t.y;
                        l2acc = fmaf(dr, dr, fmaf(di, di, l2acc));
                        const float2 gz = make_float2(2.f * dr * a.l2_inv, 2.f * di * a.l2_inv);
                        a.l2_grad[e] = gz;
                        stot = fmaf(gz.x, zr, fmaf(gz.y, v[2 * q + 1], stot));
                    }
                }
            }
            if (a.csi) {
                // Eq. 2 over the CTA's pixels: a reduce-scatter of the 16 columns over the warp's
                // 32 pixels leaves column idx(lane) summed in the lane pair (lane, lane ^ 1)
                float w[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) w[q] = inside ? (ok ? v[q] : __int_as_float(0x7fc00000)) : 0.f;
#pragma unroll
                for (int o = 16, n = 8; o >= 2; o >>= 1, n >>= 1) {
                    const bool up = (lane & o) != 0;
#pragma unroll
                    for (int q = 0; q < n; ++q) {
                        const float send = up ? w[q] : w[q + n];
                        const float keep = up ? w[q + n] : w[q];
                        w[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                    }
                }
                w[0] += __shfl_xor_sync(0xffffffffu, w[0], 1);
                const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
                if ((lane & 1) == 0) s_csi[warp * 2 * S + c + idx] = w[0];
            }
            if (c / 16 + kAhead < kChunks) load_tg(c + 16 * kAhead, tg);   // the slot just used
        }
        if (inside && a.l2_grad && a.s_tot) a.s_tot[((size_t)b * gridDim.x + strip) * plane + pix] = stot;
        if (inside && strip == 0) {
            if (a.final_logT) a.final_logT[(size_t)b * plane + pix] = logT;
            if (a.n_contrib) a.n_contrib[(size_t)b * plane + pix] = last;
            if (a.n_used) a.n_used[(size_t)b * plane + pix] = used;
        }
    }
    float* s_l2 = reinterpret_cast<float*>(sm + L::kL2);
    if (pixel && a.l2_grad) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l2acc += __shfl_xor_sync(0xffffffffu, l2acc, o);
        if (lane == 0) s_l2[warp] = l2acc;
    }
    if (pixel && a.tile_walk) {
        const uint32_t wmax = __reduce_max_sync(0xffffffffu, inside ? last : 0u);
        if (lane == 0 && wmax) atomicMax(s_walk, wmax);
    }
    tc_fence_before();
    __syncthreads();
    if (a.tile_walk && strip == 0 && tid == 0)
        a.tile_walk[(size_t)b * a.T + tile] = min(*s_walk, range.y - range.x);
    if (a.l2_grad && tid == 0) {
        float t = 0.f;
        for (int w2 = 0; w2 < kThreads / 32; ++w2) t += s_l2[w2];
        atomicAdd(a.l2_loss, t * a.l2_inv);
    }
    if (a.csi) {
        for (int e = tid; e < 2 * S; e += kFwsThreads) {
            const int k = k0 + e / 2;
            float sum = 0.f;
#pragma unroll
            for (int w2 = 0; w2 < kThreads / 32; ++w2) sum += s_csi[w2 * 2 * S + e];
            if (k < a.K) atomicAdd(reinterpret_cast<float*>(&a.csi[(size_t)b * a.K + k]) + (e & 1), sum * a.csi_scale);
        }
    }
    if (tid == 0 && *s_err != 0u) set_status(a.status, GSPARC_ERR_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(L::kCols) : "memory");
    }
}

template <int S>
int launch_fwd_tc(const RenderArgs& a, int T, cudaStream_t s) {
    using F = RFwsSmem<S>;
    if (!ensure_smem_attr(k_render_fwd_ws<S>, F::kTotal)) return GSPARC_ERR_CUDA;
    dim3 grid((a.K + S - 1) / S, T, a.B);
    return launch_after(GSPARC_OVERLAP_FORWARD, k_render_fwd_ws<S>, grid, dim3(kFwsThreads), F::kTotal, s, a);
}

}  // namespace
}  // namespace gsparc

extern "C" int gsparc_render_fwd_tc(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                                    const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                                    const float* attr, float* spectrum, float* final_logT, uint32_t* n_contrib,
                                    uint32_t* n_used, int32_t* d_status, void* stream) {
    using namespace gsparc;
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr) || !spectrum) return GSPARC_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(spectrum) & 7) return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.spin = wait_limit(kSpin);
    a.spectrum = reinterpret_cast<float2*>(spectrum);
    a.final_logT = final_logT;
    a.n_contrib = n_contrib;
    a.n_used = n_used;
    const int T = tiles_x(*view) * tiles_y(*view);
    cudaStream_t s = as_stream(stream);
    if (band->K <= 8) return launch_fwd_tc<8>(a, T, s);
    if (band->K <= 16) return launch_fwd_tc<16>(a, T, s);
    if (band->K <= 32) return launch_fwd_tc<32>(a, T, s);
    return launch_fwd_tc<64>(a, T, s);
}

extern "C" int gsparc_render_fwd_l2_tc(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                                       const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                                       const float* attr, const float* target, float* loss, float* d_spectrum,
                                       float* spectrum, float* final_logT, uint32_t* n_contrib, uint32_t* n_used,
                                       float* s_tot, uint32_t* tile_walk, int32_t* d_status, void* stream) {
    using namespace gsparc;
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr)) return GSPARC_ERR_INVALID;
    if (!target || !loss || !d_spectrum) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(spectrum) | reinterpret_cast<uintptr_t>(target) |
         reinterpret_cast<uintptr_t>(d_spectrum)) & 7)
        return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.spin = wait_limit(kSpin);
    a.spectrum = reinterpret_cast<float2*>(spectrum);
    a.final_logT = final_logT;
    a.n_contrib = n_contrib;
    a.n_used = n_used;
    a.l2_target = reinterpret_cast<const float2*>(target);
    a.l2_loss = loss;
    a.l2_grad = reinterpret_cast<float2*>(d_spectrum);
    a.s_tot = s_tot;
    a.tile_walk = tile_walk;
    const int64_t count = (int64_t)B * band->K * view->H * view->W;
    a.l2_inv = (float)(1.0 / (double)count);
    const int T = tiles_x(*view) * tiles_y(*view);
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return GSPARC_ERR_CUDA;
    if (band->K <= 8) return launch_fwd_tc<8>(a, T, s);
    if (band->K <= 16) return launch_fwd_tc<16>(a, T, s);
    if (band->K <= 32) return launch_fwd_tc<32>(a, T, s);
    return launch_fwd_tc<64>(a, T, s);
}

extern "C" int gsparc_render_csi_tc(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                                    const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                                    const float* attr, float* csi, float* spectrum, float* final_logT,
                                    uint32_t* n_contrib, uint32_t* n_used, int32_t* d_status, void* stream) {
    using namespace gsparc;
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr) || !csi) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(spectrum) | reinterpret_cast<uintptr_t>(csi)) & 7) return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.spin = wait_limit(kSpin);
    a.spectrum = reinterpret_cast<float2*>(spectrum);
    a.final_logT = final_logT;
    a.n_contrib = n_contrib;
    a.n_used = n_used;
    a.csi = reinterpret_cast<float2*>(csi);
    a.csi_scale = 1.0f / ((float)view->H * (float)view->W);
    const int T = tiles_x(*view) * tiles_y(*view);
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(csi, 0, (size_t)B * band->K * 2 * sizeof(float), s) != cudaSuccess) return GSPARC_ERR_CUDA;
    if (band->K <= 8) return launch_fwd_tc<8>(a, T, s);
    if (band->K <= 16) return launch_fwd_tc<16>(a, T, s);
    if (band->K <= 32) return launch_fwd_tc<32>(a, T, s);
    return launch_fwd_tc<64>(a, T, s);
}

namespace gsparc {
namespace {

// =============================================================================================
// Tensor-core backward.
//
// For one (transmitter, tile, strip of S subcarriers) the pixel's upstream gradient
// g = dL/dz over the strip is the A operand (constant over the walk), and each batch of E list
// entries contributes three B rows per entry j built from its unit phasors u_jk = e^{j psi_jk}:
//     row 3j   : (Re u, Im u)      ->  D = sum_k Re(conj(g_k) u_jk)         (ReG)
//     row 3j+1 : (Im u, -Re u)     ->  D = sum_k Im(conj(g_k) u_jk)         (ImG)
//     row 3j+2 : kk (Im u, -Re u)  ->  D = sum_k kk Im(conj(g_k) u_jk)      (ImF)
// (K index 2kk + {re, im} matches A = (Re g_k, Im g_k)).  Both operands are split into BF16
// hi/lo terms and the products g_hi u_hi + g_lo u_hi + g_hi u_lo are accumulated in FP32 in
// TMEM.  The CUDA cores then run the same back-to-front recursion as k_render_bwd on the three
// contractions.  The kernel is warp-specialised (below): producer warps build B and issue the
// MMAs into a ring of stages while the pixel warps consume them, with mbarriers in place of
// block-wide barriers.
// =============================================================================================


struct TbMeta {
    float4* geo;
    float2* geo2;
    float2* ext;
    float* amp;
    float* phi;    // phase_base at the strip's first subcarrier
    float* len;    // phase step L df / c
    uint32_t* gid;
};

__device__ __forceinline__ TbMeta tb_meta(uint8_t* base) {
    TbMeta m;
    m.geo = reinterpret_cast<float4*>(base);
    m.geo2 = reinterpret_cast<float2*>(base + kTbE * 16);
    m.ext = reinterpret_cast<float2*>(base + kTbE * 24);
    m.amp = reinterpret_cast<float*>(base + kTbE * 32);
    m.phi = reinterpret_cast<float*>(base + kTbE * 36);
    m.len = reinterpret_cast<float*>(base + kTbE * 40);
    m.gid = reinterpret_cast<uint32_t*>(base + kTbE * 44);
    return m;
}

// ---------------------------------------------------------------------------------------------
// Warp-specialised form of the tensor-core backward.  Warps 0-7 (one pixel per thread) are
// consumers; warps 8-10 build (synchronised among themselves by a named barrier) and warp 11
// issues the MMAs.  The builders gather each batch's per-entry records,
// builds its phasor operand B, issues its MMAs into one of kWsR stages of shared memory and
// TMEM, and flushes the gradients of batches the consumers have finished; the consumers walk
// the batches at their own pace, each warp signalling when it is done with a stage.  No
// block-wide barrier sits inside the walk:
//   full[s]  (2 arrivals): tcgen05.commit of the stage's MMAs + the producer's release of the
//            stage's records;                     consumers wait, phase (i / kWsR) & 1
//   empty[s] (8 arrivals): one per consumer warp after its TMEM reads and gradient writes;
//            the producer waits before reusing the stage (and flushes that batch)
// Every wait is bounded; an expired wait raises a shared error flag and every warp leaves
// its loop (the gradients are then incomplete, as in the other forms).
// ---------------------------------------------------------------------------------------------

constexpr int kWsR = 3;
constexpr int kWsThreads = kThreads + kWsProd + 32;   // + the MMA-issuing warp

template <int S>
struct RWsSmem {
    static constexpr int kKa = 2 * S;
    static constexpr int kATile = 128 * kKa * 2;
    static constexpr int kA = 0;                                   // [half][hi, lo]
    static constexpr int kBTile = 3 * kTbE * kKa * 2;
    static constexpr int kB = kA + 4 * kATile;                     // [stage][hi, lo]
    static constexpr int kMetaStage = kTbE * (16 + 8 + 8 + 4 + 4 + 4 + 4);
    static constexpr int kMeta = kB + kWsR * 2 * kBTile;
    static constexpr int kRedStage = 8 * kTbE * 9 * 4;
    static constexpr int kRed = kMeta + kWsR * kMetaStage;         // float [stage][warp][E][9]
    static constexpr int kMask = kRed + kWsR * kRedStage;          // uint64 [stage][warp]
    static constexpr int kBar = kMask + kWsR * 8 * 8;              // full[R], empty[R], bready[R], drain
    static constexpr int kTotal = kBar + 3 * kWsR * 8 + 8 + 16;    // + TMEM slot, maxlast, error
    static constexpr uint32_t kStageCols = 2 * 3 * kTbE;           // both halves of a stage
    static constexpr uint32_t kCols = 512;
    static_assert(kWsR * kStageCols <= kCols, "TMEM stages");
    static_assert(kTotal <= 232448, "shared memory per block");
};

template <int S>
__global__ void __launch_bounds__(kWsThreads, 1) k_render_bwd_ws(RenderArgs a) {
    using L = RWsSmem<S>;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kBar);
    const uint32_t drain_bar = smem_u32(sm + L::kBar + 3 * kWsR * 8);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::kBar + 3 * kWsR * 8 + 8);
    uint32_t* s_maxlast = tslot + 1;
    volatile uint32_t* s_err = tslot + 2;
    auto red_at = [&](int st, int w, int j, int c) -> float& {
        return reinterpret_cast<float*>(sm + L::kRed + st * L::kRedStage)[(w * kTbE + j) * 9 + c];
    };
    auto mask_at = [&](int st, int w) -> uint64_t& { return reinterpret_cast<uint64_t*>(sm + L::kMask)[st * 8 + w]; };
    auto full_bar = [&](int st) { return smem_u32(&bars[st]); };
    auto empty_bar = [&](int st) { return smem_u32(&bars[kWsR + st]); };
    auto bready_bar = [&](int st) { return smem_u32(&bars[2 * kWsR + st]); };
    grid_dep_wait();     // the schedule's items, the forward's outputs and the upstream gradient

    // work item: a scheduled chunk [chunk_lo, chunk_end) of one (transmitter, tile, strip)
    // walk, or (no item list) the whole walk, whose end is then known after the prologue
    int strip, tile, b;
    bool front = false;           // front chunk [0, chunk_end), walked front to back
    uint32_t chunk_lo = 0, chunk_end = 0;
    if (a.items) {
        const uint32_t r = blockIdx.x;
        if (r >= __ldg(a.n_items)) return;   // the whole block, before any barrier or allocation
        const uint4 it = a.items[r];
        b = (int)(it.x / (uint32_t)a.T);
        tile = (int)(it.x - (uint32_t)b * (uint32_t)a.T);
        strip = (int)(it.y & 0x7fffffffu);
        front = (it.y >> 31) != 0u;
        chunk_lo = it.z;
        chunk_end = it.w;
    } else {
        strip = blockIdx.x;
        tile = blockIdx.y;
        b = blockIdx.z;
    }
    const int k0 = strip * S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool issuer = warp == (kThreads + kWsProd) / 32;
    const bool producer = warp >= kThreads / 32 && !issuer;
    const int prod = tid - kThreads;   // builder thread index (0..95) when producer
    const int ptid = (producer || issuer) ? 0 : tid;   // pixel of a consumer thread
    const int half = ptid >> 7, m = ptid & 127;
    const int tx0 = (tile % a.TW) * kTile, ty0 = (tile / a.TW) * kTile;
    const int x = tx0 + (ptid & 15), y = ty0 + (ptid >> 4);
    const bool inside = !producer && !issuer && x < a.W && y < a.H;
    const float ux = (float)x + 0.5f, uy = (float)y + 0.5f;
    const float wcx = (float)tx0 + 8.0f, wcy = (float)(ty0 + 2 * warp) + 1.0f;
    const uint2 range = a.ranges[tile];
    const size_t plane = (size_t)a.H * a.W;
    const size_t pix = (size_t)y * a.W + x;

    // batch i of a back chunk ends kTbE * i entries before chunk_end (its last batch ragged),
    // batch i of a front chunk starts at kTbE * i
    int nbatch = (int)((chunk_end - chunk_lo + kTbE - 1) / kTbE);
    auto batch_lo = [&](int i) -> uint32_t {
        if (front) return chunk_lo + (uint32_t)i * kTbE;
        const uint32_t hp = chunk_end - (uint32_t)i * kTbE;
        return hp > chunk_lo + kTbE ? hp - kTbE : chunk_lo;
    };
    auto batch_n = [&](int i) -> int {
        if (front) return (int)min((uint32_t)kTbE, chunk_end - batch_lo(i));
        return (int)(chunk_end - (uint32_t)i * kTbE - batch_lo(i));
    };
    // the builders' prefetch of one batch's records (threads 0..E-1 of the first builder
    // warp); the list ids run one batch further ahead, so that no record load waits on its id
    const bool gatherer = producer && prod < kTbE;
    uint32_t pf_gid = 0xffffffffu, pf_nid = 0xffffffffu;
    float4 pf_p0 = make_float4(0.f, 0.f, 0.f, 0.f), pf_p1 = pf_p0, pf_at = pf_p0;
    auto load_id = [&](int i) -> uint32_t {
        return (i < nbatch && prod < batch_n(i)) ? __ldg(a.ids + range.x + batch_lo(i) + prod) : 0xffffffffu;
    };
    auto gather = [&](int i) {   // records of batch i (its id in pf_nid), then the id of batch i + 1
        if (gatherer) {
            pf_gid = pf_nid;
            if (pf_gid < (uint32_t)a.N) {
                pf_p0 = __ldg(a.proj + 2 * pf_gid);
                pf_p1 = __ldg(a.proj + 2 * pf_gid + 1);
                pf_at = __ldg(a.attr + (size_t)b * a.N + pf_gid);
            } else if (pf_gid != 0xffffffffu) {
                set_status(a.status, GSPARC_ERR_INPUT);   // a list id outside the scene: skipped
            }
            pf_nid = load_id(i + 1);
        }
    };
    // a scheduled item knows its batches already: its first records load during the prologue
    if (a.items && nbatch > 0 && gatherer) {
        pf_nid = load_id(0);
        gather(0);
    }

    if (tid == 0) {
        for (int st = 0; st < kWsR; ++st) {
            mbar_init(full_bar(st), 2);
            mbar_init(empty_bar(st), kThreads / 32);
            mbar_init(bready_bar(st), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_maxlast = 0;
        *s_err = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(L::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // A operand (consumers): this pixel's upstream gradient over the strip, split hi / lo.
    // A front chunk also needs s_tot = Re sum_k conj(g_k) z_k over the strip, the sum over the
    // whole walk of the terms the back-to-front recursion accumulates: given, or formed here
    // from the spectrum.
    float s_tot = 0.f;
    if (!producer && !issuer) {
        uint8_t* Ahi = sm + L::kA + (half * 2 + 0) * L::kATile;
        uint8_t* Alo = sm + L::kA + (half * 2 + 1) * L::kATile;
        // kChunk subcarriers per round trip: the loads are global-space (they cannot alias the
        // shared-memory stores), all issued before the first use
        constexpr int kChunk = S < 16 ? S : 16;
        const size_t base = (size_t)b * a.K * plane + pix;
        const bool form_s_tot = front && !a.s_tot;
#pragma unroll 1
        for (int k1 = 0; k1 < S; k1 += kChunk) {
            float2 g[kChunk];
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int k = k0 + k1 + q;
                g[q] = (inside && k < a.K) ? __ldcs(a.d_spectrum + base + (size_t)k * plane) : make_float2(0.f, 0.f);
            }
            if (form_s_tot) {
#pragma unroll
                for (int q = 0; q < kChunk; ++q) {
                    const int k = k0 + k1 + q;
                    const float2 z = (inside && k < a.K) ? __ldcs(a.spectrum + base + (size_t)k * plane)
                                                         : make_float2(0.f, 0.f);
                    s_tot = fmaf(g[q].x, z.x, fmaf(g[q].y, z.y, s_tot));
                }
            }
#pragma unroll
            for (int q = 0; q < kChunk; q += 4) {
                const float g8[8] = {g[q].x,     g[q].y,     g[q + 1].x, g[q + 1].y,
                                     g[q + 2].x, g[q + 2].y, g[q + 3].x, g[q + 3].y};
                const int c0 = 2 * (k1 + q);
                uint4 H, Lo;
                split8(g8, H, Lo);
                *reinterpret_cast<uint4*>(Ahi + canon_off(m, c0, L::kKa)) = H;
                *reinterpret_cast<uint4*>(Alo + canon_off(m, c0, L::kKa)) = Lo;
            }
        }
    }
    if (front && a.s_tot && inside) s_tot = a.s_tot[((size_t)b * ((a.K + S - 1) / S) + strip) * plane + pix];
    float logT = (inside && !front) ? a.final_logT[(size_t)b * plane + pix] : 0.f;
    const uint32_t last = inside ? a.n_contrib[(size_t)b * plane + pix] : 0u;
    __syncthreads();
    if (last && !a.items) atomicMax(s_maxlast, last);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (!a.items) {
        chunk_end = min(*s_maxlast, range.y - range.x);   // the walk: the largest n_contrib
        nbatch = (int)((chunk_end + kTbE - 1) / kTbE);
    }
    const uint32_t tbase = *tslot;
    auto wait_ok = [&](uint32_t bar, uint32_t parity) {
        bool w = (*s_err == 0u) && mbar_wait(bar, parity, a.spin ? a.spin : kSpin);
        w = __all_sync(0xffffffffu, w);
        if (!w && lane == 0) *s_err = 1u;
        return w;
    };

    if (producer) {
        // ---------------- builder warps
        auto flush = [&](int i, int st) {
            TbMeta md = tb_meta(sm + L::kMeta + st * L::kMetaStage);
            const int nb = batch_n(i);
            for (int e = prod; e < nb * 9; e += kWsProd) {
                const int j = e / 9, c = e - j * 9;
                float acc = 0.f;
#pragma unroll
                for (int w2 = 0; w2 < kThreads / 32; ++w2)
                    if ((mask_at(st, w2) >> j) & 1ull) acc += red_at(st, w2, j, c);
                if (acc != 0.f) {
                    const uint32_t gid = md.gid[j];
                    if (c >= 5) {
                        float* dst = reinterpret_cast<float*>(&a.d_attr[(size_t)b * a.N + gid]);
                        const int slot = c == 5 ? 2 : (c == 6 ? 0 : (c == 7 ? 1 : 3));
                        atomicAdd(dst + slot, acc);
                    } else {
                        const int slot = c < 2 ? c : c + 2;
                        atomicAdd(a.d_proj + (size_t)gid * 8 + slot, acc);
                    }
                }
            }
        };
        if (!a.items && nbatch > 0 && gatherer) {
            pf_nid = load_id(0);
            gather(0);
        }
        for (int i = 0; i < nbatch; ++i) {
            const int st = i % kWsR;
            if (i >= kWsR) {
                // the consumers released the stage (batch i - R): flush that batch, then reuse
                const bool w = wait_ok(empty_bar(st), (uint32_t)((i / kWsR) - 1) & 1u);
                if (!producer_all(w)) break;   // uniform over the producer warps
                tc_fence_after();
                flush(i - kWsR, st);
            }
            producer_sync();   // the flush has read the stage's records
            TbMeta md = tb_meta(sm + L::kMeta + st * L::kMetaStage);
            if (gatherer) {
                const int e = prod;
                if (pf_gid < (uint32_t)a.N) {
                    md.geo[e] = make_float4(pf_p0.x, pf_p0.y, pf_p1.x, pf_p1.y);
                    md.geo2[e] = make_float2(pf_p1.z, pf_at.z);
                    md.ext[e] = make_float2(pf_p0.z, pf_p0.w);
                    md.amp[e] = pf_at.x;
                    // the phasor operand's per-entry phase at the strip's first subcarrier and step
                    md.phi[e] = phase_base(a, pf_at.w, pf_at.y, k0);
                    md.len[e] = pf_at.w * a.dlam;
                    md.gid[e] = pf_gid;
                } else {
                    md.geo[e] = make_float4(0.f, 0.f, __int_as_float(0x7fc00000), 0.f);
                    md.geo2[e] = make_float2(0.f, 0.f);
                    md.ext[e] = make_float2(-1.f, -1.f);
                    md.amp[e] = 0.f;
                    md.phi[e] = 0.f;
                    md.len[e] = 0.f;
                    md.gid[e] = 0;
                }
            }
            if (i + 1 < nbatch) gather(i + 1);
            producer_sync();   // the records are in place for the phasor build
            // B rows of the batch: item (j, 8 consecutive K columns) = 4 phasors
            const int nb = batch_n(i);
            uint8_t* Bhi = sm + L::kB + (st * 2 + 0) * L::kBTile;
            uint8_t* Blo = sm + L::kB + (st * 2 + 1) * L::kBTile;
            for (int e = prod; e < kTbE * (L::kKa / 8); e += kWsProd) {
                const int j = e / (L::kKa / 8), c0 = (e % (L::kKa / 8)) * 8;
                float r0[8], r1[8], r2[8];
#pragma unroll
                for (int q = 0; q < 8; q += 2) {
                    const int kk = (c0 + q) / 2, k = k0 + kk;
                    float2 u = make_float2(0.f, 0.f);
                    if (j < nb && k < a.K) u = phasor_at(md.phi[j], md.len[j], kk);
                    r0[q] = u.x;
                    r0[q + 1] = u.y;
                    r1[q] = u.y;
                    r1[q + 1] = -u.x;
                    r2[q] = (float)kk * u.y;
                    r2[q + 1] = -(float)kk * u.x;
                }
                uint4 H, Lo;
                split8(r0, H, Lo);
                *reinterpret_cast<uint4*>(Bhi + canon_off(3 * j + 0, c0, L::kKa)) = H;
                *reinterpret_cast<uint4*>(Blo + canon_off(3 * j + 0, c0, L::kKa)) = Lo;
                split8(r1, H, Lo);
                *reinterpret_cast<uint4*>(Bhi + canon_off(3 * j + 1, c0, L::kKa)) = H;
                *reinterpret_cast<uint4*>(Blo + canon_off(3 * j + 1, c0, L::kKa)) = Lo;
                split8(r2, H, Lo);
                *reinterpret_cast<uint4*>(Bhi + canon_off(3 * j + 2, c0, L::kKa)) = H;
                *reinterpret_cast<uint4*>(Blo + canon_off(3 * j + 2, c0, L::kKa)) = Lo;
            }
            fence_async_smem();
            producer_sync();   // the operand is complete
            if (prod == 0) mbar_arrive(bready_bar(st));   // records and B of the stage, released
        }
        // flush the batches still held by the stages
        for (int i = nbatch > kWsR ? nbatch - kWsR : 0; i < nbatch; ++i) {
            const int st = i % kWsR;
            if (!wait_ok(empty_bar(st), (uint32_t)(i / kWsR) & 1u)) break;
            tc_fence_after();
            flush(i, st);
        }
    } else if (issuer) {
        // ---------------- MMA-issuing warp: waits for a stage's operand, issues its products
        constexpr uint32_t idesc = make_idesc(128, 3 * kTbE);
        const uint32_t a_base = smem_u32(sm + L::kA), b_base = smem_u32(sm + L::kB);
        for (int i = 0; i < nbatch; ++i) {
            const int st = i % kWsR;
            if (!wait_ok(bready_bar(st), (uint32_t)(i / kWsR) & 1u)) break;
            if (lane == 0) {
                tc_fence_after();
                // descriptors of the K-step-0 core matrices; a K step is 256 bytes further,
                // i.e. +16 in the descriptor's address field (no carry: shared addresses < 256 KB)
                const uint64_t bd[3] = {make_desc(b_base + (st * 2 + 0) * L::kBTile, 128, L::kKa * 16),
                                        make_desc(b_base + (st * 2 + 0) * L::kBTile, 128, L::kKa * 16),
                                        make_desc(b_base + (st * 2 + 1) * L::kBTile, 128, L::kKa * 16)};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint64_t ad[3] = {make_desc(a_base + (h * 2 + 0) * L::kATile, 128, L::kKa * 16),
                                            make_desc(a_base + (h * 2 + 1) * L::kATile, 128, L::kKa * 16),
                                            make_desc(a_base + (h * 2 + 0) * L::kATile, 128, L::kKa * 16)};
                    const uint32_t d = tbase + (uint32_t)(st * L::kStageCols + h * 3 * kTbE);
#pragma unroll
                    for (int t = 0; t < 3; ++t)
#pragma unroll
                        for (int q = 0; q < L::kKa / 16; ++q)
                            mma_bf16(d, ad[t] + (uint64_t)(q * 16), bd[t] + (uint64_t)(q * 16), idesc,
                                     (t > 0 || q > 0) ? 1u : 0u);
                }
                mma_commit(full_bar(st));
                mbar_arrive(full_bar(st));   // the builders' release, passed on to the consumers
            }
            __syncwarp();
        }
        // no product may still be in flight when the CTA frees its TMEM (after an expired wait
        // the consumers leave without waiting for the last stage)
        if (lane == 0) tc_drain(drain_bar);
        __syncwarp();
    } else {
        // ---------------- consumer warps: one pixel per thread
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const float c_f0 = (float)(a.two_pi_over_c * (a.f0 + (double)k0 * a.df));
        const float c_df = (float)(a.two_pi_over_c * a.df);
        const int slot18 = rs18_slot(lane);
        const uint32_t wlast = __reduce_max_sync(0xffffffffu, last);   // the warp's walk
        // The walk in either direction (a compile-time flag).  Back to front from the pixel's
        // final state, acc = the sum over later entries of w reG a (the suffix); front to back
        // from T = 1 (the forward's own recursion), acc = the same sum over the entries up to
        // this one, so that the suffix is s_tot - acc.
        auto walk = [&](auto dir) {
            constexpr bool kFront = decltype(dir)::value;
            float acc = 0.f;
            for (int i = 0; i < nbatch; ++i) {
                const int st = i % kWsR;
                if (!wait_ok(full_bar(st), (uint32_t)(i / kWsR) & 1u)) break;
                tc_fence_after();
                const uint32_t lo_pos = batch_lo(i);
                const int nbp = batch_n(i);
                TbMeta mdp = tb_meta(sm + L::kMeta + st * L::kMetaStage);
                float v[3 * kTbE];
#pragma unroll
                for (int c = 0; c < 3 * kTbE; c += 16) {
                    float t16[16];
                    tmem_ld16(tbase + (uint32_t)(st * L::kStageCols + half * 3 * kTbE + c) + lane_base, t16);
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[c + q] = t16[q];
                }
                uint64_t mask = warp_entry_mask<false>(mdp.geo, mdp.geo2, mdp.ext, nbp, wcx, wcy, a.W);
                // positions at or past every pixel's n_contrib are live at none of the warp's pixels
                if (lo_pos >= wlast) mask = 0ull;
                else if (wlast - lo_pos < 64u) mask &= (1ull << (wlast - lo_pos)) - 1ull;
                if (lane == 0) mask_at(st, warp) = mask;
                // entries in pairs in walk order: both entries' alpha, gradient components and
                // warp reductions sit in one block so their latencies overlap
#pragma unroll
                for (int pp = 0; pp < kTbE / 2; ++pp) {
                    const int p = kFront ? pp : kTbE / 2 - 1 - pp;
                    const uint32_t pm = (uint32_t)(mask >> (2 * p)) & 3u;
                    if (!pm) continue;   // warp-uniform
                    float gr[2][9], dxv[2], dyv[2], Gv[2], alv[2];
                    bool live[2], clv[2];
                    int jv[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = kFront ? 2 * p + h : 2 * p + 1 - h;
                        jv[h] = j;
                        const float4 gg = mdp.geo[j];
                        const float2 g2 = mdp.geo2[j];
                        float dx = __fsub_rn(ux, gg.x);
                        const float hw = 0.5f * (float)a.W;
                        dx = dx >= hw ? __fsub_rn(dx, (float)a.W) : (dx < -hw ? __fadd_rn(dx, (float)a.W) : dx);
                        const float dy = __fsub_rn(uy, gg.y);
                        float q = __fmul_rn(__fmul_rn(g2.x, dy), dy);
                        q = __fmaf_rn(__fmul_rn(__fmul_rn(2.0f, gg.w), dx), dy, q);
                        q = __fmaf_rn(__fmul_rn(gg.z, dx), dx, q);
                        const float G = ex2(__fmul_rn(-0.5f * kLog2e, q));
                        const float a0 = __fmul_rn(g2.y, G);
                        clv[h] = a0 > kAlphaMax;
                        const float alpha = clv[h] ? kAlphaMax : a0;
                        live[h] = ((pm >> (j & 1)) & 1u) && lo_pos + (uint32_t)j < last && q <= kQMax &&
                                  alpha >= kAlphaMin;
                        alv[h] = live[h] ? alpha : 0.f;
                        Gv[h] = live[h] ? G : 0.f;
                        dxv[h] = live[h] ? dx : 0.f;
                        dyv[h] = live[h] ? dy : 0.f;
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = jv[h];
                        const float alpha = alv[h];
                        const float nl = live[h] ? lg2(__fsub_rn(1.0f, alpha)) : 0.f;
                        const float reG = v[3 * j], imG = v[3 * j + 1], imF = v[3 * j + 2];
                        const float amp = mdp.amp[j];
                        const float reGa = amp * reG;
                        float T, dalpha;
                        // (1 - alpha >= 0.01: the approximate quotient is within 2 ulp)
                        if (kFront) {
                            T = ex2(logT);
                            acc = fmaf(T * alpha, reGa, acc);
                            dalpha = T * reGa - __fdividef(s_tot - acc, 1.0f - alpha);
                            logT = __fadd_rn(logT, nl);
                        } else {
                            const float logT_before = __fsub_rn(logT, nl);
                            T = ex2(logT_before);
                            dalpha = T * reGa - __fdividef(acc, 1.0f - alpha);
                            acc = fmaf(T * alpha, reGa, acc);
                            logT = logT_before;
                        }
                        const float w = T * alpha;
                        gr[h][6] = w * reG;
                        gr[h][7] = -w * amp * imG;
                        gr[h][8] = w * amp * (c_f0 * imG + c_df * imF);
                        const float da = (live[h] && !clv[h]) ? dalpha : 0.f;
                        const float4 gg = mdp.geo[j];
                        const float2 g2 = mdp.geo2[j];
                        const float G = Gv[h], dx = dxv[h], dy = dyv[h];
                        gr[h][5] = da * G;
                        const float dq = -0.5f * da * g2.y * G;
                        gr[h][0] = dq * (-2.0f * (gg.z * dx + gg.w * dy));
                        gr[h][1] = dq * (-2.0f * (gg.w * dx + g2.x * dy));
                        gr[h][2] = dq * dx * dx;
                        gr[h][3] = dq * 2.0f * dx * dy;
                        gr[h][4] = dq * dy * dy;
                    }
                    if (__any_sync(0xffffffffu, live[0] || live[1])) {
                        // both entries' components reduced together, one per lane
                        float g18[18];
#pragma unroll
                        for (int c = 0; c < 9; ++c) {
                            g18[c] = gr[0][c];
                            g18[9 + c] = gr[1][c];
                        }
                        const float tsum = warp_reduce_scatter18(g18, lane);
                        if (slot18 >= 0)
                            red_at(st, warp, slot18 < 9 ? jv[0] : jv[1], slot18 < 9 ? slot18 : slot18 - 9) = tsum;
                    } else if (lane < 18) {
                        red_at(st, warp, lane < 9 ? jv[0] : jv[1], lane < 9 ? lane : lane - 9) = 0.f;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(empty_bar(st));
            }
        };
        if (front)
            walk(std::true_type{});
        else
            walk(std::false_type{});
    }
    tc_fence_before();
    __syncthreads();
    // an expired wait left the gradients incomplete: make that visible
    if (tid == 0 && *s_err != 0u) {
        set_status(a.status, GSPARC_ERR_TIMEOUT);
        atomicAdd(reinterpret_cast<float*>(&a.d_attr[(size_t)b * a.N]), __int_as_float(0x7fc00000));
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(L::kCols) : "memory");
    }
}

template <int S>
int launch_bwd_tc(const RenderArgs& a, int T, cudaStream_t s, uint32_t max_items = 0) {
    using L = RWsSmem<S>;
    if (!ensure_smem_attr(k_render_bwd_ws<S>, L::kTotal)) return GSPARC_ERR_CUDA;
    if (a.items) return launch_after(GSPARC_OVERLAP_BACKWARD, k_render_bwd_ws<S>, dim3(max_items), dim3(kWsThreads), L::kTotal, s, a);
    dim3 grid((a.K + S - 1) / S, T, a.B);
    return launch_after(GSPARC_OVERLAP_BACKWARD, k_render_bwd_ws<S>, grid, dim3(kWsThreads), L::kTotal, s, a);
}

int launch_bwd_tc_any(const RenderArgs& a, int T, cudaStream_t s, uint32_t max_items = 0) {
    if (a.K <= 8) return launch_bwd_tc<8>(a, T, s, max_items);
    if (a.K <= 16) return launch_bwd_tc<16>(a, T, s, max_items);
    if (a.K <= 32) return launch_bwd_tc<32>(a, T, s, max_items);
    return launch_bwd_tc<64>(a, T, s, max_items);
}

}  // namespace
}  // namespace gsparc

extern "C" int gsparc_render_bwd_tc(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                                    const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                                    const float* attr, const float* final_logT, const uint32_t* n_contrib,
                                    const float* d_spectrum, float* d_attr, float* d_proj, int32_t* d_status, void* stream) {
    using namespace gsparc;
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr)) return GSPARC_ERR_INVALID;
    if (!final_logT || !n_contrib || !d_spectrum || !d_attr || !d_proj) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_spectrum) & 7) || (reinterpret_cast<uintptr_t>(d_attr) & 15))
        return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.spin = wait_limit(kSpin);
    a.final_logT = const_cast<float*>(final_logT);
    a.n_contrib = const_cast<uint32_t*>(n_contrib);
    a.d_spectrum = reinterpret_cast<const float2*>(d_spectrum);
    a.d_attr = reinterpret_cast<float4*>(d_attr);
    a.d_proj = d_proj;
    const int T = tiles_x(*view) * tiles_y(*view);
    return launch_bwd_tc_any(a, T, as_stream(stream));
}

extern "C" int gsparc_render_bwd_tc_workspace(const gsparc_view* view, const gsparc_band* band, int32_t B,
                                              size_t* ws_bytes) {
    using namespace gsparc;
    if (!view_ok(view) || !band || band->K <= 0 || band->K > 65535 || B <= 0 || B > 65535 || !ws_bytes)
        return GSPARC_ERR_INVALID;
    *ws_bytes = sched_layout(B, tiles_x(*view) * tiles_y(*view), strips_of(band->K)).total;
    return GSPARC_OK;
}

extern "C" int gsparc_render_bwd_tc_balanced(const gsparc_view* view, const gsparc_band* band, int32_t B,
                                             int32_t N, const float* proj, const uint32_t* tile_ranges,
                                             const uint32_t* sorted_ids, const float* attr,
                                             const float* spectrum, const float* s_tot, const uint32_t* tile_walk,
                                             const float* final_logT, const uint32_t* n_contrib,
                                             const float* d_spectrum, int32_t split_min, void* ws, size_t ws_bytes,
                                             float* d_attr, float* d_proj, int32_t* d_status, void* stream) {
    using namespace gsparc;
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr)) return GSPARC_ERR_INVALID;
    if (!final_logT || !n_contrib || !d_spectrum || !d_attr || !d_proj || !ws) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_spectrum) | reinterpret_cast<uintptr_t>(spectrum)) & 7) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_attr) | reinterpret_cast<uintptr_t>(ws)) & 15) return GSPARC_ERR_INVALID;
    const int T = tiles_x(*view) * tiles_y(*view), strips = strips_of(band->K);
    const SchedLayout SL = sched_layout(B, T, strips);
    if (ws_bytes < SL.total) return GSPARC_ERR_INVALID;
    const int64_t units = (int64_t)B * T * strips;
    if (2 * units >= (1ll << 31)) return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.spin = wait_limit(kSpin);
    a.spectrum = const_cast<float2*>(reinterpret_cast<const float2*>(spectrum));
    a.s_tot = const_cast<float*>(s_tot);
    a.final_logT = const_cast<float*>(final_logT);
    a.n_contrib = const_cast<uint32_t*>(n_contrib);
    a.d_spectrum = reinterpret_cast<const float2*>(d_spectrum);
    a.d_attr = reinterpret_cast<float4*>(d_attr);
    a.d_proj = d_proj;
    char* w = static_cast<char*>(ws);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(w + SL.hdr);
    a.items = reinterpret_cast<const uint4*>(w + SL.items);
    a.n_items = hdr + 1;
    cudaStream_t s = as_stream(stream);
    // splitting only pays while the units are too few to keep every SM busy
    const int allow_split = units <= 2 * (int64_t)num_sms() ? 1 : 0;
    // without s_tot or the spectrum a front chunk has no suffix: order the walks, split none
    const int smin = (!spectrum && !s_tot) ? -1 : (split_min == 0 ? kSplitMinDefault : split_min);
    if (launch_after(GSPARC_OVERLAP_SCHEDULE, k_bwd_schedule, dim3(tile_walk ? 1u : (unsigned)(B * T)), dim3(kSchedThreads), 0, s, view->H,
                     view->W, tiles_x(*view), T, B * T, strips, smin, allow_split, a.ranges, n_contrib, tile_walk,
                     hdr, reinterpret_cast<uint32_t*>(w + SL.walks),
                     reinterpret_cast<uint4*>(w + SL.items)) != GSPARC_OK)
        return GSPARC_ERR_CUDA;
    return launch_bwd_tc_any(a, T, s, (uint32_t)(2 * units));
}

extern "C" int gsparc_render_bwd_workspace(const gsparc_view* view, const gsparc_band* band, int32_t B,
                                           size_t* ws_bytes) {
    using namespace gsparc;
    if (!view_ok(view) || !band || band->K <= 0 || band->K > 65535 || B <= 0 || B > 65535 || !ws_bytes)
        return GSPARC_ERR_INVALID;
    *ws_bytes = sched_layout(B, tiles_x(*view) * tiles_y(*view), fp32_strips(band->K)).total;
    return GSPARC_OK;
}

extern "C" int gsparc_render_bwd_balanced(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                                          const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                                          const float* attr, const float* spectrum, const float* s_tot,
                                          const uint32_t* tile_walk, const float* final_logT, const uint32_t* n_contrib,
                                          const float* d_spectrum, int32_t split_min, void* ws, size_t ws_bytes,
                                          float* d_attr, float* d_proj, int32_t* d_status, void* stream) {
    using namespace gsparc;
    if (!common_ok(view, band, B, N, proj, tile_ranges, sorted_ids, attr)) return GSPARC_ERR_INVALID;
    if (!final_logT || !n_contrib || !d_spectrum || !d_attr || !d_proj || !ws) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_spectrum) | reinterpret_cast<uintptr_t>(spectrum)) & 7) return GSPARC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_attr) | reinterpret_cast<uintptr_t>(ws)) & 15) return GSPARC_ERR_INVALID;
    const int T = tiles_x(*view) * tiles_y(*view), strips = fp32_strips(band->K);
    const SchedLayout SL = sched_layout(B, T, strips);
    if (ws_bytes < SL.total) return GSPARC_ERR_INVALID;
    const int64_t units = (int64_t)B * T * strips;
    if (2 * units >= (1ll << 31)) return GSPARC_ERR_INVALID;
    RenderArgs a{};
    fill_args(view, band, B, N, proj, tile_ranges, sorted_ids, attr, a);
    a.status = d_status;
    a.spectrum = const_cast<float2*>(reinterpret_cast<const float2*>(spectrum));
    a.s_tot = const_cast<float*>(s_tot);
    a.final_logT = const_cast<float*>(final_logT);
    a.n_contrib = const_cast<uint32_t*>(n_contrib);
    a.d_spectrum = reinterpret_cast<const float2*>(d_spectrum);
    a.d_attr = reinterpret_cast<float4*>(d_attr);
    a.d_proj = d_proj;
    a.T = T;
    char* w = static_cast<char*>(ws);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(w + SL.hdr);
    a.items = reinterpret_cast<const uint4*>(w + SL.items);
    a.n_items = hdr + 1;
    cudaStream_t s = as_stream(stream);
    // two CTAs per SM: splitting pays while the units are too few to fill them twice over
    const int allow_split = units <= 4 * (int64_t)num_sms() ? 1 : 0;
    const int smin = (!spectrum && !s_tot) ? -1 : (split_min == 0 ? kSplitMinDefault : split_min);
    if (launch_after(GSPARC_OVERLAP_SCHEDULE, k_bwd_schedule, dim3(tile_walk ? 1u : (unsigned)(B * T)), dim3(kSchedThreads), 0, s, view->H,
                     view->W, tiles_x(*view), T, B * T, strips, smin, allow_split, a.ranges, n_contrib, tile_walk,
                     hdr, reinterpret_cast<uint32_t*>(w + SL.walks),
                     reinterpret_cast<uint4*>(w + SL.items)) != GSPARC_OK)
        return GSPARC_ERR_CUDA;
    return launch_bwd_any(a, T, s, (uint32_t)(2 * units));
}
