// Front-to-back compositing of complex per-subcarrier contributions and its
// gradient.
//
// Sec. 4.2 compositing rule S = sum_i alpha_i prod_{j<i}(1 - alpha_j) s_i / d_i
// with alpha_i = sigma_i G_i'; Algorithm 1 inner loop (T <- 1, z += T alpha s,
// T *= 1 - alpha).  The subcarrier k enters as the delay phase of the path
// length L_i (Sec. 3.1 channel model): s_ik = a_i exp(j(phi0_i - 2 pi f_k L_i / c)).
//
// Work item = (transmitter b, 16x16 tile, strip of S subcarriers); one CTA of
// 256 threads per item, one pixel per thread, S complex accumulators per
// thread.  Gaussian batches of the tile's sorted list are staged in shared
// memory by bulk asynchronous copies (one batch ahead of the compositing)
// together with their unit phasors e^{j psi_ik} for the strip, so the
// per-(pixel, Gaussian, subcarrier) work is one paired FMA (forward) or two paired
// FMAs and a paired add (backward) against broadcast shared-memory reads.  A warp
// visits only the entries that can be live at one of its pixels (an exact bound of q
// over its 16x2 block, and in the backward the warp's own walk).  Transmittance is carried
// as log2 T in FP32; a thread stops before T would fall below 1e-4 and the
// CTA stops fetching once every thread has stopped.  The backward can run as
// scheduled chunks of the walks (the items of k_bwd_schedule).
//
// This header holds what the FP32 kernels and the tensor-core kernels share (arguments, alpha,
// unit phasors, batch staging) and the FP32 kernels themselves, as device code with no runtime
// API, so that the same source also builds for the host under the test suite's shim (which
// defines GSPARC_HOST_SHIM and gets exp2f / log2f for the SFU's ex2 / lg2).  Launches and entry
// points are in render.cu.

#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include "device_common.cuh"

namespace gsparc {
namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 64;
constexpr float kLog2e = 1.4426950408889634f;

#ifndef GSPARC_HOST_SHIM
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// Two FP32 FMAs in one instruction (the paired FFMA of sm_100+): d.x = fma(a.x, b.x, c.x),
// d.y = fma(a.y, b.y, c.y), each an IEEE single-precision fused multiply-add, as fmaf.  The
// runtime's intrinsic keeps the operands in register pairs without repacking.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// Two FP32 additions in one instruction, each an IEEE single-precision add.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
#else
// the test suite's host shim: the library's exact counterparts of the SFU approximations
inline float ex2(float x) { return exp2f(x); }
inline float lg2(float x) { return log2f(x); }
inline float2 fma2(float2 a, float2 b, float2 c) { return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
inline float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
#endif

struct RenderArgs {
    int H, W, TW, K, N, B;
    const float4* proj;     // [N][2]
    const uint2* ranges;    // [T]
    const uint32_t* ids;    // sorted Gaussian ids
    const float4* attr;     // [B][N]
    float2* spectrum;       // [B][K][H][W]
    float* final_logT;      // [B][H][W]
    uint32_t* n_contrib;    // [B][H][W]
    uint32_t* n_used;       // [B][H][W]
    const float2* d_spectrum;
    float4* d_attr;         // [B][N]
    float* d_proj;          // [N][8]
    float2* csi;            // [B][K] spatial-mean accumulator (fused CSI head), or null
    float csi_scale;        // 1 / HW
    const float2* l2_target;   // [B][K][H][W] (fused L2 loss), with:
    float* l2_loss;            // [1] accumulator of mean |z - target|^2
    float2* l2_grad;           // [B][K][H][W] out: 2 (z - target) / count, or null
    float l2_inv;              // 1 / count
    // [B][strips][H][W]: Re sum_k conj(dL/dz_k) z_k over each strip of S subcarriers (written by
    // the fused L2 forward when not null; read by the front chunks of the scheduled backward)
    float* s_tot;
    // [B][T]: the walk of each (transmitter, tile), min(largest n_contrib, list length), written
    // by the tensor-core forward when not null (the scheduled backward's cost per tile)
    uint32_t* tile_walk;
    // Scheduled tensor-core backward: work item r of the ordered list runs on block r
    // (x = b * T + tile, y = strip | front flag << 31, entries [z, w) of the walk), or null
    // for one block per (strip, tile, transmitter).
    const uint4* items;
    const uint32_t* n_items;
    int T;                     // tiles per image
    // caller's status word (may be null): GSPARC_ERR_INPUT for a list id outside the scene,
    // GSPARC_ERR_TIMEOUT for an expired wait of the tensor-core kernels
    int32_t* status;
    // polls before a pipeline wait of the tensor-core kernels gives up
    uint32_t spin;
    // the spectrum is written with evict-first stores (a large output would otherwise push the
    // Gaussians' records out of L2 while the kernel still gathers them)
    bool stream_out;
    // cycles of subcarrier k = L * (lam0_hi + lam0_lo + k * dlam), lam = f / c
    float lam0_hi, lam0_lo, dlam;
    // d(psi)/dL = -2 pi f_k / c, split as c_f0 + kk * c_df inside a strip
    double two_pi_over_c;
    double f0, df;
};

// alpha of a staged Gaussian at a pixel centre; identical in both passes so
// that the backward pass re-takes exactly the forward's decisions.
// Returns false when the Gaussian is skipped (q > q_max or alpha < 1/255).
__device__ __forceinline__ bool eval_alpha(float ux, float uy, int W, const float4 g, const float2 g2,
                                           float& dx, float& dy, float& G, float& alpha,
                                           bool& clamped) {
    // Explicitly rounded operations: no contraction choice of the compiler
    // can make the two passes disagree.
    dx = __fsub_rn(ux, g.x);
    const float hw = 0.5f * (float)W;
    if (dx >= hw) dx = __fsub_rn(dx, (float)W);
    else if (dx < -hw) dx = __fadd_rn(dx, (float)W);
    dy = __fsub_rn(uy, g.y);
    float q = __fmul_rn(__fmul_rn(g2.x, dy), dy);
    q = __fmaf_rn(__fmul_rn(__fmul_rn(2.0f, g.w), dx), dy, q);
    q = __fmaf_rn(__fmul_rn(g.z, dx), dx, q);
    if (!(q <= kQMax)) return false;
    G = ex2(__fmul_rn(-0.5f * kLog2e, q));
    const float a = __fmul_rn(g2.y, G);
    clamped = a > kAlphaMax;
    alpha = clamped ? kAlphaMax : a;
    return alpha >= kAlphaMin;
}

// Unit phasor e^{j psi_k} of a Gaussian with path length L and phase offset phi0 at
// subcarrier k: psi = phi0 - 2 pi f_k L / c.  The cycle count L f_k / c (~10^2) is formed
// with an error-free product of the split f_0 / c, reduced to [-1/2, 1/2], and the angle
// 2 pi c (in [-pi, pi]) goes to the SFU sine/cosine.
__device__ __forceinline__ float2 unit_phasor(const RenderArgs& a, float L, float phi0, int k) {
    const float p = L * a.lam0_hi;
    const float e0 = fmaf(L, a.lam0_hi, -p);
    float c = (p - rintf(p)) + (e0 + L * a.lam0_lo);
    c += L * ((float)k * a.dlam);
    c -= phi0 * 0.15915494309189535f;
    c -= rintf(c);
    float sn, cs;
    __sincosf(6.283185307179586f * c, &sn, &cs);
    return make_float2(cs, -sn);   // e^{j psi} = e^{-j 2 pi c}
}

// The phase of a Gaussian's unit phasor at subcarrier k0 as cycles reduced to [-1/2, 1/2] (the
// steps of unit_phasor before the sine/cosine) and its step per subcarrier L df / c: the phasor at
// subcarrier k0 + kk is then phasor_at(c0, step, kk).  For kk below 64 the product kk step adds
// under 2e-7 cycles of rounding (a phase error below 1e-6 rad).
__device__ __forceinline__ float phase_base(const RenderArgs& a, float L, float phi0, int k0) {
    const float p = L * a.lam0_hi;
    const float e0 = fmaf(L, a.lam0_hi, -p);
    float c = (p - rintf(p)) + (e0 + L * a.lam0_lo);
    c += L * ((float)k0 * a.dlam);
    c -= phi0 * 0.15915494309189535f;
    return c - rintf(c);
}
__device__ __forceinline__ float2 phasor_at(float c0, float step, int kk) {
    float c = fmaf((float)kk, step, c0);
    c -= rintf(c);
    float sn, cs;
    __sincosf(6.283185307179586f * c, &sn, &cs);
    return make_float2(cs, -sn);   // e^{j psi} = e^{-j 2 pi c}
}

// ---------------------------------------------------------------------------------------------
// Staging of a batch's records for the FP32 kernels.  Entry j of a batch is its 32-byte
// projection record and 16-byte attribute record, brought into shared memory by two 1-D bulk
// asynchronous copies (cp.async.bulk, the TMA engine) that complete on the batch's mbarrier.
// The records are double-buffered: the copies of batch i + 1 are issued once every warp has
// finished batch i - 1 and fly while batch i is composited.  Under the test suite's host shim the
// copies are plain copies and the barrier is already complete.
// ---------------------------------------------------------------------------------------------

struct StageRec {
    float4 p0;   // p_x, p_y, ext_x, ext_y
    float4 p1;   // c_xx, c_xy, c_yy, r
    float4 at;   // a, phi0, sigma, L
};

#ifndef GSPARC_HOST_SHIM
__device__ __forceinline__ uint32_t smem_addr32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// one arrival per entry slot of a batch (kBatch), each with the bytes of its copies
__device__ __forceinline__ void stage_bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr32(bar)), "n"(kBatch) : "memory");
}
__device__ __forceinline__ void stage_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// generic-proxy accesses to the buffer before this point are ordered before the copies after it
__device__ __forceinline__ void stage_proxy_fence() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// the one arrival of the batch's phase, with the bytes its copies will deliver
__device__ __forceinline__ void stage_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void stage_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr32(bar))
                 : "memory");
}
// bounded wait for the phase of the given parity; false when `polls` polls found it incomplete
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity, uint32_t polls) {
    const uint32_t addr = smem_addr32(bar);
    for (uint32_t it = 0; it < polls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
#else
inline void stage_bar_init(uint64_t* bar) { *bar = 0; }
inline void stage_init_fence() {}
inline void stage_proxy_fence() {}
inline void stage_expect(uint64_t*, uint32_t) {}
inline void stage_copy(void* dst, const void* src, uint32_t bytes, uint64_t*) { memcpy(dst, src, bytes); }
// every thread of the block waits at the same program point, so a block barrier stands for the
// mbarrier: each copy was made when its issuing thread ran
inline bool stage_wait(uint64_t*, uint32_t, uint32_t) {
    __syncthreads();
    return true;
}
#endif

constexpr uint32_t kStagePolls = 1u << 22;   // bound of a staging wait (far above a healthy copy)

// Stage batch entries [list_pos, list_pos + nb) of the tile list (their ids already loaded,
// one per thread in `gid`, tid < nb) into rec: every thread tid < kBatch makes one arrival on the
// batch's mbarrier (initialised for kBatch arrivals), a thread with an entry announcing the 48
// bytes its two bulk copies deliver.  An id outside the scene (inconsistent inputs) gets a record
// with a NaN conic instead, so that every pixel skips it and it receives no gradient, and the
// status word says so.
__device__ __forceinline__ void stage_issue(const RenderArgs& a, int b, int nb, uint32_t gid, StageRec* rec,
                                            uint32_t* s_gid, uint64_t* bar) {
    const int tid = threadIdx.x;
    if (tid >= kBatch) return;
    if (tid < nb && gid < (uint32_t)a.N) {
        s_gid[tid] = gid;
        stage_expect(bar, 48u);
        stage_copy(&rec[tid].p0, a.proj + 2 * (size_t)gid, 32u, bar);
        stage_copy(&rec[tid].at, a.attr + (size_t)b * a.N + gid, 16u, bar);
    } else {
        if (tid < nb) {
            set_status(a.status, GSPARC_ERR_INPUT);
            rec[tid].p0 = make_float4(0.f, 0.f, -1.f, -1.f);
            rec[tid].p1 = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
            rec[tid].at = make_float4(0.f, 0.f, 0.f, 0.f);
            s_gid[tid] = 0u;
        }
        stage_expect(bar, 0u);
    }
}

// Unit phasors of R consecutive subcarriers k0 .. k0 + R - 1 of one Gaussian: the first by
// unit_phasor, each next one by a complex product with the step e^{-j 2 pi L df / c} (the
// cycles L df / c per subcarrier, reduced, to the SFU sine/cosine), so that at most R - 1 <= 7
// roundings of a product separate a phasor from its directly computed value (relative error
// ~1e-6, far below the 1e-3 bound on spectra).
template <int R>
__device__ __forceinline__ void phasor_run(const RenderArgs& a, float L, float phi0, int k0, float2 (&u)[R]) {
    u[0] = unit_phasor(a, L, phi0, k0);
    if constexpr (R > 1) {
        float c = L * a.dlam;
        c -= rintf(c);
        float sn, cs;
        __sincosf(6.283185307179586f * c, &sn, &cs);
        const float dx = cs, dy = -sn;   // e^{-j 2 pi c}
#pragma unroll
        for (int m = 1; m < R; ++m) {
            const float x = u[m - 1].x, y = u[m - 1].y;
            u[m] = make_float2(fmaf(x, dx, -y * dy), fmaf(x, dy, y * dx));
        }
    }
}

// Unit phasors of the strip's subcarriers for the nb entries of rec (every thread), into tab:
// each thread forms runs of up to 8 consecutive subcarriers of one entry (phasor_run).  In a
// float4 table every element is (t, -j conj t) = (t.x, t.y, t.y, -t.x), the backward's form: for an
// upstream gradient g both Re(conj(g) t) = g.x t.x + g.y t.y and Im(conj(g) t) = g.x t.y - g.y t.x
// are then one paired FMA of (g.x, g.y) against one half.  (The forward uses it.)
template <int S, class E>
__device__ __forceinline__ void stage_phasor_runs(const RenderArgs& a, const StageRec* rec, int nb, int k0,
                                                  E (*tab)[S]) {
    constexpr int R = S >= 8 ? 8 : S, NR = S / R;
    for (int it = threadIdx.x; it < nb * NR; it += kThreads) {
        const int j = it / NR, kk0 = (it - j * NR) * R;
        float2 u[R];
        if (k0 + kk0 < a.K) {
            phasor_run<R>(a, rec[j].at.w, rec[j].at.y, k0 + kk0, u);
        } else {
#pragma unroll
            for (int m = 0; m < R; ++m) u[m] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const float2 t = k0 + kk0 + m < a.K ? u[m] : make_float2(0.f, 0.f);
            if constexpr (sizeof(E) == 16) tab[j][kk0 + m] = make_float4(t.x, t.y, t.y, -t.x);
            else tab[j][kk0 + m] = t;
        }
    }
}

template <int S>
__device__ __forceinline__ void stage_phasors(const RenderArgs& a, const StageRec* rec, int nb, int k0,
                                              float2 (*tab)[S]) {
    stage_phasor_runs<S>(a, rec, nb, k0, tab);
}
// The backward's table, each phasor formed on its own (unit_phasor): the backward waits for its
// table at every batch, and eight independent phasors per thread finish sooner than a run of
// eight dependent products.
template <int S>
__device__ __forceinline__ void stage_phasors_bwd(const RenderArgs& a, const StageRec* rec, int nb, int k0,
                                                  float4 (*tab)[S]) {
    for (int e = threadIdx.x; e < nb * S; e += kThreads) {
        const int j = e / S, kk = e - j * S;
        const int k = k0 + kk;
        float2 t = make_float2(0.f, 0.f);
        if (k < a.K) t = unit_phasor(a, rec[j].at.w, rec[j].at.y, k);
        tab[j][kk] = make_float4(t.x, t.y, t.y, -t.x);
    }
}

// Whether an entry can be live at a pixel of a warp's 16x2 block of pixel centres (centre
// (wcx, wcy)): centre p, footprint half extents e, conic (cxx, cxy, cyy), opacity sig.  First the
// footprint box test (the bounding box of q <= q_max, with a 0.01 px margin for rounding at its
// edge); then the smallest q over the block (each of its two pixel rows is a quadratic in the
// column offset, minimised over the row's continuous extent, which bounds the minimum over its
// pixel centres from below) against the smaller of q_max and the q at which
// alpha = sigma e^{-q/2} falls to 1/255, with a margin of 0.01 far above the rounding of either
// side.  False therefore means eval_alpha skips the entry at every pixel of the block.  A block
// that reaches the antipode of the entry's centre (where the azimuth wrap could split its
// columns) keeps the box test's answer.
// With kExact false only the box test is made (a superset of the entries, cheaper per entry).
template <bool kExact = true>
__device__ __forceinline__ bool entry_reaches_block(float px, float py, float ex, float ey, float cxx, float cxy,
                                                    float cyy, float sig, float wcx, float wcy, int W) {
    const float hw = 0.5f * (float)W;
    float dx = wcx - px;
    if (dx >= hw) dx -= (float)W;
    else if (dx < -hw) dx += (float)W;
    const float dy = wcy - py;
    bool hit = ex >= 0.f && fabsf(dx) <= ex + 7.51f && fabsf(dy) <= ey + 0.51f;
    if (kExact && hit && fabsf(dx) < hw - 8.0f) {
        // alpha >= 1/255  <=>  q <= 2 ln(255 sigma)
        const float q_op = 2.0f * 0.6931471805599453f * lg2(255.0f * sig);
        const float thr = fminf(kQMax, q_op) + 0.01f;
        float qmin = 3.0e38f;
#pragma unroll
        for (int row = 0; row < 2; ++row) {
            const float dr = dy + (row ? 0.5f : -0.5f);
            const float t = fminf(fmaxf(__fdividef(-cxy * dr, cxx), dx - 7.5f), dx + 7.5f);
            qmin = fminf(qmin, (cxx * t + 2.0f * cxy * dr) * t + cyy * dr * dr);
        }
        hit = qmin <= thr;
    }
    return hit;
}

// Bit j set when staged entry j (of nb) can be live at a pixel of the warp's block
// (entry_reaches_block), over staged records.
__device__ __forceinline__ uint64_t warp_entry_mask_rec(const StageRec* rec, int nb, float wcx, float wcy, int W) {
    const int lane = threadIdx.x & 31;
    bool h[2] = {false, false};
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int j = lane + 32 * half;
        if (j < nb) {
            const StageRec& r = rec[j];
            h[half] = entry_reaches_block(r.p0.x, r.p0.y, r.p0.z, r.p0.w, r.p1.x, r.p1.y, r.p1.z, r.at.z, wcx, wcy, W);
        }
    }
    const uint32_t lo = __ballot_sync(0xffffffffu, h[0]);
    const uint32_t hi = __ballot_sync(0xffffffffu, h[1]);
    return ((uint64_t)hi << 32) | lo;
}

// The same over the tensor-core kernels' staging: s_geo (p_x, p_y, c_xx, c_xy), s_geo2 (c_yy,
// sigma), s_ext (half extents; negative for a culled or invalid entry).  kExact false: the box
// test alone (the tensor-core backward, where the mask sits on each batch's critical path and the
// entries it would drop are skipped by the live test at little cost).
template <bool kExact = true>
__device__ __forceinline__ uint64_t warp_entry_mask(const float4* s_geo, const float2* s_geo2, const float2* s_ext,
                                                    int nb, float wcx, float wcy, int W) {
    const int lane = threadIdx.x & 31;
    bool h[2] = {false, false};
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int j = lane + 32 * half;
        if (j < nb) {
            const float4 g = s_geo[j];
            const float2 g2 = s_geo2[j];
            const float2 e = s_ext[j];
            h[half] = entry_reaches_block<kExact>(g.x, g.y, e.x, e.y, g.z, g.w, g2.x, g2.y, wcx, wcy, W);
        }
    }
    const uint32_t lo = __ballot_sync(0xffffffffu, h[0]);
    const uint32_t hi = __ballot_sync(0xffffffffu, h[1]);
    return ((uint64_t)hi << 32) | lo;
}

// Sum of v[c] over the 32 lanes of the warp for c < 9, returned in lane 2c (and
// 2c + 1): four halving exchange rounds (8 + 4 + 2 + 1 shuffles) then one final
// pairwise add, instead of a full butterfly per component.
__device__ __forceinline__ float warp_reduce_scatter9(const float (&v)[9], int lane) {
    float a[8];
    const bool b4 = (lane >> 4) & 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float lo = v[i];
        const float hi = (i + 8 < 9) ? v[i + 8] : 0.f;
        const float send = b4 ? lo : hi;
        const float keep = b4 ? hi : lo;
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float b[4];
    const bool b3 = (lane >> 3) & 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b3 ? a[i] : a[i + 4];
        const float keep = b3 ? a[i + 4] : a[i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c[2];
    const bool b2 = (lane >> 2) & 1;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b2 ? b[i] : b[i + 2];
        const float keep = b2 ? b[i + 2] : b[i];
        c[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const bool b1 = (lane >> 1) & 1;
    float d = (b1 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b1 ? c[0] : c[1], 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
}

// Sums over the 32 lanes of v[0..17] (two entries' nine components), one component per
// lane: five halving exchange rounds of 9, 5, 3, 2 and 1 shuffles (a round pads its vector
// with a zero when it has odd length).  The lane holds component rs18_slot(lane).
__device__ __forceinline__ float warp_reduce_scatter18(const float (&v)[18], int lane) {
    const bool u4 = (lane >> 4) & 1, u3 = (lane >> 3) & 1, u2 = (lane >> 2) & 1, u1 = (lane >> 1) & 1;
    const bool u0 = lane & 1;
    float a[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float lo = v[i], hi = v[i + 9];
        a[i] = (u4 ? hi : lo) + __shfl_xor_sync(0xffffffffu, u4 ? lo : hi, 16);
    }
    float b[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float lo = a[i], hi = i + 5 < 9 ? a[i + 5] : 0.f;
        b[i] = (u3 ? hi : lo) + __shfl_xor_sync(0xffffffffu, u3 ? lo : hi, 8);
    }
    float c[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float lo = b[i], hi = i + 3 < 5 ? b[i + 3] : 0.f;
        c[i] = (u2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, u2 ? lo : hi, 4);
    }
    float d[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float lo = c[i], hi = i + 2 < 3 ? c[i + 2] : 0.f;
        d[i] = (u1 ? hi : lo) + __shfl_xor_sync(0xffffffffu, u1 ? lo : hi, 2);
    }
    return (u0 ? d[1] : d[0]) + __shfl_xor_sync(0xffffffffu, u0 ? d[0] : d[1], 1);
}

// Component of warp_reduce_scatter18 held by a lane (0..17), or -1: the kept half's index
// through the five rounds, valid while it never falls on a padding zero.
__device__ __forceinline__ int rs18_slot(int lane) {
    const int sd = lane & 1;
    const int sc = sd + 2 * ((lane >> 1) & 1);
    const int sb = sc + 3 * ((lane >> 2) & 1);
    const int sa = sb + 5 * ((lane >> 3) & 1);
    const int sv = sa + 9 * ((lane >> 4) & 1);
    return (sc <= 2 && sb <= 4 && sa <= 8) ? sv : -1;
}

// Shared memory of the FP32 kernels (dynamic): records, phasor tables and ids of two batches,
// the two staging mbarriers and a few words.  A phasor-table element is TE bytes: the unit phasor
// (8, forward) or the phasor beside its quarter turn (16, backward: see stage_phasors_bwd).
template <int S, int TE = 8>
struct F32Smem {
    static constexpr int kRec = 0;                                        // StageRec[2][kBatch]
    static constexpr int kRow = S;                                        // table row
    static constexpr int kTab = kRec + 2 * kBatch * (int)sizeof(StageRec);  // [2][kBatch][kRow] elements
    static constexpr int kGid = kTab + 2 * kBatch * kRow * TE;            // uint32[2][kBatch]
    static constexpr int kBar = kGid + 2 * kBatch * 4;                    // uint64[2]
    static constexpr int kMisc = kBar + 16;                               // float[8], uint32[4]
    static constexpr int kTotal = kMisc + 48;
    static_assert(kTab % 16 == 0 && kBar % 8 == 0, "shared-memory alignment");
};
template <int S>
using F32BwdSmem = F32Smem<S, 16>;

// Batch i of a walk over list positions [lo, end): front to back from lo, or back to front
// from end (the last batch then the ragged one).
__device__ __forceinline__ void batch_span(bool front, uint32_t lo, uint32_t end, int i, uint32_t& b_lo, int& nb) {
    if (front) {
        b_lo = lo + (uint32_t)i * kBatch;
        nb = (int)min((uint32_t)kBatch, end - b_lo);
    } else {
        const uint32_t hp = end - (uint32_t)i * kBatch;
        b_lo = hp > lo + kBatch ? hp - kBatch : lo;
        nb = (int)(hp - b_lo);
    }
}

// The forward: one CTA per (strip of S subcarriers, tile, transmitter), one pixel per thread, S
// complex accumulators per thread.  With a.l2_grad the complex L2 loss is fused into the
// epilogue (dL/dz written, bit-identical to gsparc_l2_loss on this spectrum; the loss added
// atomically), with s_tot and the tile walks written for the scheduled backward when given.
template <int S>
__global__ void __launch_bounds__(kThreads, 2) k_render_fwd(RenderArgs a) {
    using L = F32Smem<S>;
    GSPARC_DYNAMIC_SMEM(sm);
    StageRec* s_rec = reinterpret_cast<StageRec*>(sm + L::kRec);
    float2(*s_tab)[kBatch][L::kRow] = reinterpret_cast<float2(*)[kBatch][L::kRow]>(sm + L::kTab);
    uint32_t* s_gid = reinterpret_cast<uint32_t*>(sm + L::kGid);
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(sm + L::kBar);
    float* s_part = reinterpret_cast<float*>(sm + L::kMisc);
    uint32_t* s_walk = reinterpret_cast<uint32_t*>(sm + L::kMisc + 32);
    uint32_t* s_err = s_walk + 1;
    grid_dep_wait();     // the tile lists and attributes of the kernels before

    const int strip = blockIdx.x, tile = blockIdx.y, b = blockIdx.z;
    const int k0 = strip * S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx0 = (tile % a.TW) * kTile, ty0 = (tile / a.TW) * kTile;
    const int x = tx0 + (tid & 15);
    const int y = ty0 + (tid >> 4);
    const bool inside = x < a.W && y < a.H;
    const float ux = (float)x + 0.5f, uy = (float)y + 0.5f;
    const float wcx = (float)tx0 + 8.0f, wcy = (float)(ty0 + 2 * warp) + 1.0f;
    const uint2 range = a.ranges[tile];
    const uint32_t len = range.y - range.x;
    const int nbatch = (int)((len + kBatch - 1) / kBatch);

    if (tid == 0) {
        stage_bar_init(&s_bar[0]);
        stage_bar_init(&s_bar[1]);
        stage_init_fence();
        *s_walk = 0u;
        *s_err = 0u;
    }
    // list ids one batch ahead of the copies
    auto load_id = [&](int i) -> uint32_t {
        const uint32_t p = (uint32_t)i * kBatch + (uint32_t)tid;
        return (tid < kBatch && i < nbatch && p < len) ? a.ids[range.x + p] : 0xffffffffu;
    };
    uint32_t pf_id = load_id(0);
    __syncthreads();
    if (nbatch > 0) stage_issue(a, b, (int)min((uint32_t)kBatch, len), pf_id, s_rec, s_gid, &s_bar[0]);
    pf_id = load_id(1);

    float2 acc[S];
#pragma unroll
    for (int kk = 0; kk < S; ++kk) acc[kk] = make_float2(0.f, 0.f);
    float logT = 0.f;
    uint32_t last = 0, used = 0;
    bool done = !inside;

    for (int i = 0; i < nbatch; ++i) {
        const int buf = i & 1;
        const uint32_t bs = (uint32_t)i * kBatch;
        const int nb = (int)min((uint32_t)kBatch, len - bs);
        if (!stage_wait(&s_bar[buf], (uint32_t)(i >> 1) & 1u, kStagePolls)) {
            *s_err = 1u;
            stage_wait(&s_bar[buf], (uint32_t)(i >> 1) & 1u, kStagePolls);   // copies still in flight
        }
        stage_phasors<S>(a, s_rec + buf * kBatch, nb, k0, s_tab[buf]);
        // phasors of batch i in place; every warp has finished batch i - 1, whose buffers the
        // copies of batch i + 1 now take over
        if (__syncthreads_or(!done) == 0 || *s_err) break;
        if (i + 1 < nbatch) {
            if (tid < kBatch) stage_proxy_fence();
            stage_issue(a, b, (int)min((uint32_t)kBatch, len - bs - kBatch), pf_id, s_rec + (buf ^ 1) * kBatch,
                        s_gid + (buf ^ 1) * kBatch, &s_bar[buf ^ 1]);
            pf_id = load_id(i + 2);
        }
        const StageRec* rec = s_rec + buf * kBatch;
        const uint64_t mask = warp_entry_mask_rec(rec, nb, wcx, wcy, a.W);
        if (__any_sync(0xffffffffu, !done)) {
            // groups of 8 entries.  alpha and log2(1 - alpha): eval_alpha's operations in its order
            // (the backward re-takes the same decisions; a skipped entry gets al = -1), branch-free
            // over the whole group when five or more of its entries can be live at the warp's pixels (the
            // eight evaluations overlap), entry by entry otherwise.  Then the transmittance
            // recursion and the accumulation in list order.  A group that misses the warp is skipped.
            auto alpha_of = [&](int j, float& al, float& nlv) {
                const StageRec& r = rec[j];
                float dx = __fsub_rn(ux, r.p0.x);
                const float hw = 0.5f * (float)a.W;
                dx = dx >= hw ? __fsub_rn(dx, (float)a.W) : (dx < -hw ? __fadd_rn(dx, (float)a.W) : dx);
                const float dy = __fsub_rn(uy, r.p0.y);
                float qf = __fmul_rn(__fmul_rn(r.p1.z, dy), dy);
                qf = __fmaf_rn(__fmul_rn(__fmul_rn(2.0f, r.p1.y), dx), dy, qf);
                qf = __fmaf_rn(__fmul_rn(r.p1.x, dx), dx, qf);
                const float G = ex2(__fmul_rn(-0.5f * kLog2e, qf));
                const float a0 = __fmul_rn(r.at.z, G);
                const float alpha = a0 > kAlphaMax ? kAlphaMax : a0;
                const bool ok = ((mask >> j) & 1ull) && qf <= kQMax && alpha >= kAlphaMin;
                al = ok ? alpha : -1.f;
                nlv = ok ? lg2(__fsub_rn(1.0f, alpha)) : 0.f;
            };
            auto composite = [&](int j, float al, float nlv) {
                const float nt = __fadd_rn(logT, nlv);
                const bool cand = !done && al >= 0.f;
                const bool term = cand && nt < kLog2TMin;
                done = done || term;
                const bool take = cand && !term;
                if (!__any_sync(0xffffffffu, take)) return;
                const float wa = take ? ex2(logT) * al * rec[j].at.x : 0.f;
                const float2 w2 = make_float2(wa, wa);
                if constexpr (S % 2 == 0) {
                    // two subcarriers' phasors per 16-byte broadcast read
                    const float4* t4 = reinterpret_cast<const float4*>(s_tab[buf][j]);
#pragma unroll
                    for (int k2 = 0; k2 < S / 2; ++k2) {
                        const float4 t = t4[k2];
                        acc[2 * k2] = fma2(w2, make_float2(t.x, t.y), acc[2 * k2]);
                        acc[2 * k2 + 1] = fma2(w2, make_float2(t.z, t.w), acc[2 * k2 + 1]);
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < S; ++kk) acc[kk] = fma2(w2, s_tab[buf][j][kk], acc[kk]);
                }
                logT = take ? nt : logT;
                last = take ? bs + (uint32_t)j + 1u : last;
                used += take ? 1u : 0u;
            };
#pragma unroll 1
            for (int g0 = 0; g0 < kBatch; g0 += 8) {
                const uint32_t gbits = (uint32_t)(mask >> g0) & 0xffu;
                if (gbits == 0u) continue;   // warp-uniform
                if (__popc(gbits) <= 4) {
                    for (uint32_t bits = gbits; bits; bits &= bits - 1u) {
                        const int j = g0 + __ffs((int)bits) - 1;
                        float al, nlv;
                        alpha_of(j, al, nlv);
                        composite(j, al, nlv);
                    }
                } else {
                    float al[8], nlv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) alpha_of(g0 + q, al[q], nlv[q]);
#pragma unroll
                    for (int q = 0; q < 8; ++q) composite(g0 + q, al[q], nlv[q]);
                }
            }
        }
    }
    if (*s_err) set_status(a.status, GSPARC_ERR_TIMEOUT);
    // epilogue: the spectrum, and with the fused loss dL/dz, the loss and s_tot
    const size_t plane = (size_t)a.H * a.W;
    const size_t pix = (size_t)y * a.W + x;
    float l2acc = 0.f, stot = 0.f;
    if (inside) {
#pragma unroll
        for (int k8 = 0; k8 < S; k8 += 8) {
            float2 t[8];
#pragma unroll
            for (int q = 0; q < 8 && k8 + q < S; ++q) {
                const int k = k0 + k8 + q;
                t[q] = (a.l2_grad && k < a.K) ? a.l2_target[((size_t)b * a.K + k) * plane + pix]
                                              : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8 && k8 + q < S; ++q) {
                const int k = k0 + k8 + q;
                if (k >= a.K) continue;
                const size_t e = ((size_t)b * a.K + k) * plane + pix;
                const float2 z = acc[k8 + q];
                if (a.spectrum) {
                    if (a.stream_out) __stcs(&a.spectrum[e], z);
                    else a.spectrum[e] = z;
                }
                if (a.l2_grad) {
                    const float dr = z.x - t[q].x, di = z.y - t[q].y;
                    l2acc = fmaf(dr, dr, fmaf(di, di, l2acc));
                    const float2 gz = make_float2(2.f * dr * a.l2_inv, 2.f * di * a.l2_inv);
                    a.l2_grad[e] = gz;
                    stot = fmaf(gz.x, z.x, fmaf(gz.y, z.y, stot));
                }
            }
        }
        if (a.l2_grad && a.s_tot) a.s_tot[((size_t)b * gridDim.x + strip) * plane + pix] = stot;
        if (strip == 0) {
            if (a.final_logT) a.final_logT[(size_t)b * plane + pix] = logT;
            if (a.n_contrib) a.n_contrib[(size_t)b * plane + pix] = last;
            if (a.n_used) a.n_used[(size_t)b * plane + pix] = used;
        }
    }
    if (a.l2_grad) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l2acc += __shfl_xor_sync(0xffffffffu, l2acc, o);
        if (lane == 0) s_part[warp] = l2acc;
    }
    if (a.tile_walk && strip == 0) {
        uint32_t wmax = inside ? last : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        if (lane == 0 && wmax) atomicMax(s_walk, wmax);
    }
    __syncthreads();
    if (tid == 0) {
        if (a.l2_grad) {
            float t = 0.f;
            for (int w2 = 0; w2 < kThreads / 32; ++w2) t += s_part[w2];
            atomicAdd(a.l2_loss, t * a.l2_inv);
        }
        if (a.tile_walk && strip == 0) a.tile_walk[(size_t)b * a.T + tile] = min(*s_walk, len);
    }
}

// The backward.  Work item: one (transmitter, tile, strip of S subcarriers) walk over the list
// positions [0, walk), back to front from each pixel's final state (no item list: one CTA per
// walk), or a scheduled chunk of it (a.items: item r on CTA r): a back chunk [m, walk) back to
// front, or a front chunk [0, m) front to back from T = 1 with the suffix sum taken as
// s_tot - prefix (s_tot = Re sum_k conj(dL/dz_k) z_k over the strip, given or formed here from
// the spectrum).  A warp visits only the entries whose footprint box reaches its pixels (the set
// bits of its entry mask, in walk order); per visited entry its pixels' nine gradient components
// are reduced over the warp in one reduce-scatter and added to the gradients by the warp (one
// atomic per component), so a batch needs one block barrier.
template <int S>
__global__ void __launch_bounds__(kThreads, 2) k_render_bwd(RenderArgs a) {
    using L = F32BwdSmem<S>;
    GSPARC_DYNAMIC_SMEM(sm);
    StageRec* s_rec = reinterpret_cast<StageRec*>(sm + L::kRec);
    float4(*s_tab)[kBatch][L::kRow] = reinterpret_cast<float4(*)[kBatch][L::kRow]>(sm + L::kTab);
    uint32_t* s_gid = reinterpret_cast<uint32_t*>(sm + L::kGid);
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(sm + L::kBar);
    uint32_t* s_maxlast = reinterpret_cast<uint32_t*>(sm + L::kMisc + 32);
    uint32_t* s_err = s_maxlast + 1;
    grid_dep_wait();     // the schedule's items, the forward's outputs and the upstream gradient

    int strip, tile, b;
    bool front = false;
    uint32_t lo = 0, end = 0;
    if (a.items) {
        const uint32_t r = blockIdx.x;
        if (r >= *a.n_items) return;   // the whole block, before any barrier
        const uint4 it = a.items[r];
        b = (int)(it.x / (uint32_t)a.T);
        tile = (int)(it.x - (uint32_t)b * (uint32_t)a.T);
        strip = (int)(it.y & 0x7fffffffu);
        front = (it.y >> 31) != 0u;
        lo = it.z;
        end = it.w;
    } else {
        strip = blockIdx.x;
        tile = blockIdx.y;
        b = blockIdx.z;
    }
    const int k0 = strip * S;
    const int strips = (a.K + S - 1) / S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx0 = (tile % a.TW) * kTile, ty0 = (tile / a.TW) * kTile;
    const int x = tx0 + (tid & 15);
    const int y = ty0 + (tid >> 4);
    const bool inside = x < a.W && y < a.H;
    const float ux = (float)x + 0.5f, uy = (float)y + 0.5f;
    const float wcx = (float)tx0 + 8.0f, wcy = (float)(ty0 + 2 * warp) + 1.0f;
    const uint2 range = a.ranges[tile];
    const size_t plane = (size_t)a.H * a.W;
    const size_t pix = (size_t)y * a.W + x;

    float2 g[S];
#pragma unroll
    for (int kk = 0; kk < S; ++kk) {
        const int k = k0 + kk;
        g[kk] = (inside && k < a.K) ? a.d_spectrum[((size_t)b * a.K + k) * plane + pix] : make_float2(0.f, 0.f);
    }
    float s_tot = 0.f;
    if (front && inside) {
        if (a.s_tot) {
            s_tot = a.s_tot[((size_t)b * strips + strip) * plane + pix];
        } else {
#pragma unroll
            for (int kk = 0; kk < S; ++kk) {
                const int k = k0 + kk;
                if (k < a.K) {
                    const float2 z = a.spectrum[((size_t)b * a.K + k) * plane + pix];
                    s_tot = fmaf(g[kk].x, z.x, fmaf(g[kk].y, z.y, s_tot));
                }
            }
        }
    }
    float logT = (inside && !front) ? a.final_logT[(size_t)b * plane + pix] : 0.f;
    const uint32_t last = inside ? a.n_contrib[(size_t)b * plane + pix] : 0u;
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, last);   // the warp's walk
    if (tid == 0) {
        stage_bar_init(&s_bar[0]);
        stage_bar_init(&s_bar[1]);
        stage_init_fence();
        *s_maxlast = 0u;
        *s_err = 0u;
    }
    __syncthreads();
    if (!a.items) {
        if (last) atomicMax(s_maxlast, last);
        __syncthreads();
        end = min(*s_maxlast, range.y - range.x);   // the walk: the largest n_contrib
    }
    const int nbatch = (int)((end - lo + kBatch - 1) / kBatch);
    auto load_id = [&](int i) -> uint32_t {
        if (tid >= kBatch || i >= nbatch) return 0xffffffffu;
        uint32_t b_lo;
        int nb;
        batch_span(front, lo, end, i, b_lo, nb);
        return tid < nb ? a.ids[range.x + b_lo + tid] : 0xffffffffu;
    };
    uint32_t pf_id = load_id(0);
    if (nbatch > 0) {
        uint32_t b_lo;
        int nb;
        batch_span(front, lo, end, 0, b_lo, nb);
        stage_issue(a, b, nb, pf_id, s_rec, s_gid, &s_bar[0]);
    }
    pf_id = load_id(1);
    // dpsi/dL = -(2 pi / c) (f_strip0 + kk df)
    const float c_f0 = (float)(a.two_pi_over_c * (a.f0 + (double)k0 * a.df));
    const float c_df = (float)(a.two_pi_over_c * a.df);
    // Gradient slot of component c: attr slots 0 a, 1 phi0, 2 sigma, 3 L for c >= 5; projection
    // slots p_x, p_y, c_xx, c_xy, c_yy for c < 5.  A one-entry reduce-scatter leaves component
    // lane >> 1 in the even lanes below 18; a two-entry one leaves component slot18 % 9 of the
    // first (slot18 < 9) or the second entry in the lanes where slot18 >= 0.
    const int slot18 = rs18_slot(lane);
    const bool holder = (lane & 1) == 0 && (lane >> 1) < 9;
    auto add_grad = [&](int c, uint32_t gid, float v) {
        float* dst = c >= 5 ? reinterpret_cast<float*>(&a.d_attr[(size_t)b * a.N + gid]) +
                                  (c == 5 ? 2 : (c == 6 ? 0 : (c == 7 ? 1 : 3)))
                            : a.d_proj + (size_t)gid * 8 + (c < 2 ? c : c + 2);
        atomicAdd(dst, v);
    };
    // Back to front: acc = the sum over later composited entries of w a Re(conj(g) e^{j psi})
    // (the suffix); front to back: the same sum over the entries up to this one (suffix =
    // s_tot - acc).  The two directions differ in a few selects, not in code paths.
    float acc = 0.f;
    for (int i = 0; i < nbatch; ++i) {
        const int buf = i & 1;
        uint32_t b_lo;
        int nb;
        batch_span(front, lo, end, i, b_lo, nb);
        if (!stage_wait(&s_bar[buf], (uint32_t)(i >> 1) & 1u, kStagePolls)) {
            *s_err = 1u;
            stage_wait(&s_bar[buf], (uint32_t)(i >> 1) & 1u, kStagePolls);   // copies still in flight
        }
        stage_phasors_bwd<S>(a, s_rec + buf * kBatch, nb, k0, s_tab[buf]);
        // phasors of batch i in place; every warp has finished batch i - 1, whose buffers the
        // copies of batch i + 1 now take over
        __syncthreads();
        if (*s_err) break;
        if (i + 1 < nbatch) {
            uint32_t n_lo;
            int nn;
            batch_span(front, lo, end, i + 1, n_lo, nn);
            if (tid < kBatch) stage_proxy_fence();
            stage_issue(a, b, nn, pf_id, s_rec + (buf ^ 1) * kBatch, s_gid + (buf ^ 1) * kBatch, &s_bar[buf ^ 1]);
            pf_id = load_id(i + 2);
        }
        const StageRec* rec = s_rec + buf * kBatch;
        const uint32_t* gids = s_gid + buf * kBatch;
        uint64_t bits = warp_entry_mask_rec(rec, nb, wcx, wcy, a.W);
        // positions at or past every pixel's n_contrib are live at none of the warp's pixels
        if (b_lo >= wlast) bits = 0ull;
        else if (wlast - b_lo < (uint32_t)kBatch) bits &= (1ull << (wlast - b_lo)) - 1ull;
        // the gradient components of a visited entry wait in pend until a second one arrives, and
        // the two are reduced over the warp together
        float pend[9];
        int pend_j = -1;
        while (bits) {   // warp-uniform
            const int j = front ? __ffsll((long long)bits) - 1 : 63 - __clzll((long long)bits);
            bits &= ~(1ull << j);
            const StageRec& r = rec[j];
            const float4 gg = make_float4(r.p0.x, r.p0.y, r.p1.x, r.p1.y);
            const float2 g2 = make_float2(r.p1.z, r.at.z);
            float dx = 0.f, dy = 0.f, G = 0.f, alpha = 0.f;
            bool clamped = false;
            const bool live = b_lo + (uint32_t)j < last && eval_alpha(ux, uy, a.W, gg, g2, dx, dy, G, alpha, clamped);
            if (!__any_sync(0xffffffffu, live)) continue;
            // Per subcarrier, from the last down: one 16-byte broadcast read and three paired
            // operations.  re2 sums Re(conj(g) t) as two chains (g.x t.x and g.y t.y); suf2 sums
            // Im(conj(g) t) (g.x t.y and -g.y t.x) over the subcarriers from kk up, and tot2 adds
            // those suffix sums for kk >= 1, which is sum_kk kk Im_kk.
            float2 re2 = make_float2(0.f, 0.f), suf2 = make_float2(0.f, 0.f), tot2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = S - 1; kk >= 0; --kk) {
                const float4 t = s_tab[buf][j][kk];
                re2 = fma2(g[kk], make_float2(t.x, t.y), re2);
                suf2 = fma2(g[kk], make_float2(t.z, t.w), suf2);
                if (kk > 0) tot2 = add2(tot2, suf2);
            }
            const float reG = re2.x + re2.y, imG = suf2.x + suf2.y, imF = tot2.x + tot2.y;
            float gr[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) gr[c] = 0.f;
            if (live) {
                const float nl = lg2(__fsub_rn(1.0f, alpha));
                const float amp = r.at.x;
                const float reGa = amp * reG;
                // front: T before the entry is the running one, then T *= 1 - alpha; back: T
                // before the entry is recovered from the one after it
                const float logT_next = front ? __fadd_rn(logT, nl) : __fsub_rn(logT, nl);
                const float T = ex2(front ? logT : logT_next);
                const float w = T * alpha;
                const float acc_next = fmaf(w, reGa, acc);
                const float suffix = front ? s_tot - acc_next : acc;
                // 1 - alpha >= 0.01: the approximate quotient (2 ulp) is ample for a gradient term
                const float dalpha = T * reGa - __fdividef(suffix, 1.0f - alpha);
                acc = acc_next;
                logT = logT_next;
                gr[6] = w * reG;                                  // d a
                gr[7] = -w * amp * imG;                           // d phi0
                gr[8] = w * amp * (c_f0 * imG + c_df * imF);      // d L
                if (!clamped) {
                    const float sig = g2.y;
                    gr[5] = dalpha * G;                           // d sigma
                    const float dq = -0.5f * dalpha * sig * G;
                    gr[0] = dq * (-2.0f * (gg.z * dx + gg.w * dy));   // d p_x
                    gr[1] = dq * (-2.0f * (gg.w * dx + g2.x * dy));   // d p_y
                    gr[2] = dq * dx * dx;                             // d c_xx
                    gr[3] = dq * 2.0f * dx * dy;                      // d c_xy
                    gr[4] = dq * dy * dy;                             // d c_yy
                }
            }
            if (pend_j < 0) {
#pragma unroll
                for (int c = 0; c < 9; ++c) pend[c] = gr[c];
                pend_j = j;
                continue;
            }
            // reduce-scatter of both entries' 18 components over the warp; the lane holding one
            // adds it to the gradient
            float v[18];
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                v[c] = pend[c];
                v[9 + c] = gr[c];
            }
            const float tot = warp_reduce_scatter18(v, lane);
            if (slot18 >= 0 && tot != 0.f) add_grad(slot18 % 9, slot18 < 9 ? gids[pend_j] : gids[j], tot);
            pend_j = -1;
        }
        if (pend_j >= 0) {
            const float tot = warp_reduce_scatter9(pend, lane);
            if (holder && tot != 0.f) add_grad(lane >> 1, gids[pend_j], tot);
        }
    }
    if (*s_err && tid == 0) set_status(a.status, GSPARC_ERR_TIMEOUT);
}

// Subcarriers per thread: the smallest power of two covering K, at most 32.
// (Splitting K into more, narrower strips to raise the CTA count was measured
// slower: every strip re-evaluates alpha, T and the gradient reduction.)
int pick_strip(int K, int64_t) {
    int S = 1;
    while (S < K && S < 32) S <<= 1;
    return S;
}

bool fill_args(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
               const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
               const float* attr, RenderArgs& a) {
    a.H = view->H;
    a.W = view->W;
    a.TW = tiles_x(*view);
    a.T = a.TW * tiles_y(*view);
    a.K = band->K;
    a.N = N;
    a.B = B;
    a.proj = reinterpret_cast<const float4*>(proj);
    a.ranges = reinterpret_cast<const uint2*>(tile_ranges);
    a.ids = sorted_ids;
    a.attr = reinterpret_cast<const float4*>(attr);
    const double f0 = band->f_c - (double)(band->K / 2) * band->df;
    const double lam0 = f0 / kCLight;
    a.lam0_hi = (float)lam0;
    a.lam0_lo = (float)(lam0 - (double)a.lam0_hi);
    a.dlam = (float)(band->df / kCLight);
    a.two_pi_over_c = 2.0 * 3.14159265358979323846 / kCLight;
    a.f0 = f0;
    a.df = band->df;
    // an output above a quarter of the 129 MB L2 streams past it
    a.stream_out = (double)B * band->K * view->H * view->W * 8.0 > 32.0 * 1024 * 1024;
    return true;
}

}  // namespace
}  // namespace gsparc
