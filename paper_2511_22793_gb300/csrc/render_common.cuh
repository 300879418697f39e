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
// memory together with their unit phasors e^{j psi_ik} for the strip, so the
// per-(pixel, Gaussian, subcarrier) work is two FFMAs (forward) or six
// (backward) against broadcast shared-memory reads.  Transmittance is carried
// as log2 T in FP32; a thread stops before T would fall below 1e-4 and the
// CTA stops fetching once every thread has stopped.
//
// This header holds what the FP32 kernels and the tensor-core kernels share (arguments, alpha,
// unit phasors, batch staging) and the FP32 kernels themselves, as device code with no runtime
// API, so that the same source also builds for the host under the test suite's shim (which
// defines GSPARC_HOST_SHIM and gets exp2f / log2f for the SFU's ex2 / lg2).  Launches and entry
// points are in render.cu.

#pragma once

#include <math.h>
#include <stdint.h>

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
#else
// the test suite's host shim: the library's exact counterparts of the SFU approximations
inline float ex2(float x) { return exp2f(x); }
inline float lg2(float x) { return log2f(x); }
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

// Stage batch entries [list_pos, list_pos + nb) of the tile list, and the
// unit phasors of the strip's subcarriers.
template <int S>
__device__ __forceinline__ void stage_batch(const RenderArgs& a, int b, uint32_t list_pos, int nb,
                                            int k0, float4* s_geo, float2* s_geo2, float2* s_ext,
                                            float* s_amp, float2 (*s_tab)[S], uint32_t* s_gid) {
    const int tid = threadIdx.x;
    __shared__ float s_L[kBatch], s_phi[kBatch];
    if (tid < nb) {
        uint32_t gid = a.ids[list_pos + tid];
        if (gid < (uint32_t)a.N) {
            const float4 p0 = a.proj[2 * gid];
            const float4 p1 = a.proj[2 * gid + 1];
            const float4 at = a.attr[(size_t)b * a.N + gid];
            s_geo[tid] = make_float4(p0.x, p0.y, p1.x, p1.y);
            s_geo2[tid] = make_float2(p1.z, at.z);
            s_ext[tid] = make_float2(p0.z, p0.w);
            s_amp[tid] = at.x;
            s_phi[tid] = at.y;
            s_L[tid] = at.w;
        } else {
            // an id outside the scene (inconsistent inputs): a NaN conic makes
            // every pixel skip it, it receives no gradient, and the status word says so
            set_status(a.status, GSPARC_ERR_INPUT);
            s_geo[tid] = make_float4(0.f, 0.f, __int_as_float(0x7fc00000), 0.f);
            s_geo2[tid] = make_float2(0.f, 0.f);
            s_ext[tid] = make_float2(-1.f, -1.f);
            s_amp[tid] = 0.f;
            s_phi[tid] = 0.f;
            s_L[tid] = 0.f;
            gid = 0;
        }
        s_gid[tid] = gid;
    }
    __syncthreads();
    for (int e = tid; e < nb * S; e += kThreads) {
        const int j = e / S, kk = e - j * S;
        const int k = k0 + kk;
        float2 ph = make_float2(0.f, 0.f);
        if (k < a.K) ph = unit_phasor(a, s_L[j], s_phi[j], k);
        s_tab[j][kk] = ph;
    }
    __syncthreads();
}

// Bit j set when staged entry j's footprint box reaches the warp's 16x2 block of
// pixel centres (centre (wcx, wcy), half sizes 7.5 x 0.5).  The box is the
// bounding box of q <= q_max, so a cleared bit means q > q_max at every pixel
// of the warp; the 0.01 px margin covers rounding at the box edge.
__device__ __forceinline__ uint64_t warp_entry_mask(const float4* s_geo, const float2* s_ext, int nb,
                                                    float wcx, float wcy, int W) {
    const int lane = threadIdx.x & 31;
    const float hw = 0.5f * (float)W;
    bool h0 = false, h1 = false;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int j = lane + 32 * half;
        bool hit = false;
        if (j < nb) {
            const float2 e = s_ext[j];
            float dx = wcx - s_geo[j].x;
            if (dx >= hw) dx -= (float)W;
            else if (dx < -hw) dx += (float)W;
            const float dy = wcy - s_geo[j].y;
            hit = e.x >= 0.f && fabsf(dx) <= e.x + 7.51f && fabsf(dy) <= e.y + 0.51f;
        }
        if (half == 0) h0 = hit;
        else h1 = hit;
    }
    const uint32_t lo = __ballot_sync(0xffffffffu, h0);
    const uint32_t hi = __ballot_sync(0xffffffffu, h1);
    return ((uint64_t)hi << 32) | lo;
}

template <int S>
__global__ void __launch_bounds__(kThreads, 2) k_render_fwd(RenderArgs a) {
    __shared__ float4 s_geo[kBatch];
    __shared__ float2 s_geo2[kBatch];
    __shared__ float2 s_ext[kBatch];
    __shared__ float s_amp[kBatch];
    __shared__ uint32_t s_gid[kBatch];
    __shared__ __align__(16) float2 s_tab[kBatch][S];

    const int strip = blockIdx.x, tile = blockIdx.y, b = blockIdx.z;
    const int k0 = strip * S;
    const int tid = threadIdx.x;
    const int tx0 = (tile % a.TW) * kTile, ty0 = (tile / a.TW) * kTile;
    const int x = tx0 + (tid & 15);
    const int y = ty0 + (tid >> 4);
    const bool inside = x < a.W && y < a.H;
    const float ux = (float)x + 0.5f, uy = (float)y + 0.5f;
    const float wcx = (float)tx0 + 8.0f, wcy = (float)(ty0 + 2 * (tid >> 5)) + 1.0f;
    const uint2 range = a.ranges[tile];

    float2 acc[S];
#pragma unroll
    for (int kk = 0; kk < S; ++kk) acc[kk] = make_float2(0.f, 0.f);
    float logT = 0.f;
    uint32_t last = 0, used = 0;
    bool done = !inside;

    for (uint32_t bs = range.x; bs < range.y; bs += kBatch) {
        if (__syncthreads_or(!done) == 0) break;
        const int nb = (int)min((uint32_t)kBatch, range.y - bs);
        stage_batch<S>(a, b, bs, nb, k0, s_geo, s_geo2, s_ext, s_amp, s_tab, s_gid);
        uint64_t mask = warp_entry_mask(s_geo, s_ext, nb, wcx, wcy, a.W);
        if (!done) {
            while (mask) {
                const int j = __ffsll((long long)mask) - 1;
                mask &= mask - 1;
                float dx, dy, G, alpha;
                bool clamped;
                if (!eval_alpha(ux, uy, a.W, s_geo[j], s_geo2[j], dx, dy, G, alpha, clamped)) continue;
                const float nl = lg2(__fsub_rn(1.0f, alpha));
                if (__fadd_rn(logT, nl) < kLog2TMin) {
                    done = true;
                    break;
                }
                const float wa = ex2(logT) * alpha * s_amp[j];
#pragma unroll
                for (int kk = 0; kk < S; ++kk) {
                    const float2 t = s_tab[j][kk];
                    acc[kk].x = fmaf(wa, t.x, acc[kk].x);
                    acc[kk].y = fmaf(wa, t.y, acc[kk].y);
                }
                logT = __fadd_rn(logT, nl);
                last = bs - range.x + (uint32_t)j + 1u;
                ++used;
            }
        }
    }
    if (!inside) return;
    const size_t plane = (size_t)a.H * a.W;
    const size_t pix = (size_t)y * a.W + x;
#pragma unroll
    for (int kk = 0; kk < S; ++kk) {
        const int k = k0 + kk;
        if (k < a.K) a.spectrum[((size_t)b * a.K + k) * plane + pix] = acc[kk];
    }
    if (strip == 0) {
        if (a.final_logT) a.final_logT[(size_t)b * plane + pix] = logT;
        if (a.n_contrib) a.n_contrib[(size_t)b * plane + pix] = last;
        if (a.n_used) a.n_used[(size_t)b * plane + pix] = used;
    }
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

template <int S>
__global__ void __launch_bounds__(kThreads, 2) k_render_bwd(RenderArgs a) {
    __shared__ float4 s_geo[kBatch];
    __shared__ float2 s_geo2[kBatch];
    __shared__ float2 s_ext[kBatch];
    __shared__ float s_amp[kBatch];
    __shared__ uint32_t s_gid[kBatch];
    __shared__ __align__(16) float2 s_tab[kBatch][S];
    __shared__ float s_red[kThreads / 32][kBatch][9];
    __shared__ uint64_t s_wmask[kThreads / 32];
    __shared__ uint32_t s_maxlast;

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
    const size_t plane = (size_t)a.H * a.W;
    const size_t pix = (size_t)y * a.W + x;

    float2 g[S];
#pragma unroll
    for (int kk = 0; kk < S; ++kk) {
        const int k = k0 + kk;
        g[kk] = (inside && k < a.K) ? a.d_spectrum[((size_t)b * a.K + k) * plane + pix]
                                    : make_float2(0.f, 0.f);
    }
    float logT = inside ? a.final_logT[(size_t)b * plane + pix] : 0.f;
    const uint32_t last = inside ? a.n_contrib[(size_t)b * plane + pix] : 0u;
    if (tid == 0) s_maxlast = 0;
    __syncthreads();
    if (last) atomicMax(&s_maxlast, last);
    __syncthreads();
    const uint32_t maxlast = min(s_maxlast, range.y - range.x);
    // dpsi/dL = -(2 pi / c) (f_strip0 + kk df)
    const float c_f0 = (float)(a.two_pi_over_c * (a.f0 + (double)k0 * a.df));
    const float c_df = (float)(a.two_pi_over_c * a.df);
    float suffix = 0.f;   // sum over later composited m of w_m a_m Re(conj(g) e^{j psi_m})

    for (uint32_t bend = maxlast; bend > 0;) {
        const uint32_t bstart = bend > (uint32_t)kBatch ? bend - kBatch : 0u;
        const int nb = (int)(bend - bstart);
        __syncthreads();
        stage_batch<S>(a, b, range.x + bstart, nb, k0, s_geo, s_geo2, s_ext, s_amp, s_tab, s_gid);
        uint64_t mask = warp_entry_mask(s_geo, s_ext, nb, wcx, wcy, a.W);
        if (lane == 0) s_wmask[warp] = mask;
        while (mask) {
            const int j = 63 - __clzll((long long)mask);
            mask ^= 1ull << j;
            float gr[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) gr[c] = 0.f;
            bool contrib = false;
            const uint32_t pos = bstart + (uint32_t)j;
            if (pos < last) {
                const float4 gg = s_geo[j];
                const float2 g2 = s_geo2[j];
                float dx, dy, G, alpha;
                bool clamped;
                if (eval_alpha(ux, uy, a.W, gg, g2, dx, dy, G, alpha, clamped)) {
                    contrib = true;
                    const float nl = lg2(__fsub_rn(1.0f, alpha));
                    const float logT_before = __fsub_rn(logT, nl);
                    const float T = ex2(logT_before);
                    const float w = T * alpha;
                    float reG = 0.f, imG = 0.f, imF = 0.f;
#pragma unroll
                    for (int kk = 0; kk < S; ++kk) {
                        const float2 t = s_tab[j][kk];
                        reG = fmaf(g[kk].x, t.x, fmaf(g[kk].y, t.y, reG));
                        const float pi_ = fmaf(g[kk].x, t.y, -g[kk].y * t.x);
                        imG += pi_;
                        imF = fmaf((float)kk, pi_, imF);
                    }
                    const float amp = s_amp[j];
                    const float reGa = amp * reG;
                    const float dalpha = T * reGa - suffix / (1.0f - alpha);
                    suffix = fmaf(w, reGa, suffix);
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
                    logT = logT_before;
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                // reduce-scatter of the 9 components over the warp: lane l ends with the
                // warp total of component l >> 1
                const float tot = warp_reduce_scatter9(gr, lane);
                if ((lane & 1) == 0 && (lane >> 1) < 9) s_red[warp][j][lane >> 1] = tot;
            } else if (lane < 9) {
                s_red[warp][j][lane] = 0.f;
            }
        }
        __syncthreads();
        // one atomic per (Gaussian, component) for the whole CTA
        for (int e = tid; e < nb * 9; e += kThreads) {
            const int j = e / 9, c = e - j * 9;
            float v = 0.f;
#pragma unroll
            for (int w2 = 0; w2 < kThreads / 32; ++w2)
                if ((s_wmask[w2] >> j) & 1ull) v += s_red[w2][j][c];
            if (v != 0.f) {
                const uint32_t gid = s_gid[j];
                if (c >= 5) {
                    float* dst = reinterpret_cast<float*>(&a.d_attr[(size_t)b * a.N + gid]);
                    // attr slots: 0 a, 1 phi0, 2 sigma, 3 L
                    const int slot = c == 5 ? 2 : (c == 6 ? 0 : (c == 7 ? 1 : 3));
                    atomicAdd(dst + slot, v);
                } else {
                    const int slot = c < 2 ? c : c + 2;   // p_x, p_y, -, -, c_xx, c_xy, c_yy
                    atomicAdd(a.d_proj + (size_t)gid * 8 + slot, v);
                }
            }
        }
        bend = bstart;
    }
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
    return true;
}

}  // namespace
}  // namespace gsparc
