// Per-Gaussian projection onto the equirectangular hemisphere and its gradient.
//
// Sec. 4.2 ("Directional Projection and Splatting"): x' = V (mu - x_rx),
// p_x = (atan2(x', z')/pi + 1) W/2, p_y = 2 asin(y'/|x'|) H/pi, and
// Sigma' = J V Sigma V^T J^T with J the Jacobian of that map; Sec. 3.2 for
// Sigma = R S S^T R^T.  Algorithm 1 CullGaussians / TransformToView /
// ProjectGaussians.
//
// Device code only (the entry points are in project.cu), so that the same source also builds
// for the host under the test suite's shim.  One thread per Gaussian; the pass is HBM-bound
// (44 B read, 32 B written per Gaussian), the record is written as two aligned float4 stores.

#pragma once

#include <math.h>

#include "device_common.cuh"

namespace gsparc {
namespace {

struct Geo {
    float x, y, z, r2, r, rho_raw, rho_cap;
    float cx, cz;     // azimuth direction (x'/rho, z'/rho); (0, 1) at the zenith
    bool clamped;
    float sx, sy;
    float J00, J02, J10, J11, J12;
    float M[2][3];    // J V
    float R[3][3];    // rotation of the normalised quaternion
    float qn[4], qnorm;
    float A[2][3];    // M R
    float s2[3];      // exp(2 log_scale)
    float sxx, sxy, syy, det, inv;
};

__device__ __forceinline__ void rot_from_quat(const float4 q4, Geo& g) {
    float qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
    float n = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    g.qnorm = n;
    float in = 1.0f / n;
    float w = qw * in, x = qx * in, y = qy * in, z = qz * in;
    g.qn[0] = w; g.qn[1] = x; g.qn[2] = y; g.qn[3] = z;
    g.R[0][0] = 1.f - 2.f * (y * y + z * z);
    g.R[0][1] = 2.f * (x * y - w * z);
    g.R[0][2] = 2.f * (x * z + w * y);
    g.R[1][0] = 2.f * (x * y + w * z);
    g.R[1][1] = 1.f - 2.f * (x * x + z * z);
    g.R[1][2] = 2.f * (y * z - w * x);
    g.R[2][0] = 2.f * (x * z - w * y);
    g.R[2][1] = 2.f * (y * z + w * x);
    g.R[2][2] = 1.f - 2.f * (x * x + y * y);
}

// Everything up to Sigma' for Gaussian i; returns false when culled.
__device__ __forceinline__ bool geometry(const ViewDev& v, int i, const float* __restrict__ means,
                                         const float* __restrict__ ls,
                                         const float4* __restrict__ quats, Geo& g) {
    const float mx = means[3 * i + 0] - v.rx0;
    const float my = means[3 * i + 1] - v.rx1;
    const float mz = means[3 * i + 2] - v.rx2;
    g.x = v.V[0] * mx + v.V[1] * my + v.V[2] * mz;
    g.y = v.V[3] * mx + v.V[4] * my + v.V[5] * mz;
    g.z = v.V[6] * mx + v.V[7] * my + v.V[8] * mz;
    g.r2 = g.x * g.x + g.y * g.y + g.z * g.z;
    g.r = sqrtf(g.r2);
    if (!(g.r >= v.near_dist)) return false;
    g.rho_raw = sqrtf(g.x * g.x + g.z * g.z);
    const float floor_ = kRhoFloor * g.r;
    g.clamped = g.rho_raw < floor_;
    g.rho_cap = g.clamped ? floor_ : g.rho_raw;
    if (g.rho_raw > 0.f) {
        const float ir = 1.0f / g.rho_raw;
        g.cx = g.x * ir;
        g.cz = g.z * ir;
    } else {
        g.cx = 0.f;
        g.cz = 1.f;
    }
    g.sx = (float)v.W / (2.0f * kPi);
    g.sy = 2.0f * (float)v.H / kPi;
    // azimuth row: direction (cz, 0, -cx) with 1/rho capped; elevation row exact
    const float icap = 1.0f / g.rho_cap;
    const float ir2 = 1.0f / g.r2;
    g.J00 = g.sx * g.cz * icap;
    g.J02 = -g.sx * g.cx * icap;
    g.J10 = -g.sy * g.y * g.cx * ir2;
    g.J11 = g.sy * g.rho_raw * ir2;
    g.J12 = -g.sy * g.y * g.cz * ir2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        g.M[0][c] = g.J00 * v.V[0 * 3 + c] + g.J02 * v.V[2 * 3 + c];
        g.M[1][c] = g.J10 * v.V[0 * 3 + c] + g.J11 * v.V[1 * 3 + c] + g.J12 * v.V[2 * 3 + c];
    }
    rot_from_quat(quats[i], g);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            g.A[r][c] = g.M[r][0] * g.R[0][c] + g.M[r][1] * g.R[1][c] + g.M[r][2] * g.R[2][c];
    g.sxx = kDilation;
    g.sxy = 0.f;
    g.syy = kDilation;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        g.s2[c] = expf(2.0f * ls[3 * i + c]);
        g.sxx += g.A[0][c] * g.A[0][c] * g.s2[c];
        g.sxy += g.A[0][c] * g.A[1][c] * g.s2[c];
        g.syy += g.A[1][c] * g.A[1][c] * g.s2[c];
    }
    g.det = g.sxx * g.syy - g.sxy * g.sxy;
    g.inv = 1.0f / g.det;
    return true;
}

// A kept Gaussian whose covariance is not a finite positive-definite matrix (a non-finite mean
// or log-scale, a zero quaternion) has no footprint: the projection culls it and reports
// GSPARC_ERR_INPUT, and the backward passes it no gradient.
__device__ __forceinline__ bool record_ok(const Geo& g) {
    return g.qnorm > 0.f && isfinite(g.qnorm) && isfinite(g.sxx) && isfinite(g.sxy) && isfinite(g.syy) &&
           g.det > 0.f && isfinite(g.inv);
}

__global__ void __launch_bounds__(256) k_project(ViewDev v, int N, const float* __restrict__ means,
                                                 const float* __restrict__ ls,
                                                 const float4* __restrict__ quats,
                                                 float4* __restrict__ proj, int32_t* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    Geo g;
    const bool kept = geometry(v, i, means, ls, quats, g);
    if (!kept || !record_ok(g)) {
        // culled: behind the near distance, or (reported) a non-finite or degenerate input
        if (kept || !isfinite(g.r)) set_status(status, GSPARC_ERR_INPUT);
        proj[2 * i + 0] = make_float4(0.f, 0.f, -1.f, -1.f);
        proj[2 * i + 1] = make_float4(0.f, 0.f, 0.f, isfinite(g.r) ? g.r : 0.f);
        return;
    }
    const float px = (atan2f(g.x, g.z) / kPi + 1.0f) * (0.5f * (float)v.W);
    // asin(y'/r) evaluated as atan2(y', rho): the same angle, well conditioned
    // next to the zenith where asin's argument approaches 1
    const float py = 2.0f * atan2f(g.y, g.rho_raw) * ((float)v.H / kPi);
    const float ex = sqrtf(kQMax * g.sxx);
    const float ey = sqrtf(kQMax * g.syy);
    proj[2 * i + 0] = make_float4(px, py, ex, ey);
    proj[2 * i + 1] = make_float4(g.syy * g.inv, -g.sxy * g.inv, g.sxx * g.inv, g.r);
}

__global__ void __launch_bounds__(256) k_project_bwd(ViewDev v, int N, const float* __restrict__ means,
                                                     const float* __restrict__ ls,
                                                     const float4* __restrict__ quats,
                                                     const float4* __restrict__ dproj,
                                                     float* __restrict__ d_means,
                                                     float* __restrict__ d_ls,
                                                     float* __restrict__ d_quats) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    Geo g;
    if (!geometry(v, i, means, ls, quats, g) || !record_ok(g)) return;
    const float4 d0 = dproj[2 * i + 0];
    const float4 d1 = dproj[2 * i + 1];
    const float dpx = d0.x, dpy = d0.y, dcxx = d1.x, dcxy = d1.y, dcyy = d1.z;

    // conic = (Sigma')^-1 -> Sigma' = [[A, B], [B, D]]
    const float A = g.sxx, B = g.sxy, D = g.syy;
    const float inv2 = g.inv * g.inv;
    const float dA = (-dcxx * D * D + dcxy * B * D - dcyy * B * B) * inv2;
    const float dD = (-dcxx * B * B + dcxy * A * B - dcyy * A * A) * inv2;
    const float dB = (2.f * B * D * dcxx - (A * D + B * B) * dcxy + 2.f * A * B * dcyy) * inv2;

    // Sigma' = Am diag(s2) Am^T + 0.3 I, Am = M R
    float dAm[2][3];
    float dls[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a0 = g.A[0][c], a1 = g.A[1][c], s2 = g.s2[c];
        dAm[0][c] = (2.f * dA * a0 + dB * a1) * s2;
        dAm[1][c] = (2.f * dD * a1 + dB * a0) * s2;
        const float ds2 = dA * a0 * a0 + dB * a0 * a1 + dD * a1 * a1;
        dls[c] = ds2 * 2.f * s2;
    }
    // Am = M R: dM = dAm R^T, dR = M^T dAm
    float dM[2][3], dR[3][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dM[r][k] = dAm[r][0] * g.R[k][0] + dAm[r][1] * g.R[k][1] + dAm[r][2] * g.R[k][2];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) dR[k][c] = g.M[0][k] * dAm[0][c] + g.M[1][k] * dAm[1][c];

    // R(q_hat) -> q_hat -> q
    const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
    float dqh[4];
    dqh[0] = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] +
                    x * dR[2][1]);
    dqh[1] = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] -
                    w * dR[1][2] + z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
    dqh[2] = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] +
                    z * dR[1][2] - w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
    dqh[3] = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] -
                    2.f * z * dR[1][1] + y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float dot = dqh[0] * w + dqh[1] * x + dqh[2] * y + dqh[3] * z;
    const float iq = 1.0f / g.qnorm;
    d_quats[4 * i + 0] += (dqh[0] - w * dot) * iq;
    d_quats[4 * i + 1] += (dqh[1] - x * dot) * iq;
    d_quats[4 * i + 2] += (dqh[2] - y * dot) * iq;
    d_quats[4 * i + 3] += (dqh[3] - z * dot) * iq;
    d_ls[3 * i + 0] += dls[0];
    d_ls[3 * i + 1] += dls[1];
    d_ls[3 * i + 2] += dls[2];

    // M = J V: dJ = dM V^T (J01 = 0)
    float dJ[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dJ[r][j] = dM[r][0] * v.V[j * 3 + 0] + dM[r][1] * v.V[j * 3 + 1] + dM[r][2] * v.V[j * 3 + 2];

    // map position gradient: the exact derivatives of atan2 and asin
    // (p_x: sx (z', 0, -x')/rho^2; p_y: the elevation row of J)
    const float sx = g.sx, sy = g.sy, gx = g.x, gy = g.y, gz = g.z;
    float dx = dpy * g.J10, dy = dpy * g.J11, dz = dpy * g.J12;
    if (g.rho_raw > 0.f) {
        const float ir = 1.0f / g.rho_raw;
        dx += dpx * sx * g.cz * ir;
        dz -= dpx * sx * g.cx * ir;
    }
    // J(x') through u = cx, w = cz, rho, rho_cap, r2
    const float icap = 1.0f / g.rho_cap, ir2 = 1.0f / g.r2;
    const float gu = -dJ[0][2] * sx * icap - dJ[1][0] * sy * gy * ir2;
    const float gw = dJ[0][0] * sx * icap - dJ[1][2] * sy * gy * ir2;
    const float gcap = (-dJ[0][0] * sx * g.cz + dJ[0][2] * sx * g.cx) * icap * icap;
    const float gr2 = (dJ[1][0] * sy * gy * g.cx - dJ[1][1] * sy * g.rho_raw + dJ[1][2] * sy * gy * g.cz) *
                      ir2 * ir2;
    const float grho = dJ[1][1] * sy * ir2;
    dy += -dJ[1][0] * sy * g.cx * ir2 - dJ[1][2] * sy * g.cz * ir2;
    dx += gr2 * 2.f * gx;
    dy += gr2 * 2.f * gy;
    dz += gr2 * 2.f * gz;
    if (g.rho_raw > 0.f) {
        const float ir = 1.0f / g.rho_raw;
        const float ir3 = ir * ir * ir;
        // u = x/rho, w = z/rho
        dx += gu * gz * gz * ir3 - gw * gx * gz * ir3 + grho * g.cx;
        dz += -gu * gx * gz * ir3 + gw * gx * gx * ir3 + grho * g.cz;
    }
    if (g.clamped) {
        const float f = gcap * kRhoFloor / g.r;
        dx += f * gx;
        dy += f * gy;
        dz += f * gz;
    } else {
        dx += gcap * g.cx;
        dz += gcap * g.cz;
    }
    // x' = V (mu - rx): dmu = V^T dx'; atomic, so that the attribute network's backward may add
    // into the same gradient concurrently
    atomicAdd(&d_means[3 * i + 0], v.V[0] * dx + v.V[3] * dy + v.V[6] * dz);
    atomicAdd(&d_means[3 * i + 1], v.V[1] * dx + v.V[4] * dy + v.V[7] * dz);
    atomicAdd(&d_means[3 * i + 2], v.V[2] * dx + v.V[5] * dy + v.V[8] * dz);
}

}  // namespace
}  // namespace gsparc

