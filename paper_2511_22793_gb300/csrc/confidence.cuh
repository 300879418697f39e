// Confidence-weighted objective (Eq. 5, Sec. 4.2): device code only, so that the same source
// builds into the library and, under a host shim, into the test suite's CPU check of the
// kernel's logic.
//
// A network g: R^3 -> R with one ReLU hidden layer of `hidden` <= 32 units maps each sample's
// query position x_b to the confidence C_b = 1 + exp(g(x_b)); the objective is the mean over
// the batch of C_b L_b - alpha ln C_b, where L_b is the sample's task loss.  One launch forms
// C_b, the objective, dObj/dL_b = C_b / B and accumulates the weight gradients.
//
// Weights, one flat FP32 buffer: W1 [3, hidden] (input-major), b1 [hidden], W2 [hidden],
// b2 [1] -- 5 hidden + 1 values.
#pragma once

namespace gsparc {

constexpr int kConfWarps = 8;                 // one block of 8 warps; a warp per sample at a time
constexpr int kConfMaxHidden = 32;            // one lane per hidden unit

inline int conf_n_weights(int hidden) { return 5 * hidden + 1; }

// Block-wide order of the sums is fixed (warp-stride samples, then warps in index order), so the
// results do not depend on timing.
__global__ void __launch_bounds__(kConfWarps * 32)
k_confidence(int B, int hidden, const float* __restrict__ pos, const float* __restrict__ task_loss,
             const float* __restrict__ w, float alpha, float inv_B, float* __restrict__ conf,
             float* __restrict__ objective, float* __restrict__ d_task_loss, float* __restrict__ d_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool unit = lane < hidden;
    const float w1x = unit ? w[lane] : 0.0f;
    const float w1y = unit ? w[hidden + lane] : 0.0f;
    const float w1z = unit ? w[2 * hidden + lane] : 0.0f;
    const float b1 = unit ? w[3 * hidden + lane] : 0.0f;
    const float w2 = unit ? w[4 * hidden + lane] : 0.0f;
    const float b2 = w[5 * hidden];

    // per-lane weight-gradient partials of hidden unit `lane`, the output bias on lane 0
    float g_w1x = 0.0f, g_w1y = 0.0f, g_w1z = 0.0f, g_b1 = 0.0f, g_w2 = 0.0f, g_b2 = 0.0f;
    double obj = 0.0;
    for (int b = warp; b < B; b += kConfWarps) {        // uniform over the warp
        const float x = pos[3 * b], y = pos[3 * b + 1], z = pos[3 * b + 2];
        const float pre = fmaf(x, w1x, fmaf(y, w1y, fmaf(z, w1z, b1)));
        const bool on = pre > 0.0f;
        const float h = on ? pre : 0.0f;
        float s = h * w2;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float g = s + b2;
        const float e = expf(g);                        // C - 1 = dC/dg
        const float C = 1.0f + e;
        const float L = task_loss[b];
        // d/dg (C L - alpha ln C) / B = (L - alpha / C) (C - 1) / B
        const float dg = (L - alpha / C) * e * inv_B;
        if (lane == 0) {
            obj += (double)C * (double)L - (double)alpha * (double)log1pf(e);
            if (conf) conf[b] = C;
            if (d_task_loss) d_task_loss[b] = C * inv_B;
            g_b2 += dg;
        }
        g_w2 = fmaf(dg, h, g_w2);
        const float dh = on ? dg * w2 : 0.0f;
        g_w1x = fmaf(dh, x, g_w1x);
        g_w1y = fmaf(dh, y, g_w1y);
        g_w1z = fmaf(dh, z, g_w1z);
        g_b1 += dh;
    }

    __shared__ float part[kConfWarps][6][32];
    __shared__ double part_obj[kConfWarps];
    part[warp][0][lane] = g_w1x;
    part[warp][1][lane] = g_w1y;
    part[warp][2][lane] = g_w1z;
    part[warp][3][lane] = g_b1;
    part[warp][4][lane] = g_w2;
    part[warp][5][lane] = g_b2;
    if (lane == 0) part_obj[warp] = obj;
    __syncthreads();
    if (warp != 0) return;
    float t[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (int k = 0; k < kConfWarps; ++k)
        for (int c = 0; c < 6; ++c) t[c] += part[k][c][lane];
    if (d_w && unit) {
        d_w[lane] += t[0];
        d_w[hidden + lane] += t[1];
        d_w[2 * hidden + lane] += t[2];
        d_w[3 * hidden + lane] += t[3];
        d_w[4 * hidden + lane] += t[4];
    }
    if (lane == 0) {
        double o = 0.0;
        for (int k = 0; k < kConfWarps; ++k) o += part_obj[k];
        *objective = (float)(o * (double)inv_B);
        if (d_w) d_w[5 * hidden] += t[5];
    }
}

}  // namespace gsparc
