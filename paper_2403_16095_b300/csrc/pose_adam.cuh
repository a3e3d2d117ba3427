// One Adam step on the camera pose in the {so(3) | T} form of CG-SLAM Sec. 3.4,
// executed by one warp; shared by the stand-alone step (pose.cu) and the
// tracking pass, which applies it in the CTA that reduces the frame's pose
// gradient (render_fused.cu). The arithmetic is the same in both.
#pragma once

#include "gs_internal.cuh"

namespace gs {

// R = Exp(w) by Rodrigues; for |w| < 0.05 the coefficients come from their
// Taylor series (truncation below 1e-17), avoiding FP64 sin/cos.
__device__ __forceinline__ void so3_exp(const double w[3], double R[3][3]) {
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double a, b;
    if (th2 < 2.5e-3) {
        a = 1.0 - th2 * (1.0 / 6.0 - th2 * (1.0 / 120.0 - th2 * (1.0 / 5040.0)));
        b = 0.5 - th2 * (1.0 / 24.0 - th2 * (1.0 / 720.0 - th2 * (1.0 / 40320.0)));
    } else {
        const double th = sqrt(th2);
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    const double K[3][3] = {{0.0, -w[2], w[1]}, {w[2], 0.0, -w[0]}, {-w[1], w[0], 0.0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double KK = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
            R[i][j] = (i == j ? 1.0 : 0.0) + a * K[i][j] + b * KK;
        }
}

// One warp per frame: lane k < 6 updates moment k and its step; lanes 0-8 form
// one entry each of the composed rotation; lanes 9-11 the translation. st: the
// frame's GS_POSE_STATE_DOUBLES; gr: its FP64 (rho, phi) gradient; T: its
// float[3][4] pose, rewritten.
__device__ __forceinline__ void pose_adam_warp(double *st, const double *gr, float *T, const gs_adam &ad) {
    const int lane = threadIdx.x & 31;
    double *R = st, *t = st + 9, *m = st + 12, *v = st + 18;
    const double p1 = st[25] * (double)ad.beta1, p2 = st[26] * (double)ad.beta2;  // beta^step
    const float c1 = (float)(1.0 - p1), c2 = (float)(1.0 - p2);
    const double Rold = lane < 9 ? R[lane] : 0.0;
    double dk = 0.0;
    if (lane < 6) {
        double g;
        switch (lane) {  // {so(3) | T}: g_t = g_rho, g_R = g_phi - t x g_rho
            case 3: g = gr[3] - (t[1] * gr[2] - t[2] * gr[1]); break;
            case 4: g = gr[4] - (t[2] * gr[0] - t[0] * gr[2]); break;
            case 5: g = gr[5] - (t[0] * gr[1] - t[1] * gr[0]); break;
            default: g = gr[lane];
        }
        const double b1 = ad.beta1, b2 = ad.beta2;
        const double mk = b1 * m[lane] + (1.0 - b1) * g;
        const double vk = b2 * v[lane] + (1.0 - b2) * g * g;
        m[lane] = mk;
        v[lane] = vk;
        const float lr = lane < 3 ? ad.lr_trans : ad.lr_rot;
        dk = (double)(-lr * ((float)mk / c1) / (sqrtf((float)vk / c2) + ad.eps));
    }
    double d[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) d[k] = __shfl_sync(0xffffffffu, dk, k);
    double dR[3][3];
    so3_exp(d + 3, dR);
    // Rn[i][j] = sum_l dR[i][l] R[l][j]; lane i*3+j holds R[i][j] in Rold
    double Rc[3][3];
#pragma unroll
    for (int e = 0; e < 9; ++e) Rc[e / 3][e % 3] = __shfl_sync(0xffffffffu, Rold, e);
    __syncwarp();
    if (lane < 9) {
        const int i = lane / 3, j = lane % 3;
        const double rn = dR[i][0] * Rc[0][j] + dR[i][1] * Rc[1][j] + dR[i][2] * Rc[2][j];
        R[lane] = rn;
        T[4 * i + j] = (float)rn;
    } else if (lane < 12) {
        const int k = lane - 9;
        const double tn = t[k] + d[k];
        t[k] = tn;
        T[4 * k + 3] = (float)tn;
    }
    if (lane == 0) {
        st[24] += 1.0;  // step count
        st[25] = p1;
        st[26] = p2;
    }
}

}  // namespace gs
