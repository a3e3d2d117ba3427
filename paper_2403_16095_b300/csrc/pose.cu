// Camera-pose gradient reduction and pose update (CG-SLAM Sec. 3.4).
//
// k_pose_reduce  one CTA per frame: the fixed-order double-float reduction of
//                the frame's pose partials (the same routine the backward
//                kernels run in their last CTA, so results are bit-identical),
//                final value in FP64.
// k_pose_adam    one thread per frame: converts the left se(3) gradient
//                (rho, phi) into the {so(3) | T} form the paper optimises
//                (g_t = g_rho, g_R = g_phi - t x g_rho), updates the FP64 Adam
//                moments, computes the step d = -lr mhat / (sqrt(vhat) + eps) in
//                FP32 (B300 runs FP64 division/sqrt slowly; the step is ~1e-3
//                and its FP32 rounding is far below any tracking tolerance), and
//                applies R <- Exp(d_R) R, t <- t + d_t in FP64. The bias
//                corrections use beta^t kept in the state, not pow().
#include "gs_internal.cuh"
#include "dfloat.cuh"

namespace gs {
namespace {

constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads)
    k_pose_reduce(const float *__restrict__ partials, int per_frame, double *__restrict__ out,
                  const int32_t *__restrict__ status) {
    __shared__ df s_red[kRedSlots][6];
    if (status[0] != 0) return;
    const int f = blockIdx.x;
    reduce_pose_partials(partials + (size_t)f * per_frame * 12, per_frame, out + (size_t)f * 6, s_red);
}

// R = Exp(w) by Rodrigues; for |w| < 0.05 the coefficients come from their
// Taylor series (truncation below 1e-17), avoiding FP64 sin/cos.
__device__ void so3_exp(const double w[3], double R[3][3]) {
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

__global__ void k_pose_adam(double *__restrict__ state, const double *__restrict__ grad, float *__restrict__ T_cw,
                            int n_frames, gs_adam ad, const int32_t *__restrict__ status) {
    if (status[0] != 0) return;
    const int f = threadIdx.x;
    if (f >= n_frames) return;
    double *st = state + (size_t)f * GS_POSE_STATE_DOUBLES;
    double *R = st, *t = st + 9, *m = st + 12, *v = st + 18;
    const double *gr = grad + (size_t)f * 6;
    st[24] += 1.0;                 // step count
    st[25] *= (double)ad.beta1;    // beta1^step
    st[26] *= (double)ad.beta2;    // beta2^step
    const float c1 = (float)(1.0 - st[25]), c2 = (float)(1.0 - st[26]);
    double g[6];
    g[0] = gr[0];
    g[1] = gr[1];
    g[2] = gr[2];
    g[3] = gr[3] - (t[1] * gr[2] - t[2] * gr[1]);
    g[4] = gr[4] - (t[2] * gr[0] - t[0] * gr[2]);
    g[5] = gr[5] - (t[0] * gr[1] - t[1] * gr[0]);
    const double b1 = ad.beta1, b2 = ad.beta2;
    double d[6];
    for (int k = 0; k < 6; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        const float lr = k < 3 ? ad.lr_trans : ad.lr_rot;
        d[k] = (double)(-lr * ((float)m[k] / c1) / (sqrtf((float)v[k] / c2) + ad.eps));
    }
    double dR[3][3], Rn[3][3];
    so3_exp(d + 3, dR);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rn[i][j] = dR[i][0] * R[j] + dR[i][1] * R[3 + j] + dR[i][2] * R[6 + j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[3 * i + j] = Rn[i][j];
    for (int k = 0; k < 3; ++k) t[k] += d[k];
    float *T = T_cw + (size_t)f * 12;
    for (int i = 0; i < 3; ++i) {
        T[4 * i + 0] = (float)R[3 * i + 0];
        T[4 * i + 1] = (float)R[3 * i + 1];
        T[4 * i + 2] = (float)R[3 * i + 2];
        T[4 * i + 3] = (float)t[i];
    }
}

}  // namespace

cudaError_t launch_pose_reduce(const float *partials, int n_frames, int per_frame, double *out,
                               const int32_t *status, cudaStream_t s) {
    if (n_frames == 0) return cudaSuccess;
    k_pose_reduce<<<n_frames, kRedThreads, 0, s>>>(partials, per_frame, out, status);
    return cudaGetLastError();
}

cudaError_t launch_pose_adam(double *state, const double *grad, float *T_cw, int n_frames, gs_adam adam,
                             const int32_t *status, cudaStream_t s) {
    if (n_frames == 0) return cudaSuccess;
    k_pose_adam<<<1, 64, 0, s>>>(state, grad, T_cw, n_frames, adam, status);
    return cudaGetLastError();
}

}  // namespace gs
