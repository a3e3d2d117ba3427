// Camera-pose gradient reduction and pose update (CG-SLAM Sec. 3.4).
//
// k_pose_reduce  one CTA per frame: the fixed-order double-float reduction of
//                the frame's pose partials (the same routine the backward
//                kernels run in their last CTA, so results are bit-identical),
//                final value in FP64.
// k_pose_adam    one warp per frame: converts the left se(3) gradient
//                (rho, phi) into the {so(3) | T} form the paper optimises
//                (g_t = g_rho, g_R = g_phi - t x g_rho), updates the FP64 Adam
//                moments, computes the step d = -lr mhat / (sqrt(vhat) + eps) in
//                FP32 (B300 runs FP64 division/sqrt slowly; the step is ~1e-3
//                and its FP32 rounding is far below any tracking tolerance), and
//                applies R <- Exp(d_R) R, t <- t + d_t in FP64. The bias
//                corrections use beta^t kept in the state, not pow().
#include "gs_internal.cuh"
#include "dfloat.cuh"
#include "pose_adam.cuh"

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

__global__ void __launch_bounds__(32)
    k_pose_adam(double *__restrict__ state, const double *__restrict__ grad, float *__restrict__ T_cw,
                int n_frames, gs_adam ad, const int32_t *__restrict__ status) {
    if (status[0] != 0) return;
    const int f = blockIdx.x;
    if (f >= n_frames) return;
    pose_adam_warp(state + (size_t)f * GS_POSE_STATE_DOUBLES, grad + (size_t)f * 6, T_cw + (size_t)f * 12, ad);
}

// The frame's pose reduction and, with adam_state, its Adam step, as one small
// launch chained after the tracking pass (programmatic dependent launch): one
// CTA per frame waits for the pass to complete, sums the frame's per-tile
// partials in the fixed order of reduce_pose_partials (the bits of
// gs_pose_grad_reduce) and applies the pose update in warp 0. No CTA of the
// pass fences or takes an arrival ticket.
__global__ void __launch_bounds__(kRedThreads)
    k_pose_reduce_adam(const float *__restrict__ partials, int per_frame, double *__restrict__ pose_grad,
                       double *__restrict__ adam_state, gs_adam ad, float *__restrict__ T_cw,
                       const int32_t *__restrict__ status) {
    dep_wait();
    __shared__ df s_red[kRedSlots][6];
    if (status[0] != 0) return;
    const int f = blockIdx.x;
    double *st = adam_state ? adam_state + (size_t)f * GS_POSE_STATE_DOUBLES : nullptr;
    // fetch the frame's Adam state (28 doubles, up to three 128-byte lines)
    // into L1 while the partials are being summed
    if (st && threadIdx.x < 3)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(st + (threadIdx.x == 0 ? 0 : (threadIdx.x == 1 ? 14 : 27))));
    // all partials of a slot in one round trip (K <= 8 x 256 per frame at 16x16
    // tiles up to 2048x2048 pixels; longer frames take more rounds)
    reduce_pose_partials<8>(partials + (size_t)f * per_frame * 12, per_frame, pose_grad + (size_t)f * 6, s_red);
    if (st && threadIdx.x < 32) pose_adam_warp(st, pose_grad + (size_t)f * 6, T_cw + (size_t)f * 12, ad);
}

}  // namespace

cudaError_t launch_pose_reduce_adam(const float *partials, int n_frames, int per_frame, double *pose_grad,
                                    double *adam_state, const gs_adam &adam, float *T_cw, const int32_t *status,
                                    cudaStream_t s) {
    if (n_frames == 0) return cudaSuccess;
    return launch_chained(k_pose_reduce_adam, dim3(n_frames), dim3(kRedThreads), 0, s, partials, per_frame, pose_grad,
                          adam_state, adam, T_cw, status);
}

cudaError_t launch_pose_reduce(const float *partials, int n_frames, int per_frame, double *out,
                               const int32_t *status, cudaStream_t s) {
    if (n_frames == 0) return cudaSuccess;
    k_pose_reduce<<<n_frames, kRedThreads, 0, s>>>(partials, per_frame, out, status);
    return cudaGetLastError();
}

cudaError_t launch_pose_adam(double *state, const double *grad, float *T_cw, int n_frames, gs_adam adam,
                             const int32_t *status, cudaStream_t s) {
    if (n_frames == 0) return cudaSuccess;
    k_pose_adam<<<n_frames, 32, 0, s>>>(state, grad, T_cw, n_frames, adam, status);
    return cudaGetLastError();
}

}  // namespace gs
