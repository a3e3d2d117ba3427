// Per-Gaussian depth uncertainty nu (CG-SLAM Eq. 13, Sec. 3.2).
//
// The forward pass (DOM variant) leaves, per pixel, the tile-list position of
// the entry with the largest blend weight w = alpha T and that weight. Here each
// such "dominated pixel" hands w (D_p - d_i)^2 and a count of one to its
// Gaussian i; a second kernel divides, and applies the tau rule.
//
// Bound: one pass over the pixels (dom_pos, dom_weight, D: 12 B per pixel, plus
// a 4-B record read and two atomics per covered pixel) and one pass over the
// Gaussians (8 + 4 + 4 (+4) B). Both are small beside the blend they follow; the
// FP64 atomics resolve in L2.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int frame_of_pixel(const FrameTable &ft, int p) {
    int f = 0;
    while (f + 1 < ft.n && p >= ft.f[f + 1].pix_off) ++f;
    return f;
}

__global__ void __launch_bounds__(kThreads)
    k_nu_accumulate(const float *__restrict__ rec, const uint32_t *__restrict__ values, FrameTable ft, int n_gauss,
                    const float *__restrict__ obs_depth, const int32_t *__restrict__ dom_pos,
                    const float *__restrict__ dom_weight, double *__restrict__ nu_num, uint32_t *__restrict__ nu_cnt,
                    int32_t *__restrict__ dominant, const int32_t *__restrict__ status) {
    if (status[0] != 0) return;
    for (int p = blockIdx.x * kThreads + threadIdx.x; p < ft.total_pix; p += gridDim.x * kThreads) {
        const int pos = dom_pos[p];
        int gi = -1;
        if (pos >= 0) {
            const int f = frame_of_pixel(ft, p);
            const uint32_t r = values[pos];
            gi = (int)(r - (uint32_t)f * (uint32_t)n_gauss);
            const double dz = (double)rec[(size_t)r * kRecFloats + R_Z] - (double)obs_depth[p];
            atomicAdd(nu_num + gi, (double)dom_weight[p] * dz * dz);
            atomicAdd(nu_cnt + gi, 1u);
        }
        if (dominant) dominant[p] = gi;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_nu_finalize(int n, const double *__restrict__ nu_num, const uint32_t *__restrict__ nu_cnt, float *__restrict__ nu,
                  float tau, float low_logit, float *__restrict__ opacity_logit, uint32_t *__restrict__ n_over,
                  const int32_t *__restrict__ status) {
    if (status[0] != 0) return;
    unsigned over_here = 0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const uint32_t c = nu_cnt[i];
        double v;
        if (c > 0) {
            v = nu_num[i] / (double)c;
            nu[i] = (float)v;
        } else {
            v = (double)nu[i];
        }
        if (tau > 0.f && opacity_logit && v > (double)tau) {
            opacity_logit[i] = fminf(opacity_logit[i], low_logit);
            ++over_here;
        }
    }
    if (n_over) {
        const unsigned w = __reduce_add_sync(0xffffffffu, over_here);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(n_over, w);
    }
}

int grid_for(long long items) {
    const long long want = (items + kThreads - 1) / kThreads;
    const long long cap = 8LL * device_sm_count();
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_nu_accumulate(const float *rec, const uint32_t *values, const FrameTable &ft, int n_gaussians,
                                 const float *obs_depth, const int32_t *dom_pos, const float *dom_weight,
                                 double *nu_num, uint32_t *nu_cnt, int32_t *dominant, const int32_t *status,
                                 cudaStream_t s) {
    if (ft.total_pix == 0) return cudaSuccess;
    k_nu_accumulate<<<grid_for(ft.total_pix), kThreads, 0, s>>>(rec, values, ft, n_gaussians, obs_depth, dom_pos,
                                                                dom_weight, nu_num, nu_cnt, dominant, status);
    return cudaGetLastError();
}

cudaError_t launch_nu_finalize(int n, const double *nu_num, const uint32_t *nu_cnt, float *nu, float tau,
                               float low_logit, float *opacity_logit, uint32_t *n_over, const int32_t *status,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_nu_finalize<<<grid_for(n), kThreads, 0, s>>>(n, nu_num, nu_cnt, nu, tau, low_logit, opacity_logit, n_over,
                                                   status);
    return cudaGetLastError();
}

}  // namespace gs
