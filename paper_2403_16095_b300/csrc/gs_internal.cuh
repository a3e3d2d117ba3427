// Internal declarations shared by the libgs CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/gs.h"

namespace gs {

constexpr int kRecFloats = GS_REC_FLOATS;
constexpr int kJacFloats = GS_JAC_FLOATS;
constexpr int kGrad2d = 12;       // FULL-mode per-record accumulators
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Per-frame constants, passed to kernels by value (<= 64 frames, ~3 KB).
struct FrameDesc {
    int W, H;
    float fx, fy, cx, cy, znear;
    int tiles_x, tiles_y;
    int tile_off;  // first global tile id of the frame
    int pix_off;   // first pixel of the frame in the concatenated images
};
struct FrameTable {
    int n;
    int tile;
    int total_tiles;
    int total_pix;
    FrameDesc f[GS_MAX_FRAMES];
};

// Records of the projection: field offsets in the 16-float record.
enum RecField { R_MX = 0, R_MY, R_CA, R_CB, R_CC, R_OP, R_Z, R_NU, R_CR, R_CG, R_CBL, R_RAD, R_X0, R_Y0, R_X1, R_Y1 };
// FULL-mode accumulator layout per record.
enum GradField { G_MX = 0, G_MY, G_CA, G_CB, G_CC, G_OP, G_Z, G_NU, G_R, G_G, G_B };

struct GaussPtrs {
    const float *means, *log_scales, *quats, *opacity_logit, *colors, *nu;
};

struct ImagePtrs {
    float *color, *depth, *alpha, *unc, *nu_map, *median, *T_final;
    int32_t *n_last, *n_contrib, *median_pos, *dom_pos;
    float *dom_weight;
};

struct LossParams {
    int fused;  // 1: compute dL from the loss spec, 0: read upstream maps
    float w_color, w_depth, w_unc, w_nu, unc_tau, w_align;
    const float *target_color, *target_depth;
    const float *g_color, *g_depth, *g_alpha, *g_unc, *g_nu, *g_median;
};

// Programmatic dependent launch. The kernels of one iteration (projection,
// the four binning kernels, the tracking pass) are launched with
// launch_chained(): the next kernel in the stream may be scheduled while the
// current one drains, instead of after it has completed. Every such kernel
// calls dep_wait() before it touches global memory (reads or writes); the wait
// returns once all earlier work in the stream has completed and its writes are
// visible, so the stream order is kept. For a kernel launched without the
// attribute the wait returns at once. No kernel signals its dependents early
// (griddepcontrol.launch_dependents): a dependent grid parked on the SMs
// during the tail of the one before it measured 6% slower per iteration than
// launching it as the CTAs of that one retire.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                  Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// frame of a global tile id (frames are few: linear scan of a uniform table)
__device__ __forceinline__ int frame_of_tile(const FrameTable &ft, int gtile) {
    int f = 0;
    while (f + 1 < ft.n && gtile >= ft.f[f + 1].tile_off) ++f;
    return f;
}

// message returned by gs_last_error() on this host thread (api.cu)
void set_error_message(const char *msg);

// streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// read once per device and cached; api.cu); grid caps are multiples of it
int device_sm_count();

// The per-tile pair counters of a binning: tile t's counter is p[t stride].
// Each (record, tile) pair of the count and fill passes adds to its tile's
// counter with an atomic; see tile_counters (binning.cu) for where they live.
struct TileCtr {
    uint32_t *p;
    int stride;
};

// ----------------------------------------------------------------- launchers
// project.cu
// tile_counts: p NULL, or the tile counters of a following binning
// (tile_counters), zeroed by launch_bin_clear: the projection then also counts
// the pairs
cudaError_t launch_project(const GaussPtrs &g, int n, const FrameTable &ft, const float *T_cw, float jclamp,
                           float nu_cull, int mode, float *rec, int *touched, float *jac, TileCtr tile_counts,
                           const int32_t *status, cudaStream_t s);
cudaError_t launch_project_bf16(const float *anchors, const uint16_t *packed, int n, const FrameTable &ft,
                                const float *T_cw, float jclamp, float nu_cull, int mode, float *rec, int *touched,
                                float *jac, TileCtr tile_counts, const int32_t *status, cudaStream_t s);
// touched: the projection's tiles_touched (a record is visible iff > 0);
// grad2d: the blend backward's per-record accumulators
cudaError_t launch_project_bwd(const GaussPtrs &g, int n, const FrameTable &ft, const float *T_cw, float jclamp,
                               const int *touched, const float *grad2d, gs_grads grads, float *pose_partials,
                               int per_frame, double *pose_grad, unsigned *counters, const int32_t *status,
                               cudaStream_t s);
// binning.cu
size_t bin_workspace_bytes(int n_records, int capacity);
cudaError_t launch_bin_tiles(const float *rec, const int *touched, int n_records, int n_per_frame,
                             const FrameTable &ft, int capacity, uint32_t *values, uint64_t *keys_out,
                             uint32_t *ranges, uint32_t *order, int32_t *status, void *ws, cudaStream_t s,
                             bool counted = false);  // counted: clear + count already done (counting projection)
// zeroes the tile counters and the binning's scalars (ws) ahead of a counting projection
cudaError_t launch_bin_clear(uint32_t *ranges, const FrameTable &ft, int capacity, void *ws, cudaStream_t s);
// where the binning of this call keeps its tile counters (ranges, or ws)
TileCtr tile_counters(uint32_t *ranges, const FrameTable &ft, int capacity, void *ws);
// render_fwd.cu
// batch: list entries staged per batch at 16x16 and 32x32 tiles (256 or 512;
// other values take 512); queue: NULL for one CTA per tile, else the two
// counters of the persistent form (work_queue.cuh)
cudaError_t launch_render_fwd(const float *rec, const uint32_t *values, const uint32_t *ranges, const uint32_t *order,
                              const FrameTable &ft, const float *obs_depth, const ImagePtrs &out,
                              const int32_t *status, int batch, unsigned *queue, cudaStream_t s);
// render_bwd.cu
// batch / queue as for launch_render_fwd, FULL mode only (POSE mode stages
// 256 entries per batch and runs one CTA per tile)
cudaError_t launch_render_bwd(int mode, const float *rec, const float *jac, const uint32_t *values,
                              const uint32_t *ranges, const uint32_t *order, const FrameTable &ft, const float *obs_depth,
                              const ImagePtrs &fwd, const LossParams &lp, float *grad2d, float *pose_partials,
                              int per_frame, double *pose_grad, unsigned *counters, const int32_t *status,
                              int batch, unsigned *queue, cudaStream_t s);
// pack.cu
size_t spatial_order_workspace_bytes(int n);
cudaError_t launch_spatial_order(const float *means, int n, uint32_t *perm, void *ws, const int32_t *status,
                                 cudaStream_t s);
cudaError_t launch_pack_bf16(const GaussPtrs &g, int n, const uint32_t *perm, float *anchors, uint16_t *packed,
                             const int32_t *status, cudaStream_t s);
// render_fused.cu
// writes one pose partial per tile; launch_pose_reduce_adam then sums them
cudaError_t launch_render_fused_pose(const float *rec, const float *jac, const uint32_t *values,
                                     const uint32_t *ranges, const uint32_t *order, const FrameTable &ft,
                                     const ImagePtrs &out, const LossParams &lp, float *pose_partials, int per_frame,
                                     const int32_t *status, cudaStream_t s);
// nu.cu
cudaError_t launch_nu_accumulate(const float *rec, const uint32_t *values, const FrameTable &ft, int n_gaussians,
                                 const float *obs_depth, const int32_t *dom_pos, const float *dom_weight,
                                 double *nu_num, uint32_t *nu_cnt, int32_t *dominant, const int32_t *status,
                                 cudaStream_t s);
cudaError_t launch_nu_finalize(int n, const double *nu_num, const uint32_t *nu_cnt, float *nu, float tau,
                               float low_logit, float *opacity_logit, uint32_t *n_over, const int32_t *status,
                               cudaStream_t s);
// pose.cu
cudaError_t launch_pose_reduce(const float *partials, int n_frames, int per_frame, double *out,
                               const int32_t *status, cudaStream_t s);
cudaError_t launch_pose_adam(double *state, const double *grad, float *T_cw, int n_frames, gs_adam adam,
                             const int32_t *status, cudaStream_t s);
// pose reduction (+ Adam step when adam_state is not NULL), chained after the tracking pass
cudaError_t launch_pose_reduce_adam(const float *partials, int n_frames, int per_frame, double *pose_grad,
                                    double *adam_state, const gs_adam &adam, float *T_cw, const int32_t *status,
                                    cudaStream_t s);

}  // namespace gs
