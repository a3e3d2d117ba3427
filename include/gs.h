/*
 * gs.h -- C ABI of libgs, a B300 (sm_103a) implementation of the
 * differentiable tile-based 3D Gaussian rasterizer that CG-SLAM
 * (arXiv 2403.16095) runs in every tracking and mapping iteration.
 *
 * Pipeline for one iteration (all calls asynchronous on one CUDA stream, no
 * host synchronisation, no allocation -- the sequence can be captured in a
 * CUDA graph):
 *
 *   gs_project          Eq. 1-2   activate parameters, EWA-project each Gaussian
 *   gs_bin_tiles        Sec. 3.1  duplicate per overlapped tile, sort the 64-bit
 *                                 (tile id, depth) keys per tile, tile ranges
 *                                 (gs_project_bin: both calls in one, the
 *                                 projection counting the pairs)
 *   gs_render_fwd       Eq. 3-10  front-to-back alpha blending per pixel
 *   gs_render_bwd       Eq. 3-10 adjoint (+ Eq. 14/16/19 loss when fused):
 *                                 reverse walk of each tile list; gradients to the
 *                                 pose (POSE mode) or to every Gaussian parameter
 *                                 and the pose (FULL mode)
 *   gs_pose_grad_reduce Sec. 3.4  deterministic FP64 sum of the pose partials
 *   gs_pose_adam_step   Sec. 3.4/4 one Adam step of the pose in {so(3)|T} form
 *
 * Conventions shared by every call
 *   - Memory: the caller owns every buffer. Pointers documented "device" must
 *     be device memory of the current device; "host" means host memory read
 *     during the call only. The library never allocates, frees, or keeps a
 *     pointer past the call. Scratch space is passed as (ws, ws_bytes) after
 *     querying the *_workspace_size function.
 *   - Errors: argument errors return a status synchronously (nothing is
 *     launched). Conditions only the device can see (pair-buffer overflow) are
 *     written to the device status word `status` (int32[4]): status[0] is a
 *     gs_status code (0 = OK), status[1] the number of (Gaussian, tile) pairs
 *     the last gs_bin_tiles needed. Every kernel reads status[0] first and does
 *     nothing if it is non-zero, so a failed iteration never reads past a
 *     buffer. The caller zeroes the status word (e.g. per frame). A failed CUDA
 *     launch returns GS_ERR_CUDA. gs_last_error() gives a message for the last
 *     non-OK status returned on the calling host thread.
 *   - Camera: pinhole intrinsics, world->camera pose T_cw = [R | t] (3x4
 *     row-major float), camera axes x right, y down, z forward. Pixel (i, j)
 *     (column i, row j) has its centre at (i + 0.5, j + 0.5).
 *   - Frames: a call may process F frames at once (F <= GS_MAX_FRAMES) with
 *     their own camera and pose. Records are indexed r = f * n_gaussians + i.
 *     Images of frame f occupy pixels [pix_off_f, pix_off_f + H_f * W_f) with
 *     pix_off the exclusive prefix sum of H_f * W_f; a one-channel image is
 *     [pix][...] = buf[pix_off_f + y * W_f + x]; the colour image is planar per
 *     frame: buf[3 * pix_off_f + c * H_f * W_f + y * W_f + x] (i.e. [F][3][H][W]
 *     for equal frames). Tiles of frame f are numbered tile_off_f + ty * tx_f + tx.
 *   - Threshold constants (prior-art readings where the paper is silent):
 *     near-plane cull z <= znear, 0.3 px^2 dilation, q <= 9 footprint,
 *     alpha = min(0.99, opacity * G), entries with alpha < 1/255 skipped,
 *     blending stops before an entry that would take T below 1e-4.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_MAX_FRAMES 64
#define GS_ABI_VERSION 9

typedef struct CUstream_st *gs_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or option            */
    GS_ERR_CAPACITY = 2,      /* pair buffer too small; status[1] holds the need   */
    GS_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed              */
    GS_ERR_TIMEOUT = 4,       /* a bounded device wait gave up                     */
    GS_ERR_UNSUPPORTED = 5    /* option combination not built                      */
} gs_status;

enum { GS_MODE_FWD = 0, GS_MODE_POSE = 1, GS_MODE_FULL = 2 };

/* Pinhole camera of one frame (host struct). */
typedef struct {
    int width, height;     /* pixels, 1..16384                                  */
    float fx, fy, cx, cy;  /* focal lengths and principal point in pixels       */
    float znear;           /* Gaussians with camera z <= znear are culled       */
} gs_camera;

/* Gaussian parameters (Eq. 1), FP32, device, row-major, [n][k]. */
typedef struct {
    int n;                      /* number of Gaussians                          */
    const float *means;         /* [n][3] world-space centres X                 */
    const float *log_scales;    /* [n][3] s = exp(log_scale)                    */
    const float *quats;         /* [n][4] (w,x,y,z), normalised inside; |q|=0 culls */
    const float *opacity_logit; /* [n]    opacity = sigmoid(logit)              */
    const float *colors;        /* [n][3] RGB (degree-0 colour used as is)      */
    const float *nu;            /* [n]    per-Gaussian uncertainty (Eq. 13)     */
} gs_gaussians;

enum { GS_SCHED_TILE = 0, GS_SCHED_PERSISTENT = 1 };

typedef struct {
    int tile;        /* tile edge in pixels: 8, 16 or 32                         */
    int mode;        /* GS_MODE_FWD / GS_MODE_POSE / GS_MODE_FULL                 */
    float jclamp;    /* clamp of x/z, y/z in the EWA Jacobian, in units of the half
                        field of view (1.3 typical); <= 0 disables the clamp       */
    float nu_cull;   /* > 0: Gaussians with nu > nu_cull are culled (Sec. 3.2);
                        <= 0: off                                                  */
    int batch;       /* list entries gs_render_fwd and the FULL-mode gs_render_bwd
                        stage in shared memory per batch at 16x16 and 32x32 tiles:
                        256 or 512 (0 = 512); 8x8 tiles stage 64. Speed only: the
                        results do not depend on it                                */
    int sched;       /* GS_SCHED_TILE: one CTA per tile, heaviest tiles first;
                        GS_SCHED_PERSISTENT: gs_render_fwd and the FULL-mode
                        gs_render_bwd run as many CTAs as fit on the GPU, each
                        pulling (frame, tile) items in launch order from the device
                        work queue tiles->queue (required then). Speed only; the
                        POSE-mode backward and the tracking pass always run one CTA
                        per tile                                                   */
} gs_opts;

/* Projected records (output of gs_project), device, caller-allocated.
 * rec: GS_REC_FLOATS floats per record, 16-byte aligned:
 *   [0..1] mean2d (pixels)   [2..4] conic (A, B, C): q = A dx^2 + 2B dx dy + C dy^2
 *   [5] opacity  [6] depth z  [7] nu  [8..10] RGB  [11] radius (pixels)
 *   [12..15] int32 inclusive pixel rect x0, y0, x1, y1 (x0 > x1: culled; the
 *   other fields of a culled record are not written).                        */
#define GS_REC_FLOATS 16
#define GS_JAC_FLOATS 36
typedef struct {
    int n_gaussians;      /* N                                                 */
    int n_frames;         /* F; records = F * N                                */
    float *rec;           /* [F*N][16]                                         */
    int *tiles_touched;   /* [F*N] tiles overlapped (0 if culled); read by the
                             binning and the FULL-mode gs_render_bwd. The blend
                             calls that read only rec (gs_render_fwd, the POSE
                             backward, gs_render_fwd_bwd_pose, gs_nu_accumulate)
                             accept NULL here                                   */
    float *pose_jac;      /* [F*N][6][6] d(mean2d.x, mean2d.y, A, B, C, z)/d(rho, phi),
                             written in POSE mode only; may be NULL otherwise
                             (and when F*N = 0)                                 */
} gs_projected;

/* Tile lists (output of gs_bin_tiles), device, caller-allocated. */
typedef struct {
    int capacity;         /* pairs the value/key buffers hold                  */
    int n_tiles;          /* sum over frames of tiles_x * tiles_y              */
    uint32_t *values;     /* [capacity] record index of each pair, sorted by
                             (tile id, float bits of depth, record index)      */
    uint64_t *keys;       /* [capacity] sorted keys (tile << 32 | depth bits), or NULL */
    uint32_t *ranges;     /* [n_tiles][2] [start, end) of each tile's pairs;
                             an empty tile has start == end                    */
    uint32_t *order;      /* NULL, or [n_tiles]: every tile id once, longest
                             list first (lengths bucketed by 4, order within a
                             bucket unspecified). gs_bin_tiles writes it;
                             gs_render_fwd / gs_render_bwd then start the
                             heaviest tiles first. Results do not depend on it. */
    uint32_t *queue;      /* NULL, or [2] device counters of the persistent
                             blend kernels (opts->sched = GS_SCHED_PERSISTENT):
                             zero-filled by the caller before first use; every
                             persistent launch leaves them at zero again. A
                             persistent launch owns them until it completes, so
                             two launches sharing one queue must be ordered on
                             one stream. No kernel waits on another CTA.        */
} gs_tiles;

/* Rendered channels (Eq. 3-10), device, FP32 except n_last. A NULL member is not
 * written; color, T_final and n_last are required. */
typedef struct {
    float *color;    /* [.][3][H][W] Eq. 3                                       */
    float *depth;    /* alpha-blended depth, Eq. 6 (not normalised by opacity)   */
    float *alpha;    /* accumulated opacity, Eq. 9                               */
    float *unc;      /* depth uncertainty U, Eq. 10 (needs obs_depth)            */
    float *nu_map;   /* blended per-Gaussian uncertainty sum w_i nu_i            */
    float *median;   /* median depth, Eq. 7-8 (0 if T never drops below 0.5)     */
    float *T_final;  /* transmittance after the last blended Gaussian            */
    int32_t *n_last; /* one past the tile-list position of the last blended entry */
    int32_t *n_contrib; /* number of blended entries per pixel, or NULL            */
    int32_t *median_pos; /* tile-list position of the median entry (-1: none), or
                            NULL; needed by a backward with a median-depth gradient */
    int32_t *dom_pos;    /* tile-list position of the pixel's dominant entry, the one
                            with the largest blend weight w = alpha T (the first in
                            blend order on ties; -1: none), or NULL (Sec. 3.2)    */
    float *dom_weight;   /* that weight (0: none); set iff dom_pos is set          */
} gs_image;

/* Upstream gradients dL/d(channel) per pixel (same layouts); NULL = zero. A
 * median-depth gradient flows to the depth of the median entry (Eq. 7-8). */
typedef struct {
    const float *color, *depth, *alpha, *unc, *nu_map, *median;
} gs_image_grad;

/* Fused per-pixel loss (Eq. 14, 16, 19; Eq. 11 and 12 optional), per frame f:
 *   L_f = 1/(H W) sum_p [ m_p (w_color sum_c |C - C*| + w_depth |D - D*|)
 *                          + w_unc |U| + w_nu nu_map + w_align |D - D_median| ],
 *   m_p = 1 / (1 + nu_map_p / unc_tau) if unc_tau > 0 else 1 (no gradient through m).
 * The total loss is sum_f L_f. sign(0) = 0. w_align needs the forward's median
 * and median_pos channels. */
typedef struct {
    float w_color, w_depth, w_unc, w_nu, unc_tau;
    const float *target_color;  /* [.][3][H][W] device                        */
    const float *target_depth;  /* [.][H][W] device (also the sensor depth of U) */
    float w_align;              /* L_align of Eq. 12                          */
} gs_loss;

/* 16-bit storage of the Gaussians (tracking and rendering; mapping keeps FP32).
 * Gaussian i is the 32-byte record packed[i] of 16 16-bit values
 *   (q x, y, z: uint16 fixed-point mean; then BF16 log-scale x, y, z,
 *    quat w, x, y, z, opacity logit, r, g, b, nu, 0)
 * and chunk c = i / GS_BF16_CHUNK has the FP32 box anchors[c] =
 *   (lo x, lo y, lo z, step x, step y, step z, 0, 0);
 * mean = lo + step * q per axis (FP32 multiply, then add). Written by
 * gs_pack_bf16.                                                            */
#define GS_BF16_CHUNK 256
typedef struct {
    int n;
    const float *anchors;    /* [ceil(n / GS_BF16_CHUNK)][8], 16-byte aligned */
    const uint16_t *packed;  /* [n][16], 16-byte aligned                     */
} gs_gaussians_bf16;

/* Parameter gradients (FULL mode), device, same layouts as gs_gaussians,
 * summed over frames; overwritten (not accumulated). NULL member = skipped. */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logit, *colors, *nu;
} gs_grads;

/* Adam hyper-parameters of the pose step (Sec. 4: lr_rot 0.0015, lr_trans 0.00215). */
typedef struct {
    float lr_rot, lr_trans, beta1, beta2, eps;
} gs_adam;

#define GS_POSE_STATE_DOUBLES 28  /* R[9], t[3], m[6], v[6], step, beta1^step, beta2^step, unused */

/* ------------------------------------------------------------------ calls */

/* ABI version and a message for the last non-OK status on this host thread. */
int gs_abi_version(void);
const char *gs_last_error(void);

/* Eq. 1-2. For each frame f and Gaussian i: s = exp(ls), q_hat = q/|q|,
 * Sigma = R S S^T R^T, opacity = sigmoid(logit); p = R_cw X + t_cw, cull
 * z <= znear; J = [[fx/z, 0, -fx u/z], [0, fy/z, -fy v/z]] with (u, v) = (x/z, y/z)
 * clamped to +-jclamp * (W/2fx, H/2fy); Sigma_2d = J R_cw Sigma R_cw^T J^T + 0.3 I,
 * conic = Sigma_2d^-1; mean2d = (fx x/z + cx, fy y/z + cy);
 * radius = ceil(3 sqrt(lambda_max)); pixel rect = [ceil(mx - .5 - r), floor(mx - .5 + r)]
 * clipped to the image (same in y); tiles_touched = area of the tile rect.
 * In POSE mode also writes pose_jac (forward-mode derivative of mean2d, conic and
 * z w.r.t. a left perturbation Exp(xi) T_cw, xi = (rho, phi)).
 *   cams: host [n_frames]; T_cw: device [n_frames][3][4].                    */
gs_status gs_project(const gs_gaussians *g, int n_frames, const gs_camera *cams, const float *T_cw,
                     const gs_opts *opts, gs_projected *out, const int32_t *status, gs_stream stream);

/* gs_project with BF16 storage (same outputs; FWD and POSE modes; FULL mode,
 * which differentiates the stored parameters, returns GS_ERR_UNSUPPORTED). */
gs_status gs_project_bf16(const gs_gaussians_bf16 *g, int n_frames, const gs_camera *cams, const float *T_cw,
                          const gs_opts *opts, gs_projected *out, const int32_t *status, gs_stream stream);

/* Spatial order for BF16 packing (no counterpart in the paper; it makes the
 * chunks of GS_BF16_CHUNK Gaussians compact). perm[j] = index of the j-th
 * Gaussian in the order of the 30-bit Morton code of its mean, quantised to
 * 1024 steps per axis over the bounding box of all means:
 *   q = min(1023, floor((m - lo) * (1024 / (hi - lo))))  in FP32 (round to
 *   nearest; q = 0 on an axis with hi == lo), bits interleaved x, y, z from
 *   the lowest up; ties in index order. Deterministic.
 *   means: device [n][3]; perm: device uint32 [n]; ws: 256-byte aligned.    */
size_t gs_spatial_order_workspace_size(int n);
gs_status gs_spatial_order(const float *means, int n, uint32_t *perm, void *ws, size_t ws_bytes,
                           const int32_t *status, gs_stream stream);

/* Packs FP32 Gaussians (in the order perm, or as they are if perm is NULL) into
 * the 16-bit layout above. Per chunk, from its means' bounding box [lo, hi]:
 * step = (hi - lo) / 65535 and q = rint((m - lo) / step) clamped to [0, 65535]
 * (FP32, round to nearest even; q = 0 where step = 0), so a stored mean is
 * within step/2 (plus FP32 rounding) of the original. The other values are
 * rounded to the nearest BF16 (ties to even).
 *   anchors: device float [ceil(n/GS_BF16_CHUNK)][8]; packed: device [n][16].  */
gs_status gs_pack_bf16(const gs_gaussians *src, const uint32_t *perm, float *anchors, uint16_t *packed,
                       const int32_t *status, gs_stream stream);

/* Sec. 3.1 pre-sort. Emits one (key, record) pair per tile overlapped by each
 * record's tile rect, key = (global tile id << 32) | float bits of z, sorts the
 * pairs by key, ties in record order (a counting pass by tile, then a radix sort
 * of (z bits, record) inside each tile), and writes each tile's [start, end). The result is bit-exact and independent of the
 * launch configuration. If the pairs exceed tiles->capacity, status[0] is set to
 * GS_ERR_CAPACITY and status[1] to the pairs needed; later kernels then no-op.
 *   status: device int32[4]; ws: device scratch of
 *   gs_bin_tiles_workspace_size(records, capacity) bytes, 256-byte aligned.   */
size_t gs_bin_tiles_workspace_size(int n_records, int capacity);
gs_status gs_bin_tiles(const gs_projected *proj, int n_frames, const gs_camera *cams,
                       const gs_opts *opts, gs_tiles *tiles, int32_t *status, void *ws,
                       size_t ws_bytes, gs_stream stream);

/* gs_project (gs_project_bf16) followed by gs_bin_tiles, in one call: the
 * projection kernel also counts each visible record's (record, tile) pairs into
 * the tile counters, so the binning skips its count pass (one pass over the
 * records and one launch fewer). Arguments: those of the two calls (ws: the
 * binning workspace); the same validation; outputs (records, tiles_touched,
 * pose_jac, tiles) bit-identical to the two calls. It pays for one frame at a
 * time (tracking: 199.7 -> 196.5 us per iteration at 640x480 / 300k); on
 * multi-frame batches the separate count kernel, 8 records per thread, is the
 * faster one (8 x 640x480 / 1M: 0.92 vs 0.96 ms).                          */
gs_status gs_project_bin(const gs_gaussians *g, int n_frames, const gs_camera *cams, const float *T_cw,
                         const gs_opts *opts, gs_projected *out, gs_tiles *tiles, int32_t *status,
                         void *ws, size_t ws_bytes, gs_stream stream);
gs_status gs_project_bin_bf16(const gs_gaussians_bf16 *g, int n_frames, const gs_camera *cams,
                              const float *T_cw, const gs_opts *opts, gs_projected *out, gs_tiles *tiles,
                              int32_t *status, void *ws, size_t ws_bytes, gs_stream stream);

/* gs_bin_tiles for callers that cannot allocate device memory (the paper has no
 * counterpart; this is an interface convenience). Some callers cannot call
 * cudaMalloc where they bin -- a real-time tracking thread that must not block
 * on the allocator, a process whose device memory belongs to another
 * framework's pool, a plug-in limited to memory declared at load time. This
 * call takes the same arguments as gs_bin_tiles minus the workspace, and uses a
 * static device scratch array of 12 MiB held by every GPU that loads libgs
 * until exit. Limits: tiles->capacity <= GS_NOALLOC_MAX_PAIRS, else
 * GS_ERR_INVALID_ARG with a message. It allocates nothing. Its first call on a
 * device (with that device current) looks up the array's address; make that
 * first call before any stream capture. After the device's context is
 * destroyed (cudaDeviceReset), the next call is a first call again: it finds a
 * new context current and looks the address up anew. All calls share the array: calls that
 * overlap on the GPU race; sequential calls are independent (every scratch word
 * is written before it is read). Outputs and errors as gs_bin_tiles.          */
#define GS_NOALLOC_MAX_PAIRS (1 << 19)
gs_status gs_bin_tiles_noalloc(const gs_projected *proj, int n_frames, const gs_camera *cams,
                               const gs_opts *opts, gs_tiles *tiles, int32_t *status, gs_stream stream);

/* Eq. 3-10. One CTA per tile: the tile's sorted list is staged in shared memory
 * in batches and every pixel blends front to back (alpha test, stop rule,
 * median crossing of T = 0.5) until all of the tile's pixels are done. A list
 * entry is blended by the pixels with q <= 9 (and alpha >= 1/255): the pixel
 * rect of the record contains that ellipse (q >= dx^2 / lambda_max and
 * r >= 3 sqrt(lambda_max)), so the rect is not tested per pixel; in FP32 the
 * two can differ only where q is within ~1e-6 of 9.
 *   obs_depth: device [.][H][W] sensor depth D for U (Eq. 10), or NULL (U not written). */
gs_status gs_render_fwd(const gs_projected *proj, const gs_tiles *tiles, int n_frames,
                        const gs_camera *cams, const float *obs_depth, const gs_opts *opts,
                        gs_image *out, const int32_t *status, gs_stream stream);

/* Adjoint of gs_render_fwd. Each tile's list is walked back to front from the
 * last blended entry, recovering T_i = T_{i+1} / (1 - alpha_i) instead of
 * storing it. Per-pixel dL/d(channel) come from `dL` or, when `loss` is not
 * NULL, from the fused loss above (dL is then ignored).
 *   POSE mode: every pixel contracts its gradient w.r.t. (mean2d, conic, z) of
 *     each blended Gaussian with that record's pose_jac; the tile's pixels are
 *     reduced by warp shuffles and a fixed block tree into one compensated
 *     partial per tile: pose_partials[f][local tile][6].
 *   FULL mode: per-record gradients of (mean2d, conic, opacity, z, nu, RGB) are
 *     accumulated (warp-reduced, then atomics), chained through the projection
 *     to `grads` (needs `g` and T_cw) and the pose partial of each block of 256
 *     records is written to pose_partials[f][block][6].
 * Partials are double-floats: float [F][K][6][2] = (hi, lo) with value hi + lo,
 * K = gs_pose_partials_per_frame(); unused slots are zeroed. If pose_grad is
 * not NULL, the last CTA of each frame also reduces that frame's partials into
 * pose_grad[f][6] (FP64), exactly as gs_pose_grad_reduce would (bit-identical),
 * saving a launch. ws: gs_render_bwd_workspace_size bytes, 256-byte aligned,
 * zero-filled before its first use (one cudaMemset after allocating it): its
 * last 256 bytes hold the arrival counters of that reduction, which every call
 * leaves at zero again, so no call clears them. A ws whose counters are not
 * zero gives a wrong pose_grad. The FULL backward takes a record's
 * visibility from proj->tiles_touched (> 0), as gs_project wrote it.         */
int gs_pose_partials_per_frame(int mode, int n_gaussians, int n_frames, const gs_camera *cams, int tile);
size_t gs_render_bwd_workspace_size(int n_records, int mode);
gs_status gs_render_bwd(const gs_projected *proj, const gs_tiles *tiles, int n_frames,
                        const gs_camera *cams, const float *T_cw, const gs_gaussians *g,
                        const float *obs_depth, const gs_image *fwd, const gs_image_grad *dL,
                        const gs_loss *loss, const gs_opts *opts, gs_grads *grads,
                        float *pose_partials, double *pose_grad, const int32_t *status, void *ws,
                        size_t ws_bytes, gs_stream stream);

/* Tracking pass: the forward blend (Eq. 3-10) and the POSE-mode backward of the
 * fused tracking loss (Eq. 14, 16, 19: L1 colour and depth, optionally weighted
 * by 1/(1 + nu_map/unc_tau)) in one pass per tile, with nothing written in
 * between. Equal bit for bit to gs_render_fwd followed by gs_render_bwd (POSE)
 * with the same loss. Only losses with w_unc = w_nu = w_align = 0
 * (GS_ERR_UNSUPPORTED otherwise). `out` may be NULL, or name any of color,
 * depth, nu_map, T_final and n_last to have them written as well (its other
 * members are ignored). pose_partials, pose_grad and ws as for gs_render_bwd
 * in POSE mode (ws: gs_render_bwd_workspace_size(records, GS_MODE_POSE)).
 * Two launches: the pass writes one pose partial per tile; if pose_grad is not
 * NULL, a chained launch then sums each frame's partials into pose_grad, bit
 * for bit as gs_pose_grad_reduce, and, if adam_state is not NULL (then adam
 * and T_cw are required), applies gs_pose_adam_step to every frame (same
 * arithmetic), rewriting T_cw for the next iteration.                        */
gs_status gs_render_fwd_bwd_pose(const gs_projected *proj, const gs_tiles *tiles, int n_frames,
                                 const gs_camera *cams, const gs_loss *loss, const gs_opts *opts,
                                 gs_image *out, float *pose_partials, double *pose_grad,
                                 double *adam_state, const gs_adam *adam, float *T_cw,
                                 const int32_t *status, void *ws, size_t ws_bytes, gs_stream stream);

/* Per-Gaussian depth uncertainty, Eq. 13 (Sec. 3.2), accumulation half. Each
 * pixel of the n_frames images whose forward found a dominant entry
 * (fwd->dom_pos >= 0) adds, for that entry's Gaussian i,
 *     nu_num[i] += w (D_p - d_i)^2   (FP64; w = fwd->dom_weight, D_p = obs_depth,
 *                                     d_i = the record's projected depth z)
 *     nu_cnt[i] += 1                 (its dominated pixels M)
 * Calls add to the caller's arrays: zero them, then accumulate every frame of the
 * keyframe window (one batched call or several). The FP64 additions run in an
 * unspecified order (atomics): nu_num is reproducible to FP64 rounding, nu_cnt
 * exactly. dominant: NULL or int32 [.][H][W], set to the Gaussian index of each
 * pixel's dominant entry (-1: none).
 *   nu_num: device double [N]; nu_cnt: device uint32 [N].                     */
gs_status gs_nu_accumulate(const gs_projected *proj, const gs_tiles *tiles, int n_frames,
                           const gs_camera *cams, const float *obs_depth, const gs_image *fwd,
                           double *nu_num, uint32_t *nu_cnt, int32_t *dominant,
                           const int32_t *status, gs_stream stream);

/* Eq. 13 finish and the tau rule of Sec. 3.2. For each of the n Gaussians with
 * nu_cnt > 0: nu = nu_num / nu_cnt (FP64, stored as FP32); the others keep nu.
 * If tau > 0 and opacity_logit is not NULL, every Gaussian whose FP64 nu
 * exceeds tau gets opacity_logit = min(opacity_logit, low_opacity_logit) (the
 * paper lowers uncertain primitives to a low opacity instead of deleting them)
 * and, if n_over is not NULL, is counted into *n_over (device uint32, added). */
gs_status gs_nu_finalize(int n, const double *nu_num, const uint32_t *nu_cnt, float *nu, float tau,
                         float low_opacity_logit, float *opacity_logit, uint32_t *n_over,
                         const int32_t *status, gs_stream stream);

/* Deterministic pose-gradient reduction (Sec. 3.4): pose_grad[f][k] =
 * sum_j partials[f][j][k], summed as double-floats (FP32 hi/lo pairs with
 * TwoSum compensation, ~48-bit precision; B300 runs FP64 at a small fraction
 * of its FP32 rate) in a fixed order, the final value in FP64; bit-identical
 * across runs. partials: float [n_frames][per_frame][6][2]; pose_grad: device
 * double [n_frames][6], (rho, phi) of the left perturbation Exp(xi) T_cw.    */
gs_status gs_pose_grad_reduce(const float *partials, int n_frames, int per_frame,
                              double *pose_grad, const int32_t *status, gs_stream stream);

/* One Adam step per frame on the pose in the {so(3) | T} form of Sec. 3.4:
 * g_t = g_rho, g_R = g_phi - t x g_rho; moments m, v in FP64;
 * d = -lr * mhat / (sqrt(vhat) + eps) (bias corrections from beta^t kept in the
 * state; d evaluated in FP32); R <- Exp(d_R) R, t <- t + d_t in FP64. The state
 * (GS_POSE_STATE_DOUBLES per frame: R[9], t[3], m[6], v[6], step, beta1^step,
 * beta2^step, unused; start with m = v = step = 0 and beta powers = 1) is
 * updated in place and T_cw (float [F][3][4]) rewritten for the next
 * gs_project.                                                                */
gs_status gs_pose_adam_step(double *state, const double *pose_grad, float *T_cw, int n_frames,
                            const gs_adam *adam, const int32_t *status, gs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H_ */
