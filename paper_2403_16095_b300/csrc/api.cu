// C ABI entry points of libgs (declared in include/gs.h): argument checks,
// frame tables and kernel launches. Nothing here allocates memory or
// synchronises with the host.
#include <atomic>
#include <climits>
#include <cstdarg>
#include <cstdio>

#include "gs_internal.cuh"

namespace {

thread_local char g_msg[512] = "";

gs_status fail(gs_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

gs_status cuda_status(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return GS_OK;
    return fail(GS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Builds the per-frame table; returns GS_OK or an argument error.
gs_status make_frames(int n_frames, const gs_camera *cams, int tile, gs::FrameTable &ft) {
    if (n_frames < 1 || n_frames > GS_MAX_FRAMES) return fail(GS_ERR_INVALID_ARG, "n_frames=%d outside [1,%d]", n_frames, GS_MAX_FRAMES);
    if (!cams) return fail(GS_ERR_INVALID_ARG, "cams is NULL");
    if (tile != 8 && tile != 16 && tile != 32) return fail(GS_ERR_INVALID_ARG, "tile=%d not in {8,16,32}", tile);
    ft.n = n_frames;
    ft.tile = tile;
    long long tiles = 0, pix = 0;
    for (int f = 0; f < n_frames; ++f) {
        const gs_camera &c = cams[f];
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
            return fail(GS_ERR_INVALID_ARG, "frame %d: image %dx%d outside 1..16384", f, c.width, c.height);
        if (!(c.fx > 0.f) || !(c.fy > 0.f) || !(c.znear > 0.f))
            return fail(GS_ERR_INVALID_ARG, "frame %d: fx, fy and znear must be > 0", f);
        gs::FrameDesc &d = ft.f[f];
        d.W = c.width;
        d.H = c.height;
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.znear = c.znear;
        d.tiles_x = (c.width + tile - 1) / tile;
        d.tiles_y = (c.height + tile - 1) / tile;
        d.tile_off = (int)tiles;
        d.pix_off = (int)pix;
        tiles += (long long)d.tiles_x * d.tiles_y;
        pix += (long long)c.width * c.height;
        if (tiles > INT_MAX / 2 || pix > INT_MAX / 4) return fail(GS_ERR_INVALID_ARG, "frames too large");
    }
    ft.total_tiles = (int)tiles;
    ft.total_pix = (int)pix;
    return GS_OK;
}

gs_status check_opts(const gs_opts *o) {
    if (!o) return fail(GS_ERR_INVALID_ARG, "opts is NULL");
    if (o->mode != GS_MODE_FWD && o->mode != GS_MODE_POSE && o->mode != GS_MODE_FULL)
        return fail(GS_ERR_INVALID_ARG, "mode=%d unknown", o->mode);
    if (o->batch != 0 && o->batch != 256 && o->batch != 512)
        return fail(GS_ERR_INVALID_ARG, "batch=%d not in {0, 256, 512}", o->batch);
    if (o->sched != GS_SCHED_TILE && o->sched != GS_SCHED_PERSISTENT)
        return fail(GS_ERR_INVALID_ARG, "sched=%d unknown", o->sched);
    return GS_OK;
}

// The work queue of a persistent launch (NULL: one CTA per tile).
gs_status sched_queue(const gs_opts *o, const gs_tiles *t, unsigned **queue) {
    *queue = nullptr;
    if (o->sched != GS_SCHED_PERSISTENT) return GS_OK;
    if (!t->queue || !aligned(t->queue, 4))
        return fail(GS_ERR_INVALID_ARG, "GS_SCHED_PERSISTENT needs tiles.queue (2 x uint32, zero-filled once)");
    *queue = t->queue;
    return GS_OK;
}

// need_touched: the call reads (or writes) tiles_touched; the blend calls read
// only rec, and for them tiles_touched may be NULL
gs_status check_proj(const gs_projected *p, int n_frames, bool need_touched = true) {
    if (!p) return fail(GS_ERR_INVALID_ARG, "projected is NULL");
    if (p->n_gaussians < 0) return fail(GS_ERR_INVALID_ARG, "n_gaussians < 0");
    if (p->n_frames != n_frames) return fail(GS_ERR_INVALID_ARG, "projected.n_frames=%d != n_frames=%d", p->n_frames, n_frames);
    if ((long long)p->n_gaussians * n_frames > (long long)INT_MAX) return fail(GS_ERR_INVALID_ARG, "records exceed 2^31-1");
    if (p->n_gaussians > 0 && !p->rec) return fail(GS_ERR_INVALID_ARG, "rec NULL");
    if (p->n_gaussians > 0 && need_touched && !p->tiles_touched) return fail(GS_ERR_INVALID_ARG, "tiles_touched NULL");
    if (!aligned(p->rec, 16)) return fail(GS_ERR_INVALID_ARG, "rec must be 16-byte aligned");
    return GS_OK;
}

gs::GaussPtrs gauss_ptrs(const gs_gaussians *g) {
    return gs::GaussPtrs{g->means, g->log_scales, g->quats, g->opacity_logit, g->colors, g->nu};
}

gs_status check_gauss(const gs_gaussians *g) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0) return fail(GS_ERR_INVALID_ARG, "n < 0");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logit || !g->colors || !g->nu))
        return fail(GS_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
    if (!aligned(g->quats, 16)) return fail(GS_ERR_INVALID_ARG, "quats must be 16-byte aligned");
    return GS_OK;
}

gs_status check_tiles(const gs_tiles *t, const gs::FrameTable &ft) {
    if (!t) return fail(GS_ERR_INVALID_ARG, "tiles is NULL");
    if (t->capacity < 1) return fail(GS_ERR_INVALID_ARG, "tiles.capacity must be >= 1");
    if (!t->values || !t->ranges) return fail(GS_ERR_INVALID_ARG, "tiles.values/ranges NULL");
    if (t->n_tiles != ft.total_tiles) return fail(GS_ERR_INVALID_ARG, "tiles.n_tiles=%d but the frames have %d tiles", t->n_tiles, ft.total_tiles);
    if (!aligned(t->ranges, 8)) return fail(GS_ERR_INVALID_ARG, "tiles.ranges must be 8-byte aligned");
    return GS_OK;
}

#define GS_TRY(expr)                           \
    do {                                       \
        const gs_status st__ = (expr);         \
        if (st__ != GS_OK) return st__;        \
    } while (0)

// Backward workspace: [FULL: per-record 2D gradient accumulators][per-frame
// arrival counters of the fused pose reduction, GS_MAX_FRAMES x uint32]. The
// counters are zero before the first call (the caller zero-fills ws once) and
// every launch leaves them zero: each wraps back to 0 at its last arrival.
constexpr size_t kAlign = 256;
size_t grad2d_bytes(int n_records, int mode) {
    if (mode != GS_MODE_FULL) return 0;
    return (((size_t)n_records * gs::kGrad2d * sizeof(float)) + kAlign - 1) / kAlign * kAlign;
}
size_t bwd_ws_bytes(int n_records, int mode) { return grad2d_bytes(n_records, mode) + kAlign; }

}  // namespace

namespace gs {
void set_error_message(const char *msg) { snprintf(g_msg, sizeof(g_msg), "%s", msg); }

int device_sm_count() {
    // one slot per device ordinal; 0 = not read yet. A host attribute query,
    // allowed while a stream is being captured.
    static std::atomic<int> cache[64];
    int dev = 0;
    // (148, the B300 count, only if the query itself fails)
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
    if (dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 148;
    if (dev < 64) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}
}  // namespace gs

extern "C" {

int gs_abi_version(void) { return GS_ABI_VERSION; }

const char *gs_last_error(void) { return g_msg; }

gs_status gs_project(const gs_gaussians *g, int n_frames, const gs_camera *cams, const float *T_cw,
                     const gs_opts *opts, gs_projected *out, const int32_t *status, gs_stream stream) {
    GS_TRY(check_gauss(g));
    GS_TRY(check_opts(opts));
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, opts->tile, ft));
    GS_TRY(check_proj(out, n_frames));
    if (out->n_gaussians != g->n) return fail(GS_ERR_INVALID_ARG, "projected.n_gaussians != gaussians.n");
    if (!T_cw || !status) return fail(GS_ERR_INVALID_ARG, "T_cw/status NULL");
    if (opts->mode == GS_MODE_POSE && g->n > 0 && n_frames > 0 && (!out->pose_jac || !aligned(out->pose_jac, 16)))
        return fail(GS_ERR_INVALID_ARG, "POSE mode needs a 16-byte aligned pose_jac");
    return cuda_status(gs::launch_project(gauss_ptrs(g), g->n, ft, T_cw, opts->jclamp, opts->nu_cull, opts->mode,
                                          out->rec, out->tiles_touched, out->pose_jac, gs::TileCtr{nullptr, 0}, status, stream),
                       "gs_project");
}

gs_status gs_project_bf16(const gs_gaussians_bf16 *g, int n_frames, const gs_camera *cams, const float *T_cw,
                          const gs_opts *opts, gs_projected *out, const int32_t *status, gs_stream stream) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0) return fail(GS_ERR_INVALID_ARG, "n < 0");
    if (g->n > 0 && (!g->anchors || !g->packed)) return fail(GS_ERR_INVALID_ARG, "anchors/packed NULL");
    if (!aligned(g->anchors, 16) || !aligned(g->packed, 16)) return fail(GS_ERR_INVALID_ARG, "anchors/packed must be 16-byte aligned");
    GS_TRY(check_opts(opts));
    if (opts->mode == GS_MODE_FULL) return fail(GS_ERR_UNSUPPORTED, "FULL mode needs FP32 parameters (gs_project)");
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, opts->tile, ft));
    GS_TRY(check_proj(out, n_frames));
    if (out->n_gaussians != g->n) return fail(GS_ERR_INVALID_ARG, "projected.n_gaussians != gaussians.n");
    if (!T_cw || !status) return fail(GS_ERR_INVALID_ARG, "T_cw/status NULL");
    if (opts->mode == GS_MODE_POSE && g->n > 0 && n_frames > 0 && (!out->pose_jac || !aligned(out->pose_jac, 16)))
        return fail(GS_ERR_INVALID_ARG, "POSE mode needs a 16-byte aligned pose_jac");
    return cuda_status(gs::launch_project_bf16(g->anchors, g->packed, g->n, ft, T_cw, opts->jclamp, opts->nu_cull,
                                               opts->mode, out->rec, out->tiles_touched, out->pose_jac, gs::TileCtr{nullptr, 0}, status,
                                               stream),
                       "gs_project_bf16");
}

size_t gs_spatial_order_workspace_size(int n) { return n < 0 ? 0 : gs::spatial_order_workspace_bytes(n); }

gs_status gs_spatial_order(const float *means, int n, uint32_t *perm, void *ws, size_t ws_bytes,
                           const int32_t *status, gs_stream stream) {
    if (n < 0) return fail(GS_ERR_INVALID_ARG, "n < 0");
    if (!status) return fail(GS_ERR_INVALID_ARG, "status NULL");
    if (n > 0 && (!means || !perm)) return fail(GS_ERR_INVALID_ARG, "means/perm NULL");
    const size_t need = gs::spatial_order_workspace_bytes(n);
    if (n > 0 && (!ws || ws_bytes < need)) return fail(GS_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (!aligned(ws, 256)) return fail(GS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return cuda_status(gs::launch_spatial_order(means, n, perm, ws, status, stream), "gs_spatial_order");
}

gs_status gs_pack_bf16(const gs_gaussians *src, const uint32_t *perm, float *anchors, uint16_t *packed,
                       const int32_t *status, gs_stream stream) {
    GS_TRY(check_gauss(src));
    if (!status) return fail(GS_ERR_INVALID_ARG, "status NULL");
    if (src->n > 0 && (!anchors || !packed)) return fail(GS_ERR_INVALID_ARG, "anchors/packed NULL");
    if (!aligned(anchors, 16) || !aligned(packed, 16)) return fail(GS_ERR_INVALID_ARG, "anchors/packed must be 16-byte aligned");
    return cuda_status(gs::launch_pack_bf16(gauss_ptrs(src), src->n, perm, anchors, packed, status, stream),
                       "gs_pack_bf16");
}

size_t gs_bin_tiles_workspace_size(int n_records, int capacity) {
    if (n_records < 0 || capacity < 1) return 0;
    return gs::bin_workspace_bytes(n_records, capacity);
}

gs_status gs_bin_tiles(const gs_projected *proj, int n_frames, const gs_camera *cams, const gs_opts *opts,
                       gs_tiles *tiles, int32_t *status, void *ws, size_t ws_bytes, gs_stream stream) {
    GS_TRY(check_opts(opts));
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, opts->tile, ft));
    GS_TRY(check_proj(proj, n_frames));
    GS_TRY(check_tiles(tiles, ft));
    if (!status) return fail(GS_ERR_INVALID_ARG, "status NULL");
    const int M = proj->n_gaussians * n_frames;
    const size_t need = gs::bin_workspace_bytes(M, tiles->capacity);
    if (!ws || ws_bytes < need) return fail(GS_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (!aligned(ws, 256)) return fail(GS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const int npf = proj->n_gaussians > 0 ? proj->n_gaussians : 1;
    return cuda_status(gs::launch_bin_tiles(proj->rec, proj->tiles_touched, M, npf, ft, tiles->capacity, tiles->values,
                                            tiles->keys, tiles->ranges, tiles->order, status, ws, stream),
                       "gs_bin_tiles");
}

// gs_project (or gs_project_bf16) followed by gs_bin_tiles in one call, with
// the pair count done by the projection kernel: clear, project + count, scan,
// fill, sort. The arguments are those of the two calls; validated the same way.
namespace {
gs_status check_bin_call(const gs_projected *out, int n_frames, const gs::FrameTable &ft, const gs_tiles *tiles,
                         const int32_t *status, const void *ws, size_t ws_bytes) {
    GS_TRY(check_tiles(tiles, ft));
    if (!status) return fail(GS_ERR_INVALID_ARG, "status NULL");
    const size_t need = gs::bin_workspace_bytes(out->n_gaussians * n_frames, tiles->capacity);
    if (!ws || ws_bytes < need) return fail(GS_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (!aligned(ws, 256)) return fail(GS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return GS_OK;
}

gs_status bin_after_counting_projection(const gs_projected *out, int n_frames, const gs::FrameTable &ft,
                                        gs_tiles *tiles, int32_t *status, void *ws, gs_stream stream) {
    const int npf = out->n_gaussians > 0 ? out->n_gaussians : 1;
    return cuda_status(gs::launch_bin_tiles(out->rec, out->tiles_touched, out->n_gaussians * n_frames, npf, ft,
                                            tiles->capacity, tiles->values, tiles->keys, tiles->ranges, tiles->order,
                                            status, ws, stream, true),
                       "gs_project_bin (binning)");
}
}  // namespace

gs_status gs_project_bin(const gs_gaussians *g, int n_frames, const gs_camera *cams, const float *T_cw,
                         const gs_opts *opts, gs_projected *out, gs_tiles *tiles, int32_t *status, void *ws,
                         size_t ws_bytes, gs_stream stream) {
    GS_TRY(check_gauss(g));
    GS_TRY(check_opts(opts));
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, opts->tile, ft));
    GS_TRY(check_proj(out, n_frames));
    if (out->n_gaussians != g->n) return fail(GS_ERR_INVALID_ARG, "projected.n_gaussians != gaussians.n");
    if (!T_cw) return fail(GS_ERR_INVALID_ARG, "T_cw NULL");
    if (opts->mode == GS_MODE_POSE && g->n > 0 && n_frames > 0 && (!out->pose_jac || !aligned(out->pose_jac, 16)))
        return fail(GS_ERR_INVALID_ARG, "POSE mode needs a 16-byte aligned pose_jac");
    GS_TRY(check_bin_call(out, n_frames, ft, tiles, status, ws, ws_bytes));
    GS_TRY(cuda_status(gs::launch_bin_clear(tiles->ranges, ft, tiles->capacity, ws, stream), "gs_project_bin (clear)"));
    GS_TRY(cuda_status(gs::launch_project(gauss_ptrs(g), g->n, ft, T_cw, opts->jclamp, opts->nu_cull, opts->mode,
                                          out->rec, out->tiles_touched, out->pose_jac,
                                          gs::tile_counters(tiles->ranges, ft, tiles->capacity, ws), status, stream),
                       "gs_project_bin (projection)"));
    return bin_after_counting_projection(out, n_frames, ft, tiles, status, ws, stream);
}

gs_status gs_project_bin_bf16(const gs_gaussians_bf16 *g, int n_frames, const gs_camera *cams, const float *T_cw,
                              const gs_opts *opts, gs_projected *out, gs_tiles *tiles, int32_t *status, void *ws,
                              size_t ws_bytes, gs_stream stream) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0) return fail(GS_ERR_INVALID_ARG, "n < 0");
    if (g->n > 0 && (!g->anchors || !g->packed)) return fail(GS_ERR_INVALID_ARG, "anchors/packed NULL");
    if (!aligned(g->anchors, 16) || !aligned(g->packed, 16)) return fail(GS_ERR_INVALID_ARG, "anchors/packed must be 16-byte aligned");
    GS_TRY(check_opts(opts));
    if (opts->mode == GS_MODE_FULL) return fail(GS_ERR_UNSUPPORTED, "FULL mode needs FP32 parameters (gs_project_bin)");
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, opts->tile, ft));
    GS_TRY(check_proj(out, n_frames));
    if (out->n_gaussians != g->n) return fail(GS_ERR_INVALID_ARG, "projected.n_gaussians != gaussians.n");
    if (!T_cw) return fail(GS_ERR_INVALID_ARG, "T_cw NULL");
    if (opts->mode == GS_MODE_POSE && g->n > 0 && n_frames > 0 && (!out->pose_jac || !aligned(out->pose_jac, 16)))
        return fail(GS_ERR_INVALID_ARG, "POSE mode needs a 16-byte aligned pose_jac");
    GS_TRY(check_bin_call(out, n_frames, ft, tiles, status, ws, ws_bytes));
    GS_TRY(cuda_status(gs::launch_bin_clear(tiles->ranges, ft, tiles->capacity, ws, stream),
                       "gs_project_bin_bf16 (clear)"));
    GS_TRY(cuda_status(gs::launch_project_bf16(g->anchors, g->packed, g->n, ft, T_cw, opts->jclamp, opts->nu_cull,
                                               opts->mode, out->rec, out->tiles_touched, out->pose_jac,
                                               gs::tile_counters(tiles->ranges, ft, tiles->capacity, ws), status,
                                               stream),
                       "gs_project_bin_bf16 (projection)"));
    return bin_after_counting_projection(out, n_frames, ft, tiles, status, ws, stream);
}

gs_status gs_render_fwd(const gs_projected *proj, const gs_tiles *tiles, int n_frames, const gs_camera *cams,
                        const float *obs_depth, const gs_opts *opts, gs_image *out, const int32_t *status,
                        gs_stream stream) {
    GS_TRY(check_opts(opts));
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, opts->tile, ft));
    GS_TRY(check_proj(proj, n_frames, false));
    GS_TRY(check_tiles(tiles, ft));
    if (!out || !out->color || !out->T_final || !out->n_last) return fail(GS_ERR_INVALID_ARG, "image color/T_final/n_last required");
    if (!status) return fail(GS_ERR_INVALID_ARG, "status NULL");
    if ((out->dom_pos == nullptr) != (out->dom_weight == nullptr))
        return fail(GS_ERR_INVALID_ARG, "dom_pos and dom_weight go together");
    gs::ImagePtrs ip{out->color, out->depth, out->alpha, out->unc, out->nu_map, out->median, out->T_final, out->n_last,
                     out->n_contrib, out->median_pos, out->dom_pos, out->dom_weight};
    unsigned *queue = nullptr;
    GS_TRY(sched_queue(opts, tiles, &queue));
    return cuda_status(gs::launch_render_fwd(proj->rec, tiles->values, tiles->ranges, tiles->order, ft, obs_depth, ip,
                                             status, opts->batch, queue, stream),
                       "gs_render_fwd");
}

int gs_pose_partials_per_frame(int mode, int n_gaussians, int n_frames, const gs_camera *cams, int tile) {
    if (mode == GS_MODE_FULL) return n_gaussians > 0 ? (n_gaussians + 255) / 256 : 1;
    if (!cams || n_frames < 1 || (tile != 8 && tile != 16 && tile != 32)) return 0;
    int mx = 1;
    for (int f = 0; f < n_frames; ++f) {
        const int t = ((cams[f].width + tile - 1) / tile) * ((cams[f].height + tile - 1) / tile);
        if (t > mx) mx = t;
    }
    return mx;
}

size_t gs_render_bwd_workspace_size(int n_records, int mode) { return bwd_ws_bytes(n_records, mode); }

gs_status gs_render_bwd(const gs_projected *proj, const gs_tiles *tiles, int n_frames, const gs_camera *cams,
                        const float *T_cw, const gs_gaussians *g, const float *obs_depth, const gs_image *fwd,
                        const gs_image_grad *dL, const gs_loss *loss, const gs_opts *opts, gs_grads *grads,
                        float *pose_partials, double *pose_grad, const int32_t *status, void *ws, size_t ws_bytes,
                        gs_stream stream) {
    GS_TRY(check_opts(opts));
    const int mode = opts->mode;
    if (mode != GS_MODE_POSE && mode != GS_MODE_FULL) return fail(GS_ERR_INVALID_ARG, "backward needs POSE or FULL mode");
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, opts->tile, ft));
    GS_TRY(check_proj(proj, n_frames, opts->mode == GS_MODE_FULL));
    GS_TRY(check_tiles(tiles, ft));
    if (!status || !pose_partials) return fail(GS_ERR_INVALID_ARG, "status/pose_partials NULL");
    if (!fwd || !fwd->T_final || !fwd->n_last) return fail(GS_ERR_INVALID_ARG, "forward T_final/n_last required");
    gs::LossParams lp{};
    if (loss) {
        lp.fused = 1;
        lp.w_color = loss->w_color; lp.w_depth = loss->w_depth; lp.w_unc = loss->w_unc;
        lp.w_nu = loss->w_nu; lp.unc_tau = loss->unc_tau; lp.w_align = loss->w_align;
        lp.target_color = loss->target_color; lp.target_depth = loss->target_depth;
        if (lp.w_color != 0.f && (!fwd->color || !lp.target_color)) return fail(GS_ERR_INVALID_ARG, "colour loss needs fwd.color and target_color");
        if (lp.w_depth != 0.f && (!fwd->depth || !lp.target_depth)) return fail(GS_ERR_INVALID_ARG, "depth loss needs fwd.depth and target_depth");
        if (lp.w_unc != 0.f && (!fwd->unc || !obs_depth)) return fail(GS_ERR_INVALID_ARG, "|U| loss needs fwd.unc and obs_depth");
        if (lp.unc_tau > 0.f && !fwd->nu_map) return fail(GS_ERR_INVALID_ARG, "unc_tau weighting needs fwd.nu_map");
        if (lp.w_align != 0.f && (!fwd->depth || !fwd->median || !fwd->median_pos))
            return fail(GS_ERR_INVALID_ARG, "L_align needs fwd.depth, fwd.median and fwd.median_pos");
    } else if (dL) {
        lp.g_color = dL->color; lp.g_depth = dL->depth; lp.g_alpha = dL->alpha; lp.g_unc = dL->unc; lp.g_nu = dL->nu_map;
        lp.g_median = dL->median;
        if (lp.g_unc && !obs_depth) return fail(GS_ERR_INVALID_ARG, "a gradient on U needs obs_depth");
        if (lp.g_median && !fwd->median_pos) return fail(GS_ERR_INVALID_ARG, "a median-depth gradient needs fwd.median_pos");
    } else {
        return fail(GS_ERR_INVALID_ARG, "either dL or loss is required");
    }
    gs::ImagePtrs ip{fwd->color, fwd->depth, fwd->alpha, fwd->unc, fwd->nu_map, fwd->median, fwd->T_final, fwd->n_last,
                     fwd->n_contrib, fwd->median_pos, nullptr, nullptr};
    const int N = proj->n_gaussians;
    const int M = N * n_frames;
    const int per_frame = gs_pose_partials_per_frame(mode, N, n_frames, cams, opts->tile);
    const size_t need = bwd_ws_bytes(M, mode);
    if (!ws || ws_bytes < need || !aligned(ws, 256))
        return fail(GS_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed (256-aligned)", ws_bytes, need);
    unsigned *counters = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + grad2d_bytes(M, mode));
    cudaError_t e;
    if (mode == GS_MODE_POSE) {
        if (!proj->pose_jac && proj->n_gaussians > 0) return fail(GS_ERR_INVALID_ARG, "POSE mode needs projected.pose_jac");
        for (int f = 0; f < n_frames; ++f) {
            const int used = ft.f[f].tiles_x * ft.f[f].tiles_y;
            if (used < per_frame) {
                e = cudaMemsetAsync(pose_partials + ((size_t)f * per_frame + used) * 12, 0,
                                    sizeof(float) * 12 * (size_t)(per_frame - used), stream);
                if (e != cudaSuccess) return cuda_status(e, "gs_render_bwd memset");
            }
        }
        return cuda_status(gs::launch_render_bwd(mode, proj->rec, proj->pose_jac, tiles->values, tiles->ranges,
                                                 tiles->order, ft,
                                                 obs_depth, ip, lp, nullptr, pose_partials, per_frame, pose_grad,
                                                 counters, status, opts->batch, nullptr, stream),
                           "gs_render_bwd");
    }
    GS_TRY(check_gauss(g));
    if (g->n != N) return fail(GS_ERR_INVALID_ARG, "gaussians.n != projected.n_gaussians");
    if (!T_cw || !grads) return fail(GS_ERR_INVALID_ARG, "FULL mode needs T_cw and grads");
    float *grad2d = static_cast<float *>(ws);
    if ((e = cudaMemsetAsync(grad2d, 0, sizeof(float) * gs::kGrad2d * (size_t)M, stream)) != cudaSuccess)
        return cuda_status(e, "gs_render_bwd memset");
    unsigned *queue = nullptr;
    GS_TRY(sched_queue(opts, tiles, &queue));
    if ((e = gs::launch_render_bwd(mode, proj->rec, nullptr, tiles->values, tiles->ranges, tiles->order, ft, obs_depth,
                                   ip, lp, grad2d, pose_partials, per_frame, nullptr, nullptr, status, opts->batch,
                                   queue, stream)) != cudaSuccess)
        return cuda_status(e, "gs_render_bwd");
    return cuda_status(gs::launch_project_bwd(gauss_ptrs(g), N, ft, T_cw, opts->jclamp, proj->tiles_touched, grad2d, *grads,
                                              pose_partials, per_frame, pose_grad, counters, status, stream),
                       "gs_render_bwd (projection adjoint)");
}

gs_status gs_render_fwd_bwd_pose(const gs_projected *proj, const gs_tiles *tiles, int n_frames, const gs_camera *cams,
                                 const gs_loss *loss, const gs_opts *opts, gs_image *out, float *pose_partials,
                                 double *pose_grad, double *adam_state, const gs_adam *adam, float *T_cw,
                                 const int32_t *status, void *ws, size_t ws_bytes, gs_stream stream) {
    GS_TRY(check_opts(opts));
    if (opts->mode != GS_MODE_POSE) return fail(GS_ERR_INVALID_ARG, "the tracking pass needs POSE mode");
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, opts->tile, ft));
    GS_TRY(check_proj(proj, n_frames, false));
    GS_TRY(check_tiles(tiles, ft));
    if (!status || !pose_partials) return fail(GS_ERR_INVALID_ARG, "status/pose_partials NULL");
    if (!proj->pose_jac && proj->n_gaussians > 0) return fail(GS_ERR_INVALID_ARG, "POSE mode needs projected.pose_jac");
    if (!loss) return fail(GS_ERR_INVALID_ARG, "loss is NULL");
    if (loss->w_unc != 0.f || loss->w_nu != 0.f || loss->w_align != 0.f)
        return fail(GS_ERR_UNSUPPORTED, "the tracking pass supports colour and depth L1 terms only");
    if (adam_state && (!pose_grad || !adam || !T_cw))
        return fail(GS_ERR_INVALID_ARG, "the pose update needs pose_grad, adam and T_cw");
    gs::LossParams lp{};
    lp.fused = 1;
    lp.w_color = loss->w_color; lp.w_depth = loss->w_depth; lp.unc_tau = loss->unc_tau;
    lp.target_color = loss->target_color; lp.target_depth = loss->target_depth;
    if (lp.w_color != 0.f && !lp.target_color) return fail(GS_ERR_INVALID_ARG, "colour loss needs target_color");
    if (lp.w_depth != 0.f && !lp.target_depth) return fail(GS_ERR_INVALID_ARG, "depth loss needs target_depth");
    gs::ImagePtrs ip{};
    if (out) {
        ip.color = out->color; ip.depth = out->depth; ip.nu_map = out->nu_map;
        ip.T_final = out->T_final; ip.n_last = out->n_last;
    }
    const int N = proj->n_gaussians;
    const int M = N * n_frames;
    const int per_frame = gs_pose_partials_per_frame(GS_MODE_POSE, N, n_frames, cams, opts->tile);
    const size_t need = bwd_ws_bytes(M, GS_MODE_POSE);
    if (!ws || ws_bytes < need || !aligned(ws, 256))
        return fail(GS_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed (256-aligned)", ws_bytes, need);
    cudaError_t e;
    for (int f = 0; f < n_frames; ++f) {
        const int used = ft.f[f].tiles_x * ft.f[f].tiles_y;
        if (used < per_frame) {
            e = cudaMemsetAsync(pose_partials + ((size_t)f * per_frame + used) * 12, 0,
                                sizeof(float) * 12 * (size_t)(per_frame - used), stream);
            if (e != cudaSuccess) return cuda_status(e, "gs_render_fwd_bwd_pose memset");
        }
    }
    const gs_adam ad = adam ? *adam : gs_adam{};
    // the pass writes one pose partial per tile; the frame's fixed-order sum
    // (and the Adam step) follow as one small chained launch
    e = gs::launch_render_fused_pose(proj->rec, proj->pose_jac, tiles->values, tiles->ranges, tiles->order, ft, ip,
                                     lp, pose_partials, per_frame, status, stream);
    if (e != cudaSuccess || !pose_grad) return cuda_status(e, "gs_render_fwd_bwd_pose");
    return cuda_status(gs::launch_pose_reduce_adam(pose_partials, n_frames, per_frame, pose_grad, adam_state, ad, T_cw,
                                                   status, stream),
                       "gs_render_fwd_bwd_pose (pose reduction)");
}

gs_status gs_nu_accumulate(const gs_projected *proj, const gs_tiles *tiles, int n_frames, const gs_camera *cams,
                           const float *obs_depth, const gs_image *fwd, double *nu_num, uint32_t *nu_cnt,
                           int32_t *dominant, const int32_t *status, gs_stream stream) {
    gs::FrameTable ft;
    GS_TRY(make_frames(n_frames, cams, 16, ft));
    GS_TRY(check_proj(proj, n_frames, false));
    if (!tiles || !tiles->values) return fail(GS_ERR_INVALID_ARG, "tiles.values NULL");
    if (!fwd || !fwd->dom_pos || !fwd->dom_weight)
        return fail(GS_ERR_INVALID_ARG, "fwd.dom_pos and fwd.dom_weight (from gs_render_fwd) required");
    if (!obs_depth) return fail(GS_ERR_INVALID_ARG, "obs_depth (sensor depth D of Eq. 13) required");
    if (!nu_num || !nu_cnt || !status) return fail(GS_ERR_INVALID_ARG, "nu_num/nu_cnt/status NULL");
    if (!aligned(nu_num, 8) || !aligned(nu_cnt, 4)) return fail(GS_ERR_INVALID_ARG, "nu_num/nu_cnt misaligned");
    return cuda_status(gs::launch_nu_accumulate(proj->rec, tiles->values, ft, proj->n_gaussians, obs_depth, fwd->dom_pos,
                                                fwd->dom_weight, nu_num, nu_cnt, dominant, status, stream),
                       "gs_nu_accumulate");
}

gs_status gs_nu_finalize(int n, const double *nu_num, const uint32_t *nu_cnt, float *nu, float tau,
                         float low_opacity_logit, float *opacity_logit, uint32_t *n_over, const int32_t *status,
                         gs_stream stream) {
    if (n < 0) return fail(GS_ERR_INVALID_ARG, "n < 0");
    if (!status) return fail(GS_ERR_INVALID_ARG, "status NULL");
    if (n > 0 && (!nu_num || !nu_cnt || !nu)) return fail(GS_ERR_INVALID_ARG, "nu_num/nu_cnt/nu NULL");
    if (!(tau == tau) || !(low_opacity_logit == low_opacity_logit)) return fail(GS_ERR_INVALID_ARG, "tau/low_opacity_logit NaN");
    return cuda_status(gs::launch_nu_finalize(n, nu_num, nu_cnt, nu, tau, low_opacity_logit, opacity_logit, n_over,
                                              status, stream),
                       "gs_nu_finalize");
}

gs_status gs_pose_grad_reduce(const float *partials, int n_frames, int per_frame, double *pose_grad,
                              const int32_t *status, gs_stream stream) {
    if (!partials || !pose_grad || !status) return fail(GS_ERR_INVALID_ARG, "NULL pointer");
    if (n_frames < 1 || n_frames > GS_MAX_FRAMES || per_frame < 1) return fail(GS_ERR_INVALID_ARG, "bad n_frames/per_frame");
    return cuda_status(gs::launch_pose_reduce(partials, n_frames, per_frame, pose_grad, status, stream),
                       "gs_pose_grad_reduce");
}

gs_status gs_pose_adam_step(double *state, const double *pose_grad, float *T_cw, int n_frames, const gs_adam *adam,
                            const int32_t *status, gs_stream stream) {
    if (!state || !pose_grad || !T_cw || !adam || !status) return fail(GS_ERR_INVALID_ARG, "NULL pointer");
    if (n_frames < 1 || n_frames > GS_MAX_FRAMES) return fail(GS_ERR_INVALID_ARG, "bad n_frames");
    return cuda_status(gs::launch_pose_adam(state, pose_grad, T_cw, n_frames, *adam, status, stream),
                       "gs_pose_adam_step");
}

}  // extern "C"
