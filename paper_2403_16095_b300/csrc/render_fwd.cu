// Front-to-back alpha blending of the depth-sorted tile lists (CG-SLAM Eq. 3-10).
//
// One CTA per tile (TILE x TILE pixels, one thread per pixel), or, in the
// persistent form, one resident CTA per slot of the GPU pulling tiles from a
// device work queue. Each warp owns an 8x4 pixel block so that the
// warp-uniform rectangle test against a Gaussian's pixel rect skips most
// non-overlapping list entries without divergence. The tile's list is staged
// in shared memory in batches (256 or 512 records at 16x16 and 32x32 tiles,
// the whole CTA's 64 at 8x8); a pixel stops when the next entry would take T
// below 1e-4, a warp skips a batch once all of its pixels are done, and the
// tile ends once every pixel is done.
//
// The per-pixel arithmetic (q, G, alpha, T) is the same function as in the
// backward pass, written with explicitly rounded operations, so both passes take
// identical accept/stop decisions and the result does not depend on TILE.
//
// The DOM variant also tracks each pixel's dominant entry (largest w = alpha T,
// the first on ties; Sec. 3.2) for the per-Gaussian uncertainty of Eq. 13; the
// LITE variant (taken when opacity, U, median and the contribution count are
// not requested, as in tracking) accumulates only colour, depth and the nu map.
// Separate instantiations, so each caller pays only for what it reads.
#include "gs_internal.cuh"
#include "blend_common.cuh"
#include "work_queue.cuh"

namespace gs {
namespace {

constexpr int kFwdBatch = 512;  // default entries staged per batch at 16x16 and larger tiles (512: half
                                // the CTA barriers of 256; mapping forward 1.20 -> 1.05 ms)

// The blend of one tile (one thread per pixel). The per-tile CTA kernel and the
// persistent kernel below run this same code, so their images are identical.
template <int TILE, bool DOM, bool LITE, int BATCH>
__device__ __forceinline__ void fwd_tile(const int gtile, const float4 *__restrict__ rec,
                                         const uint32_t *__restrict__ values, const uint2 *__restrict__ ranges,
                                         const FrameTable &ft, const float *__restrict__ obs_depth,
                                         const ImagePtrs &out, float4 *s_a, float4 *s_b, float4 *s_c, int4 *s_r) {
    constexpr int NT = TILE * TILE;
    const int f = frame_of_tile(ft, gtile);
    const FrameDesc &fd = ft.f[f];
    const int lt = gtile - fd.tile_off;
    const int tx = lt % fd.tiles_x, ty = lt / fd.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int WPR = TILE / 8;
    const int wx0 = tx * TILE + (warp % WPR) * 8, wy0 = ty * TILE + (warp / WPR) * 4;
    const int px = wx0 + (lane & 7), py = wy0 + (lane >> 3);
    const bool inside = px < fd.W && py < fd.H;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const size_t pix = (size_t)fd.pix_off + (size_t)py * fd.W + px;
    const uint2 range = ranges[gtile];
    const float Dp = (obs_depth != nullptr && inside) ? obs_depth[pix] : 0.f;

    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, dep = 0.f, opa = 0.f, unc = 0.f, nus = 0.f, med = 0.f;
    uint32_t last = range.x;
    int n_blend = 0;
    int med_pos = -1;  // tile-list position of the median entry
    float wmax = 0.f;  // DOM: largest blend weight so far and its position
    int dom_pos = -1;
    bool done = !inside;

    for (uint32_t base = range.x; base < range.y; base += BATCH) {
        if (__syncthreads_count(done) == NT) break;  // also orders smem reuse
        for (int e = tid; e < BATCH && base + e < range.y; e += NT) {
            const float4 *R = rec + (size_t)values[base + e] * 4;
            s_a[e] = R[0];
            s_b[e] = R[1];
            s_c[e] = R[2];
            s_r[e] = reinterpret_cast<const int4 *>(R)[3];
        }
        __syncthreads();
        const int cnt = min(BATCH, (int)(range.y - base));
        if (!__all_sync(0xffffffffu, done)) {
            for (int g0 = 0; g0 < cnt; g0 += 32) {
                // lane l tests entry g0 + l against this warp's pixel block
                const int kt = g0 + lane;
                const bool hit = kt < cnt && warp_block_may_hit(s_a[kt], s_b[kt], s_r[kt], wx0, wy0);
                unsigned mask = __ballot_sync(0xffffffffu, hit);
                while (mask) {  // surviving entries, front to back
                    const int k = g0 + __ffs(mask) - 1;
                    mask &= mask - 1;
                    const float4 a = s_a[k];
                    const float4 b = s_b[k];
                    const float4 c = s_c[k];  // loaded with a and b: off the blend's dependency chain
                    float dx, dy, G, sg, alpha;
                    // saturated lanes evaluate alpha too and discard it: no branch around the evaluation
                    if (!((!done) & eval_alpha(pxc, pyc, a, b, dx, dy, G, sg, alpha))) continue;
                    const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
                    if (Tn < kTMin) { done = true; continue; }
                    const float w = __fmul_rn(alpha, T);
                    c0 = fmaf(w, c.x, c0);
                    c1 = fmaf(w, c.y, c1);
                    c2 = fmaf(w, c.z, c2);
                    dep = fmaf(w, b.z, dep);
                    nus = fmaf(w, b.w, nus);
                    if (!LITE) {
                        opa = __fadd_rn(opa, w);
                        const float dz = __fsub_rn(b.z, Dp);
                        unc = fmaf(w, __fmul_rn(dz, dz), unc);
                        if (T >= 0.5f && Tn < 0.5f) {
                            med = b.z;
                            med_pos = (int)(base + k);
                        }
                        ++n_blend;
                    }
                    if (DOM && w > wmax) {
                        wmax = w;
                        dom_pos = (int)(base + k);
                    }
                    T = Tn;
                    last = base + k + 1;
                }
                if (__all_sync(0xffffffffu, done)) break;
            }
        }
    }
    if (!inside) return;
    const int HW = fd.W * fd.H;
    const size_t cbase = 3 * (size_t)fd.pix_off + (size_t)py * fd.W + px;
    out.color[cbase] = c0;
    out.color[cbase + HW] = c1;
    out.color[cbase + 2 * (size_t)HW] = c2;
    if (out.depth) out.depth[pix] = dep;
    if (out.nu_map) out.nu_map[pix] = nus;
    out.T_final[pix] = T;
    out.n_last[pix] = (int32_t)last;
    if (!LITE) {
        if (out.alpha) out.alpha[pix] = opa;
        if (out.unc && obs_depth) out.unc[pix] = unc;
        if (out.median) out.median[pix] = med;
        if (out.n_contrib) out.n_contrib[pix] = n_blend;
        if (out.median_pos) out.median_pos[pix] = med_pos;
    }
    if (DOM) {
        out.dom_pos[pix] = dom_pos;
        out.dom_weight[pix] = wmax;
    }
}

// One CTA per tile, heaviest tiles first when the launch order is given.
template <int TILE, bool DOM, bool LITE, int BATCH>
__global__ void __launch_bounds__(TILE *TILE, 1024 / (TILE * TILE))
    k_render_fwd(const float4 *__restrict__ rec, const uint32_t *__restrict__ values,
                 const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, FrameTable ft,
                 const float *__restrict__ obs_depth, ImagePtrs out, const int32_t *__restrict__ status) {
    __shared__ float4 s_a[BATCH], s_b[BATCH], s_c[BATCH];
    __shared__ int4 s_r[BATCH];
    if (status[0] != 0) return;
    const int gtile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    fwd_tile<TILE, DOM, LITE, BATCH>(gtile, rec, values, ranges, ft, obs_depth, out, s_a, s_b, s_c, s_r);
}

// Persistent form: as many CTAs as fit on the GPU at once, each pulling the
// next (frame, tile) item -- in launch order, heaviest first -- from a device
// counter until the batch is exhausted (work_queue.cuh).
template <int TILE, bool DOM, bool LITE, int BATCH>
__global__ void __launch_bounds__(TILE *TILE, 1024 / (TILE * TILE))
    k_render_fwd_persist(const float4 *__restrict__ rec, const uint32_t *__restrict__ values,
                         const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, FrameTable ft,
                         const float *__restrict__ obs_depth, ImagePtrs out, const int32_t *__restrict__ status,
                         unsigned *__restrict__ queue) {
    __shared__ float4 s_a[BATCH], s_b[BATCH], s_c[BATCH];
    __shared__ int4 s_r[BATCH];
    __shared__ int s_item[2];
    if (status[0] != 0) return;
    for (int it = 0;; ++it) {
        const int item = queue_next(queue, s_item, it);
        if (item >= ft.total_tiles) break;
        const int gtile = order ? (int)order[item] : item;
        fwd_tile<TILE, DOM, LITE, BATCH>(gtile, rec, values, ranges, ft, obs_depth, out, s_a, s_b, s_c, s_r);
    }
    queue_exit(queue);
}

template <int TILE, bool DOM, bool LITE, int BATCH>
cudaError_t launch_variant(const float4 *r4, const uint32_t *values, const uint2 *rg, const uint32_t *order,
                           const FrameTable &ft, const float *obs_depth, const ImagePtrs &out, const int32_t *status,
                           unsigned *queue, cudaStream_t s) {
    if (!queue) {
        k_render_fwd<TILE, DOM, LITE, BATCH><<<ft.total_tiles, TILE * TILE, 0, s>>>(r4, values, rg, order, ft,
                                                                                    obs_depth, out, status);
        return cudaGetLastError();
    }
    int grid = 0;
    cudaError_t e = persistent_grid<k_render_fwd_persist<TILE, DOM, LITE, BATCH>>(TILE * TILE, 0, ft.total_tiles,
                                                                                   &grid);
    if (e != cudaSuccess) return e;
    k_render_fwd_persist<TILE, DOM, LITE, BATCH><<<grid, TILE * TILE, 0, s>>>(r4, values, rg, order, ft, obs_depth,
                                                                              out, status, queue);
    return cudaGetLastError();
}

template <int TILE, int BATCH>
cudaError_t launch_batch(const float4 *r4, const uint32_t *values, const uint2 *rg, const uint32_t *order,
                         const FrameTable &ft, const float *obs_depth, const ImagePtrs &out, const int32_t *status,
                         unsigned *queue, cudaStream_t s) {
    const bool lite = !out.alpha && !out.unc && !out.median && !out.median_pos && !out.n_contrib;
    if (out.dom_pos)
        return launch_variant<TILE, true, false, BATCH>(r4, values, rg, order, ft, obs_depth, out, status, queue, s);
    if (lite)
        return launch_variant<TILE, false, true, BATCH>(r4, values, rg, order, ft, obs_depth, out, status, queue, s);
    return launch_variant<TILE, false, false, BATCH>(r4, values, rg, order, ft, obs_depth, out, status, queue, s);
}

template <int TILE>
cudaError_t launch_tile(const float4 *r4, const uint32_t *values, const uint2 *rg, const uint32_t *order,
                        const FrameTable &ft, const float *obs_depth, const ImagePtrs &out, const int32_t *status,
                        int batch, unsigned *queue, cudaStream_t s) {
    constexpr int NT = TILE * TILE;
    if (NT < 256)  // a batch is the whole CTA's worth of entries at 8x8
        return launch_batch<TILE, (NT < 256 ? NT : 256)>(r4, values, rg, order, ft, obs_depth, out, status, queue, s);
    if (batch == 256)
        return launch_batch<TILE, 256>(r4, values, rg, order, ft, obs_depth, out, status, queue, s);
    return launch_batch<TILE, kFwdBatch>(r4, values, rg, order, ft, obs_depth, out, status, queue, s);
}

}  // namespace

cudaError_t launch_render_fwd(const float *rec, const uint32_t *values, const uint32_t *ranges, const uint32_t *order,
                              const FrameTable &ft, const float *obs_depth, const ImagePtrs &out,
                              const int32_t *status, int batch, unsigned *queue, cudaStream_t s) {
    if (ft.total_tiles == 0) return cudaSuccess;
    const float4 *r4 = reinterpret_cast<const float4 *>(rec);
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
    switch (ft.tile) {
        case 8: return launch_tile<8>(r4, values, rg, order, ft, obs_depth, out, status, batch, queue, s);
        case 16: return launch_tile<16>(r4, values, rg, order, ft, obs_depth, out, status, batch, queue, s);
        case 32: return launch_tile<32>(r4, values, rg, order, ft, obs_depth, out, status, batch, queue, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gs
