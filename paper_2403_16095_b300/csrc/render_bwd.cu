// Adjoint of the front-to-back blend (CG-SLAM Eq. 3-10), walking each tile's
// depth-sorted list from the pixel's last blended entry back to the front.
//
// Per pixel the transmittance in front of entry j is recovered from the one
// behind it, T_j = T_{j+1} / (1 - alpha_j), starting from the stored T_final;
// nothing per entry is stored by the forward pass. With g the per-pixel
// gradient of the loss w.r.t. the blended channels f = (R, G, B, depth, opacity,
// U, nu) and GS_j = sum_{i > j} w_i <g, f_i> (one running scalar, since g does
// not depend on the entry):
//     dL/dalpha_j = T_j <g, f_j> - GS_j / (1 - alpha_j),
//     dL/dz_j     = w_j (g_depth + 2 g_U (z_j - D)),   dL/dc_j = w_j g_color,
//     dL/d(power) = alpha_j dL/dalpha_j  (0 when alpha is clamped at 0.99),
// and the power -q/2 gives the gradients of the 2D centre and the conic.
//
// POSE mode: each pixel contracts (d mean2d, d conic, dz) of every entry with
// that record's 6x6 pose Jacobian into six FP32 accumulators; at the end the
// tile reduces them in FP64 by warp shuffles and a fixed block tree into one
// partial per tile (deterministic, no atomics).
// FULL mode: the eleven per-entry gradients are reduced across the warp (only
// when some lane contributed) and lane 0 adds them to the record's accumulators;
// it also has a persistent form (resident CTAs pulling tiles from a device work
// queue) and a choice of 256 or 512 staged entries per batch.
#include <atomic>

#include "gs_internal.cuh"
#include "blend_common.cuh"
#include "dfloat.cuh"
#include "work_queue.cuh"

namespace gs {
namespace {

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

// Entries staged per batch and the dynamic shared memory that holds them:
// record (4 x 16 B) + index (4 B), plus the 144-B pose Jacobian in POSE mode.
// The last CTA of a frame reuses the same bytes for the pose reduction.
constexpr int kFullBatch = 512;

template <int TILE, int MODE, int FULL_BATCH = kFullBatch, bool PERSIST = false>
struct BwdSmem {
    static constexpr int NT = TILE * TILE;
    static constexpr bool POSE = MODE == GS_MODE_POSE;
    // FULL mode stages 512 entries per batch by default (68 B each): half the
    // CTA barriers of 256, which bound the kernel's warps (they wait for the
    // tile's busiest warp at every batch); 256 is the other choice offered
    static constexpr int BATCH = NT < 256 ? NT : (POSE ? 256 : FULL_BATCH);
    static constexpr size_t kEntry = 4 * sizeof(float4) + sizeof(uint32_t) + (POSE ? 9 * sizeof(float4) : 0);
    static constexpr size_t kStage = BATCH * kEntry;
    // per-tile FULL mode: each thread's rarely used loss terms (opacity, nu and
    // median gradients, median position), kept here instead of in registers;
    // at the 48-register cap of the 16x16 build this keeps the walk from
    // spilling. The persistent kernel keeps them in registers: with the slot
    // (4 KB more per CTA) its backward measured 8.1-8.8 against 5.5 ms on the
    // uneven batch.
    static constexpr size_t kLoss = (POSE || PERSIST) ? 0 : NT * sizeof(float4);
    static constexpr size_t kRed = POSE ? sizeof(df) * kRedSlots * 6 : 0;
    static constexpr size_t bytes = kStage + kLoss > kRed ? kStage + kLoss : kRed;
};

// FULL mode: an entry blended by at most kDirectLanes lanes of the warp is
// accumulated by each of those lanes with three 128-bit atomics; above that,
// by a warp reduction and one atomic per field. The reduction costs ~64
// instructions per entry whatever the lane count, while L2 absorbs the extra
// atomics until nearly every lane adds (measured on an 8-frame 640x480
// window: backward 2.59 ms with direct adds for a single lane only, 2.33 /
// 2.31 / 2.31 / 2.91 ms with thresholds 16 / 20 / 24 / 32).
constexpr int kDirectLanes = 20;

// CD: the loss touches only colour and depth (the tracking loss), so the
// opacity, U and nu terms of every contribution are compiled out.
template <int TILE>
struct BwdShared {  // the static shared state of a backward CTA
    static constexpr int NWARP = TILE * TILE / 32 > 0 ? TILE * TILE / 32 : 1;
    uint32_t wmax[NWARP];
    df wdf[NWARP][6];
    int flag;
    int item[2];  // persistent form: the work-queue slots
};

// The backward of one tile. The per-tile CTA kernel and the persistent kernel
// below run this same code, so their gradients agree up to the order of the
// FULL-mode atomic additions.
template <int TILE, int MODE, bool CD, int FULL_BATCH, bool PERSIST = false>
__device__ __forceinline__ void bwd_tile(const int gtile, const float4 *__restrict__ rec,
                                         const float4 *__restrict__ jac, const uint32_t *__restrict__ values,
                                         const uint2 *__restrict__ ranges, const FrameTable &ft,
                                         const float *__restrict__ obs_depth, const ImagePtrs &fwd,
                                         const LossParams &lp, float *__restrict__ grad2d,
                                         float *__restrict__ pose_partials, int per_frame,
                                         double *__restrict__ pose_grad, unsigned *__restrict__ counters,
                                         unsigned char *s_dyn, BwdShared<TILE> &sh) {
    using SM = BwdSmem<TILE, MODE, FULL_BATCH, PERSIST>;
    constexpr int NT = SM::NT;
    constexpr bool POSE = SM::POSE;
    constexpr int BATCH = SM::BATCH;
    constexpr int NWARP = NT / 32 > 0 ? NT / 32 : 1;
    float4 *s_a = reinterpret_cast<float4 *>(s_dyn);
    float4 *s_b = s_a + BATCH;
    float4 *s_c = s_b + BATCH;
    int4 *s_r = reinterpret_cast<int4 *>(s_c + BATCH);
    float4 *s_j = reinterpret_cast<float4 *>(s_r + BATCH);                   // POSE only
    uint32_t *s_idx = reinterpret_cast<uint32_t *>(s_j + (POSE ? 9 * BATCH : 0));
    float4 *s_gx = reinterpret_cast<float4 *>(s_dyn + SM::kStage);           // FULL only
    df(*s_red)[6] = reinterpret_cast<df(*)[6]>(s_dyn);                       // tail only
    uint32_t *s_wmax = sh.wmax;

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
    const int HW = fd.W * fd.H;
    const size_t cbase = 3 * (size_t)fd.pix_off + (size_t)py * fd.W + px;
    const uint2 range = ranges[gtile];

    // ---- per-pixel loss gradient w.r.t. the blended channels
    float gc0 = 0.f, gc1 = 0.f, gc2 = 0.f, gD = 0.f, gO = 0.f, gU = 0.f, gN = 0.f, gM = 0.f;
    float T = 1.f, Dp = 0.f;
    uint32_t my_last = range.x;
    int my_med = -1;  // tile-list position of the median entry (receives gM on its depth)
    if (inside) {
        T = fwd.T_final[pix];
        my_last = min(max((uint32_t)fwd.n_last[pix], range.x), range.y);  // stay inside this tile's list
        Dp = obs_depth ? obs_depth[pix] : 0.f;
        if (lp.fused) {
            const float inv_hw = 1.f / (float)HW;
            float m = 1.f;
            if (lp.unc_tau > 0.f) m = 1.f / (1.f + fwd.nu_map[pix] / lp.unc_tau);
            const float kc = inv_hw * m * lp.w_color, kd = inv_hw * m * lp.w_depth;
            if (lp.w_color != 0.f) {
                gc0 = kc * sgnf(fwd.color[cbase] - lp.target_color[cbase]);
                gc1 = kc * sgnf(fwd.color[cbase + HW] - lp.target_color[cbase + HW]);
                gc2 = kc * sgnf(fwd.color[cbase + 2 * (size_t)HW] - lp.target_color[cbase + 2 * (size_t)HW]);
            }
            if (lp.w_depth != 0.f) gD = kd * sgnf(fwd.depth[pix] - lp.target_depth[pix]);
            if (lp.w_unc != 0.f) gU = inv_hw * lp.w_unc * sgnf(fwd.unc[pix]);
            gN = inv_hw * lp.w_nu;
            if (lp.w_align != 0.f) {  // Eq. 12: |D_alpha - D_median|
                const float ga = inv_hw * lp.w_align * sgnf(fwd.depth[pix] - fwd.median[pix]);
                gD += ga;
                gM = -ga;
            }
        } else {
            if (lp.g_color) {
                gc0 = lp.g_color[cbase];
                gc1 = lp.g_color[cbase + HW];
                gc2 = lp.g_color[cbase + 2 * (size_t)HW];
            }
            if (lp.g_depth) gD = lp.g_depth[pix];
            if (lp.g_alpha) gO = lp.g_alpha[pix];
            if (lp.g_unc) gU = lp.g_unc[pix];
            if (lp.g_nu) gN = lp.g_nu[pix];
            if (lp.g_median) gM = lp.g_median[pix];
        }
        if (gM != 0.f) my_med = fwd.median_pos[pix];
    }
    constexpr bool kLossSmem = SM::kLoss > 0 && !CD;  // see BwdSmem
    if (kLossSmem) s_gx[tid] = make_float4(gO, gN, gM, __int_as_float(my_med));
    if (CD) {  // the launcher picked this variant because these are zero
        gO = 0.f;
        gU = 0.f;
        gN = 0.f;
        gM = 0.f;
        my_med = -1;
    }
    // ---- extent of the walk: block max and warp max of the last blended entry
    const uint32_t warp_last = __reduce_max_sync(0xffffffffu, my_last);
    if (lane == 0) s_wmax[warp] = warp_last;
    __syncthreads();
    uint32_t block_last = range.x;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) block_last = max(block_last, s_wmax[w]);

    float GS = 0.f;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

    for (int bend = (int)block_last; bend > (int)range.x; bend -= BATCH) {
        const int bstart = max((int)range.x, bend - BATCH);
        __syncthreads();
        for (int e = tid; e < bend - bstart; e += NT) {
            const uint32_t r = values[bstart + e];
            const float4 *R = rec + (size_t)r * 4;
            s_a[e] = R[0];
            s_b[e] = R[1];
            s_c[e] = R[2];
            s_r[e] = reinterpret_cast<const int4 *>(R)[3];
            s_idx[e] = r;
            if (POSE) {
                const float4 *J = jac + (size_t)r * 9;
#pragma unroll
                for (int q = 0; q < 9; ++q) s_j[e * 9 + q] = J[q];
            }
        }
        __syncthreads();
        const int cnt = bend - bstart;
        for (int g1 = cnt, g0 = max(0, cnt - 32); g1 > 0; g1 = g0, g0 = max(0, g0 - 32)) {
          // lane l tests entry g0 + l (before the warp's last blended entry) against its pixel block
          const int kt = g0 + lane;
          const bool hit = kt < g1 && (uint32_t)(bstart + kt) < warp_last &&
                           warp_block_may_hit(s_a[kt], s_b[kt], s_r[kt], wx0, wy0);
          unsigned mask = __ballot_sync(0xffffffffu, hit);
          while (mask) {  // surviving entries, back to front
            const int bit = 31 - __clz(mask);
            mask &= ~(1u << bit);
            const int k = g0 + bit;
            const int j = bstart + k;
            const float4 a = s_a[k];
            const float4 b = s_b[k];
            float dx = 0.f, dy = 0.f, G = 0.f, sg = 0.f, alpha = 0.f;
            bool act;
            if (!POSE && !CD) {  // one path for all lanes up to the act test (measured faster here)
                act = ((uint32_t)j < my_last) & eval_alpha(pxc, pyc, a, b, dx, dy, G, sg, alpha);
            } else {  // branching spills less in these builds
                act = (uint32_t)j < my_last;
                if (act) act = eval_alpha(pxc, pyc, a, b, dx, dy, G, sg, alpha);
            }
            float v[11];
            if (act && CD) {  // colour + depth only: the tracking pass's arithmetic, bit for bit
                float th[6], w, dal;
                entry_grad_cd(alpha, sg, dx, dy, a, b, s_c[k], gc0, gc1, gc2, gD, T, GS, th, w, dal);
                v[G_MX] = th[0];
                v[G_MY] = th[1];
                v[G_CA] = th[2];
                v[G_CB] = th[3];
                v[G_CC] = th[4];
                v[G_Z] = th[5];
                if (!POSE) {
                    v[G_OP] = sg >= kAlphaMax ? 0.f : dal * G;
                    v[G_NU] = 0.f;  // nu is not in this loss
                    v[G_R] = w * gc0;
                    v[G_G] = w * gc1;
                    v[G_B] = w * gc2;
                }
            } else if (act) {
                const float one_m = __fsub_rn(1.f, alpha);
                const float inv = __fdividef(1.f, one_m);
                T = T * inv;  // transmittance in front of entry j
                const float w = alpha * T;
                const float4 c = s_c[k];
                // (gO, gN, gM, median position): from shared memory in the per-tile FULL kernel
                const float4 gx = kLossSmem ? s_gx[tid] : make_float4(gO, gN, gM, __int_as_float(my_med));
                const float dz = b.z - Dp;
                const float dot = gc0 * c.x + gc1 * c.y + gc2 * c.z + gD * b.z + gx.x + gU * dz * dz + gx.y * b.w;
                const float dal = T * dot - inv * GS;
                GS = fmaf(w, dot, GS);
                const bool clamped = sg >= kAlphaMax;
                const float dpow = clamped ? 0.f : dal * alpha;
                v[G_MX] = dpow * (a.z * dx + a.w * dy);
                v[G_MY] = dpow * (a.w * dx + b.x * dy);
                v[G_CA] = -0.5f * dpow * dx * dx;
                v[G_CB] = -dpow * dx * dy;
                v[G_CC] = -0.5f * dpow * dy * dy;
                v[G_Z] = w * (gD + 2.f * gU * dz);
                if (j == __float_as_int(gx.w)) v[G_Z] += gx.z;  // D_median = z of the median entry (Eq. 7)
                if (!POSE) {
                    v[G_OP] = clamped ? 0.f : dal * G;
                    v[G_NU] = w * gx.y;
                    v[G_R] = w * gc0;
                    v[G_G] = w * gc1;
                    v[G_B] = w * gc2;
                }
            } else {
#pragma unroll
                for (int m = 0; m < 11; ++m) v[m] = 0.f;
            }
            if (POSE) {
                if (act) {
                    const float th[6] = {v[G_MX], v[G_MY], v[G_CA], v[G_CB], v[G_CC], v[G_Z]};
                    pose_contract(acc, th, &s_j[k * 9]);
                }
            } else {
                const unsigned am = __ballot_sync(0xffffffffu, act);
                if (am != 0u && __popc(am) <= kDirectLanes) {
                    // few lanes blended the entry: each adds its own gradients
                    // (three 128-bit atomics per lane; no warp reduction)
                    if (act) {
                        float4 *gp = reinterpret_cast<float4 *>(grad2d + (size_t)s_idx[k] * kGrad2d);
                        atomicAdd(gp, make_float4(v[0], v[1], v[2], v[3]));
                        atomicAdd(gp + 1, make_float4(v[4], v[5], v[6], v[7]));
                        atomicAdd(gp + 2, make_float4(v[8], v[9], v[10], 0.f));
                    }
                } else if (am != 0u) {
                    // warp sum of the 11 gradients by recursive halving: at each
                    // step a lane keeps half of its values and adds its partner's
                    // copy of them (16 shuffles instead of 11 x 5); lane pairs end
                    // up holding one total each, and 11 lanes add them with one
                    // warp-wide atomic instruction
                    float h[16];
#pragma unroll
                    for (int m = 0; m < 16; ++m) h[m] = m < 11 ? v[m] : 0.f;
#pragma unroll
                    for (int n = 16, o = 16; n > 1; n >>= 1, o >>= 1) {
                        const bool up = (lane & o) != 0;
#pragma unroll
                        for (int i = 0; i < n / 2; ++i) {
                            const float send = up ? h[i] : h[i + n / 2];
                            const float keep = up ? h[i + n / 2] : h[i];
                            h[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                        }
                    }
                    h[0] += __shfl_xor_sync(0xffffffffu, h[0], 1);
                    const int field = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                                      ((lane >> 1) & 1);
                    if ((lane & 1) == 0 && field < 11)
                        atomicAdd(grad2d + (size_t)s_idx[k] * kGrad2d + field, h[0]);
                }
            }
          }
        }
    }
    if (POSE) {
        // per-tile partial (double-float, fixed tree), then the last tile of the
        // frame reduces all of the frame's partials into the FP64 pose gradient
        float *part_f = pose_partials + (size_t)f * per_frame * 12;
        cta_pose_partial(acc, part_f + (size_t)lt * 12, sh.wdf);
        if (pose_grad)
            last_cta_pose_reduce(part_f, per_frame, fd.tiles_x * fd.tiles_y, counters + f, pose_grad + 6 * f, s_red,
                                 &sh.flag);
    }
}

// One CTA per tile, heaviest tiles first when the launch order is given.
// FULL mode at 16x16 is held to 48 registers (5 CTAs per SM, no spills): the
// kernel is bound by instruction issue and the per-entry warp reductions, and
// the fifth CTA hides their latency (2.70 -> 2.60 ms on an 8-frame 640x480
// window).
template <int TILE, int MODE, bool CD, int FULL_BATCH>
__global__ void __launch_bounds__(TILE *TILE, (TILE == 16 && MODE == GS_MODE_FULL) ? 5 : 1)
    k_render_bwd(const float4 *__restrict__ rec, const float4 *__restrict__ jac, const uint32_t *__restrict__ values,
                 const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, FrameTable ft,
                 const float *__restrict__ obs_depth, ImagePtrs fwd,
                 LossParams lp, float *__restrict__ grad2d, float *__restrict__ pose_partials, int per_frame,
                 double *__restrict__ pose_grad, unsigned *__restrict__ counters, const int32_t *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ BwdShared<TILE> sh;
    if (status[0] != 0) return;
    const int gtile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    bwd_tile<TILE, MODE, CD, FULL_BATCH>(gtile, rec, jac, values, ranges, ft, obs_depth, fwd, lp, grad2d,
                                         pose_partials, per_frame, pose_grad, counters, s_dyn, sh);
}

// Persistent form of the FULL-mode backward: as many CTAs as fit on the GPU,
// each pulling the next (frame, tile) item in launch order from the device
// work queue (work_queue.cuh). FULL mode only: its per-record accumulators take
// atomic adds in any order, so no tile waits for another.
template <int TILE, bool CD, int FULL_BATCH>
__global__ void __launch_bounds__(TILE *TILE, TILE == 16 ? 5 : 1)
    k_render_bwd_persist(const float4 *__restrict__ rec, const uint32_t *__restrict__ values,
                         const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, FrameTable ft,
                         const float *__restrict__ obs_depth, ImagePtrs fwd, LossParams lp,
                         float *__restrict__ grad2d, const int32_t *__restrict__ status, unsigned *__restrict__ queue) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ BwdShared<TILE> sh;
    if (status[0] != 0) return;
    for (int it = 0;; ++it) {
        const int item = queue_next(queue, sh.item, it);
        if (item >= ft.total_tiles) break;
        const int gtile = order ? (int)order[item] : item;
        bwd_tile<TILE, GS_MODE_FULL, CD, FULL_BATCH, true>(gtile, rec, nullptr, values, ranges, ft, obs_depth, fwd, lp,
                                                           grad2d, nullptr, 0, nullptr, nullptr, s_dyn, sh);
    }
    queue_exit(queue);
}

// Raises the dynamic shared-memory limit of one kernel once per device (a
// host-side attribute; the first call happens outside any stream capture).
template <auto KERNEL>
cudaError_t set_smem_once(size_t smem) {
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !((done.load() >> dev) & 1)) {
        e = cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) done.fetch_or(1ull << dev);
    }
    return cudaSuccess;
}

template <int TILE, int MODE, bool CD, int FULL_BATCH>
cudaError_t launch_variant(const float4 *rec, const float4 *jac, const uint32_t *values, const uint2 *ranges,
                           const uint32_t *order, const FrameTable &ft, const float *obs_depth, const ImagePtrs &fwd, const LossParams &lp,
                           float *grad2d, float *pp, int per_frame, double *pg, unsigned *cnt, const int32_t *status,
                           unsigned *queue, cudaStream_t s) {
    constexpr size_t smem = BwdSmem<TILE, MODE, FULL_BATCH>::bytes;
    cudaError_t e;
    if (MODE == GS_MODE_FULL && queue) {
        constexpr size_t smem_p = BwdSmem<TILE, MODE, FULL_BATCH, true>::bytes;
        constexpr auto kern = k_render_bwd_persist<TILE, CD, FULL_BATCH>;
        if ((e = set_smem_once<kern>(smem_p)) != cudaSuccess) return e;
        int grid = 0;
        if ((e = persistent_grid<kern>(TILE * TILE, smem_p, ft.total_tiles, &grid)) != cudaSuccess) return e;
        kern<<<grid, TILE * TILE, smem_p, s>>>(rec, values, ranges, order, ft, obs_depth, fwd, lp, grad2d, status, queue);
        return cudaGetLastError();
    }
    constexpr auto kern = k_render_bwd<TILE, MODE, CD, FULL_BATCH>;
    if ((e = set_smem_once<kern>(smem)) != cudaSuccess) return e;
    kern<<<ft.total_tiles, TILE * TILE, smem, s>>>(rec, jac, values, ranges, order, ft, obs_depth, fwd, lp, grad2d, pp,
                                                   per_frame, pg, cnt, status);
    return cudaGetLastError();
}

template <int TILE, int FULL_BATCH>
cudaError_t launch_batch(int mode, bool cd, const float4 *rec, const float4 *jac, const uint32_t *values,
                         const uint2 *ranges, const uint32_t *order, const FrameTable &ft, const float *obs_depth,
                         const ImagePtrs &fwd, const LossParams &lp, float *grad2d, float *pp, int per_frame,
                         double *pg, unsigned *cnt, const int32_t *status, unsigned *queue, cudaStream_t s) {
#define GS_BWD_ARGS rec, jac, values, ranges, order, ft, obs_depth, fwd, lp, grad2d, pp, per_frame, pg, cnt, status, queue, s
    if (mode == GS_MODE_POSE)  // the POSE backward stages 256 entries (with their Jacobians) per batch
        return cd ? launch_variant<TILE, GS_MODE_POSE, true, kFullBatch>(GS_BWD_ARGS)
                  : launch_variant<TILE, GS_MODE_POSE, false, kFullBatch>(GS_BWD_ARGS);
    return cd ? launch_variant<TILE, GS_MODE_FULL, true, FULL_BATCH>(GS_BWD_ARGS)
              : launch_variant<TILE, GS_MODE_FULL, false, FULL_BATCH>(GS_BWD_ARGS);
#undef GS_BWD_ARGS
}

template <int TILE>
cudaError_t launch_tile(int mode, const float4 *rec, const float4 *jac, const uint32_t *values, const uint2 *ranges,
                        const uint32_t *order, const FrameTable &ft, const float *obs_depth, const ImagePtrs &fwd, const LossParams &lp,
                        float *grad2d, float *pp, int per_frame, double *pg, unsigned *cnt, const int32_t *status,
                        int batch, unsigned *queue, cudaStream_t s) {
    const bool cd = lp.fused ? (lp.w_unc == 0.f && lp.w_nu == 0.f && lp.w_align == 0.f)
                             : (!lp.g_alpha && !lp.g_unc && !lp.g_nu && !lp.g_median);
    if (mode == GS_MODE_FULL && TILE >= 16 && batch == 256)
        return launch_batch<TILE, 256>(mode, cd, rec, jac, values, ranges, order, ft, obs_depth, fwd, lp, grad2d, pp,
                                       per_frame, pg, cnt, status, queue, s);
    return launch_batch<TILE, kFullBatch>(mode, cd, rec, jac, values, ranges, order, ft, obs_depth, fwd, lp, grad2d,
                                          pp, per_frame, pg, cnt, status, queue, s);
}

}  // namespace

cudaError_t launch_render_bwd(int mode, const float *rec, const float *jac, const uint32_t *values,
                              const uint32_t *ranges, const uint32_t *order, const FrameTable &ft, const float *obs_depth,
                              const ImagePtrs &fwd, const LossParams &lp, float *grad2d, float *pose_partials,
                              int per_frame, double *pose_grad, unsigned *counters, const int32_t *status,
                              int batch, unsigned *queue, cudaStream_t s) {
    if (ft.total_tiles == 0) return cudaSuccess;
    const float4 *r4 = reinterpret_cast<const float4 *>(rec);
    const float4 *j4 = reinterpret_cast<const float4 *>(jac);
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
#define GS_BWD_ARGS mode, r4, j4, values, rg, order, ft, obs_depth, fwd, lp, grad2d, pose_partials, per_frame, pose_grad, counters, status, batch, queue, s
    switch (ft.tile) {
        case 8: return launch_tile<8>(GS_BWD_ARGS);
        case 16: return launch_tile<16>(GS_BWD_ARGS);
        case 32: return launch_tile<32>(GS_BWD_ARGS);
        default: return cudaErrorInvalidValue;
    }
#undef GS_BWD_ARGS
}

}  // namespace gs
