// Forward blend and POSE-mode backward of the tracking loss in one pass per
// tile (CG-SLAM Eq. 3-10 and their adjoint, with the fused loss of Eq. 14, 16,
// 19).
//
// Tracking needs, per pixel, only the loss gradient w.r.t. its own rendered
// colour and depth, so nothing has to wait for other tiles between the forward
// and the backward of a tile. One CTA therefore renders its tile front to back,
// keeps colour, depth, the nu map, T_final and the last blended position in
// registers, forms the loss gradient, and walks the same list back to front.
// Against gs_render_fwd + gs_render_bwd this saves:
//   - the image round trip through memory;
//   - the second staging of the last batch: records and pose Jacobians staged
//     for the forward stay in shared memory for the backward when the batch
//     boundaries coincide, i.e. whenever the walk fits in one batch;
//   - one launch and one tail of idle SMs;
//   - the pose reduction's arrival ticket and memory fence in every CTA: the
//     per-tile partials are summed (and the Adam step applied) by one small
//     launch chained after this one (launch_pose_reduce_adam), which measured
//     ~2 us per tracking iteration faster than a last-CTA tail in this kernel.
// The per-pixel arithmetic is the same as in the two kernels (same helpers,
// same order), so images and pose gradients are bit-identical to them.
#include "gs_internal.cuh"
#include "blend_common.cuh"
#include "dfloat.cuh"

#include <atomic>

namespace gs {
namespace {

__device__ __forceinline__ float sgn_f(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

constexpr int kCullGroups = 64;  // cached warp-cull ballots per warp: lists of up to 2,048 entries

template <int TILE>
struct FusedSmem {
    static constexpr int NT = TILE * TILE;
    static constexpr int BATCH = NT < 256 ? NT : 256;
    static constexpr size_t bytes = (size_t)BATCH * 13 * sizeof(float4);  // record (4) + Jacobian (9)
};

// At tile 16 the pass is built for 3 CTAs per SM (80 registers). A 4-CTA
// build (63 registers, no spills) was faster at ~1,550 records per tile
// before the per-entry chains were shortened (2.14 vs 2.27 ms per iteration
// at 1200x680 / 5M); with them it is slower at both measured list lengths:
// 126.2 vs 116.0 us per launch at 640x480 / 300k (~250 records per tile) and
// 1.360 vs 1.350 ms at 1200x680 / 5M.
template <int TILE, int MINB>
__global__ void __launch_bounds__(TILE *TILE, MINB)
    k_render_fused_pose(const float4 *__restrict__ rec, const float4 *__restrict__ jac,
                        const uint32_t *__restrict__ values, const uint2 *__restrict__ ranges,
                        const uint32_t *__restrict__ order, FrameTable ft, ImagePtrs out, LossParams lp,
                        float *__restrict__ pose_partials, int per_frame, const int32_t *__restrict__ status) {
    dep_wait();
    using SM = FusedSmem<TILE>;
    constexpr int NT = SM::NT;
    constexpr int BATCH = SM::BATCH;
    constexpr int NWARP = NT / 32 > 0 ? NT / 32 : 1;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    float4 *s_a = reinterpret_cast<float4 *>(s_dyn);
    float4 *s_b = s_a + BATCH;
    float4 *s_c = s_b + BATCH;
    int4 *s_r = reinterpret_cast<int4 *>(s_c + BATCH);
    float4 *s_j = reinterpret_cast<float4 *>(s_r + BATCH);
    __shared__ uint32_t s_wmax[NWARP];
    __shared__ df s_wdf[NWARP][6];
    // the forward's warp-cull ballot of every 32-entry group of the list (first
    // kCullGroups groups): the backward walks the same entries with the same
    // warp and reuses them instead of evaluating warp_block_may_hit again
    __shared__ uint32_t s_cull[NWARP][kCullGroups];
    // the tile (heaviest first) and its list range are loaded alongside the
    // status word instead of after it; the index is clamped because, with the
    // status set, an earlier kernel of the iteration may have left `order`
    // unwritten
    const int gtile = order ? (int)min(order[blockIdx.x], (uint32_t)(ft.total_tiles - 1)) : (int)blockIdx.x;
    const uint2 range = ranges[gtile];
    if (status[0] != 0) return;

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

    // stages list entries [lo, hi) of the tile into shared memory
    auto stage = [&](int lo, int hi) {
        for (int i = tid; i < hi - lo; i += NT) {
            const uint32_t r = values[lo + i];
            const float4 *R = rec + (size_t)r * 4;
            s_a[i] = R[0];
            s_b[i] = R[1];
            s_c[i] = R[2];
            s_r[i] = reinterpret_cast<const int4 *>(R)[3];
            const float4 *J = jac + (size_t)r * 9;
#pragma unroll
            for (int q = 0; q < 9; ++q) s_j[i * 9 + q] = J[q];
        }
    };

    // ---------------------------------------------------------- forward
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, dep = 0.f, nus = 0.f;
    uint32_t last = range.x;
    bool done = !inside;
    int staged_lo = -1;  // first list position held in shared memory (-1: none)
    for (uint32_t base = range.x; base < range.y; base += BATCH) {
        if (__syncthreads_count(done) == NT) break;  // also orders smem reuse
        const int hi = (int)min(range.y, base + BATCH);
        stage((int)base, hi);
        staged_lo = (int)base;
        __syncthreads();
        const int cnt = hi - (int)base;
        if (!__all_sync(0xffffffffu, done)) {
            for (int g0 = 0; g0 < cnt; g0 += 32) {
                const int kt = g0 + lane;
                const bool hit = kt < cnt && warp_block_may_hit(s_a[kt], s_b[kt], s_r[kt], wx0, wy0);
                unsigned mask = __ballot_sync(0xffffffffu, hit);
                const int gi = ((int)(base - range.x) + g0) >> 5;
                if (lane == 0 && gi < kCullGroups) s_cull[warp][gi] = mask;
                while (mask) {  // surviving entries, front to back
                    const int k = g0 + __ffs(mask) - 1;
                    mask &= mask - 1;
                    const float4 a = s_a[k];
                    const float4 b = s_b[k];
                    const float4 c = s_c[k];  // loaded with a and b: off the blend's dependency chain
                    // the tests are predicates, not exits: the lanes stay on one path
                    // (saturated lanes evaluate alpha too, and discard it)
                    float dx = 0.f, dy = 0.f, G = 0.f, sg = 0.f, alpha = 0.f;
                    const bool ok = (!done) & eval_alpha(pxc, pyc, a, b, dx, dy, G, sg, alpha);
                    const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
                    const bool stop = ok && Tn < kTMin;  // stop before T would drop below 1e-4
                    done = done || stop;
                    if (ok && !stop) {
                        const float w = __fmul_rn(alpha, T);
                        c0 = fmaf(w, c.x, c0);
                        c1 = fmaf(w, c.y, c1);
                        c2 = fmaf(w, c.z, c2);
                        dep = fmaf(w, b.z, dep);
                        nus = fmaf(w, b.w, nus);
                        T = Tn;
                        last = base + k + 1;
                    }
                }
                if (__all_sync(0xffffffffu, done)) break;
            }
        }
    }
    if (inside) {  // optional image outputs (bit-identical to gs_render_fwd)
        if (out.color) {
            out.color[cbase] = c0;
            out.color[cbase + HW] = c1;
            out.color[cbase + 2 * (size_t)HW] = c2;
        }
        if (out.depth) out.depth[pix] = dep;
        if (out.nu_map) out.nu_map[pix] = nus;
        if (out.T_final) out.T_final[pix] = T;
        if (out.n_last) out.n_last[pix] = (int32_t)last;
    }

    // ------------------------------------------- loss gradient (Eq. 14, 16, 19)
    float gc0 = 0.f, gc1 = 0.f, gc2 = 0.f, gD = 0.f;
    const uint32_t my_last = last;
    if (inside) {
        const float inv_hw = 1.f / (float)HW;
        float m = 1.f;
        if (lp.unc_tau > 0.f) m = 1.f / (1.f + nus / lp.unc_tau);
        const float kc = inv_hw * m * lp.w_color, kd = inv_hw * m * lp.w_depth;
        if (lp.w_color != 0.f) {
            gc0 = kc * sgn_f(c0 - lp.target_color[cbase]);
            gc1 = kc * sgn_f(c1 - lp.target_color[cbase + HW]);
            gc2 = kc * sgn_f(c2 - lp.target_color[cbase + 2 * (size_t)HW]);
        }
        if (lp.w_depth != 0.f) gD = kd * sgn_f(dep - lp.target_depth[pix]);
    }

    // ---------------------------------------------------------- backward
    const uint32_t warp_last = __reduce_max_sync(0xffffffffu, my_last);
    // A list of at most one batch is still staged whole (nothing is restaged
    // below), so each warp walks back from its own last entry without waiting
    // for the others' forwards. Longer lists restage batch by batch, with every
    // warp, from the CTA's last entry.
    const bool one_batch = range.y - range.x <= (uint32_t)BATCH;
    uint32_t block_last = warp_last;
    if (!one_batch) {
        if (lane == 0) s_wmax[warp] = warp_last;
        __syncthreads();
        block_last = range.x;
#pragma unroll
        for (int w = 0; w < NWARP; ++w) block_last = max(block_last, s_wmax[w]);
    }

    float GS = 0.f;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // batches aligned with the forward's, last first: the last forward batch is
    // still staged when the walk ends inside it
    const int nbatch = block_last > range.x ? (int)((block_last - 1 - range.x) / BATCH) + 1 : 0;
    for (int m = nbatch - 1; m >= 0; --m) {
        const int bstart = (int)range.x + m * BATCH;
        const int bend = min((int)block_last, bstart + BATCH);
        if (bstart != staged_lo) {
            __syncthreads();
            stage(bstart, min((int)range.y, bstart + BATCH));
            staged_lo = bstart;
            __syncthreads();
        }
        const int cnt = bend - bstart;
        // groups aligned with the forward's (batch start + 32 i), last first
        for (int g0 = ((cnt - 1) >> 5) << 5; g0 >= 0; g0 -= 32) {
            const int kt = g0 + lane;
            const bool live = kt < cnt && (uint32_t)(bstart + kt) < warp_last;
            const int gi = (bstart - (int)range.x + g0) >> 5;
            unsigned mask;
            if (gi < kCullGroups) {
                __syncwarp();
                mask = __ballot_sync(0xffffffffu, live) & s_cull[warp][gi];
            } else {
                mask = __ballot_sync(0xffffffffu, live && warp_block_may_hit(s_a[kt], s_b[kt], s_r[kt], wx0, wy0));
            }
            while (mask) {  // surviving entries, back to front
                const int bit = 31 - __clz(mask);
                mask &= ~(1u << bit);
                const int k = g0 + bit;
                const int j = bstart + k;
                const float4 a = s_a[k];
                const float4 b = s_b[k];
                const float4 c = s_c[k];
                float dx = 0.f, dy = 0.f, G = 0.f, sg = 0.f, alpha = 0.f;
                bool act;
                if (MINB == 3) {  // one path for all lanes up to the act test
                    act = ((uint32_t)j < my_last) & eval_alpha(pxc, pyc, a, b, dx, dy, G, sg, alpha);
                } else {  // the other builds: branching spills less
                    act = (uint32_t)j < my_last;
                    if (act) act = eval_alpha(pxc, pyc, a, b, dx, dy, G, sg, alpha);
                }
                if (act) {
                    float th[6], w, dal;
                    entry_grad_cd(alpha, sg, dx, dy, a, b, c, gc0, gc1, gc2, gD, T, GS, th, w, dal);
                    pose_contract(acc, th, &s_j[k * 9]);
                }
            }
        }
    }
    // per-tile partial (double-float, fixed tree); the frame's partials are
    // summed by the chained reduction launch. The barrier lets every warp
    // finish its walk before the tile's sum (cta_pose_partial orders its own
    // shared-memory exchange).
    float *part_f = pose_partials + (size_t)f * per_frame * 12;
    __syncthreads();
    cta_pose_partial(acc, part_f + (size_t)lt * 12, s_wdf);
}

template <int TILE>
cudaError_t launch_tile(const float4 *rec, const float4 *jac, const uint32_t *values, const uint2 *ranges,
                        const uint32_t *order, const FrameTable &ft, const ImagePtrs &out, const LossParams &lp,
                        float *pp, int per_frame, const int32_t *status, cudaStream_t s) {
    // raise the dynamic shared-memory limit once per device (a host-side
    // attribute; the first call happens outside any stream capture)
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    constexpr size_t smem = FusedSmem<TILE>::bytes;
    constexpr int kMinb = TILE == 16 ? 3 : 1;
    if (dev >= 64 || !((done.load() >> dev) & 1)) {
        e = cudaFuncSetAttribute(k_render_fused_pose<TILE, kMinb>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) done.fetch_or(1ull << dev);
    }
    auto kernel = k_render_fused_pose<TILE, kMinb>;
    return launch_chained(kernel, dim3(ft.total_tiles), dim3(TILE * TILE), smem, s, rec, jac, values, ranges, order, ft,
                          out, lp, pp, per_frame, status);
}

}  // namespace

cudaError_t launch_render_fused_pose(const float *rec, const float *jac, const uint32_t *values,
                                     const uint32_t *ranges, const uint32_t *order, const FrameTable &ft,
                                     const ImagePtrs &out, const LossParams &lp, float *pose_partials, int per_frame,
                                     const int32_t *status, cudaStream_t s) {
    if (ft.total_tiles == 0) return cudaSuccess;
    const float4 *r4 = reinterpret_cast<const float4 *>(rec);
    const float4 *j4 = reinterpret_cast<const float4 *>(jac);
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
    switch (ft.tile) {
        case 8: return launch_tile<8>(r4, j4, values, rg, order, ft, out, lp, pose_partials, per_frame, status, s);
        case 16: return launch_tile<16>(r4, j4, values, rg, order, ft, out, lp, pose_partials, per_frame, status, s);
        case 32: return launch_tile<32>(r4, j4, values, rg, order, ft, out, lp, pose_partials, per_frame, status, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gs
