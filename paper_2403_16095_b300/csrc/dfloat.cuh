// Double-float (hi, lo FP32 pair) compensated summation for the pose-gradient
// reductions. B300 executes FP64 at a small fraction of its FP32 rate, so the
// reductions carry ~48-bit sums in FP32 pairs (Knuth's TwoSum, every operation
// explicitly rounded so the compiler cannot reassociate) and convert to FP64
// only for the final value.
#pragma once

#include <cuda_runtime.h>

namespace gs {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s.hi, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s.hi))};
}


// Warp sum of six FP32 values per lane as double-floats, by recursive halving:
// at each of three steps (lane bits 4, 3, 2) a lane keeps half of its slots
// (8 slots, the last two zero) and adds its partner's copy of them, then two
// full butterfly steps (lane bits 1, 0) finish. Lane l ends with the total of
// slot ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1), written to
// `slot`; the four lanes sharing bits 2-4 hold the same value (df_add is
// symmetric). A fixed order, so the result is deterministic; ~14 shuffles
// instead of 60 for six separate butterflies.
__device__ __forceinline__ df df_warp_sum6(const float v[6], int &slot) {
    const int lane = threadIdx.x & 31;
    const bool up4 = (lane & 16) != 0, up3 = (lane & 8) != 0, up2 = (lane & 4) != 0;
    df h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float lo_slot = v[i], hi_slot = i + 4 < 6 ? v[i + 4] : 0.f;
        const float keep = up4 ? hi_slot : lo_slot, send = up4 ? lo_slot : hi_slot;
        h[i] = df_two_sum(keep, __shfl_xor_sync(0xffffffffu, send, 16));
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const df keep = up3 ? h[i + 2] : h[i], send = up3 ? h[i] : h[i + 2];
        h[i] = df_add(keep, df{__shfl_xor_sync(0xffffffffu, send.hi, 8), __shfl_xor_sync(0xffffffffu, send.lo, 8)});
    }
    {
        const df keep = up2 ? h[1] : h[0], send = up2 ? h[0] : h[1];
        h[0] = df_add(keep, df{__shfl_xor_sync(0xffffffffu, send.hi, 4), __shfl_xor_sync(0xffffffffu, send.lo, 4)});
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1)
        h[0] = df_add(h[0], df{__shfl_xor_sync(0xffffffffu, h[0].hi, o), __shfl_xor_sync(0xffffffffu, h[0].lo, o)});
    slot = (up4 ? 4 : 0) + (up3 ? 2 : 0) + (up2 ? 1 : 0);
    return h[0];
}

}  // namespace gs

namespace gs {

// Pose partials: [K][6] double-floats stored as [K][6][2] floats (hi, lo).
constexpr int kRedSlots = 256;

// Fixed-order sum of K pose partials into six FP64 values. Slot s in [0, 256)
// accumulates partials j = s, s + 256, ... in increasing j, then a fixed binary
// tree combines the slots (slot s takes slot s + stride, stride 128 down to 1).
// The order depends only on K -- not on the number of threads running it -- so
// every caller gets bit-identical results. Loads bypass L1 (the partials may
// have been written by other CTAs of the same launch) and are issued several
// partials at a time, so a slot waits for one L2 round trip per kAhead
// partials instead of one per partial (kAhead = 4 by default);
// the adds keep their order, so kAhead changes no bits. The tree runs through
// shared memory down to 32 slots, then in warp 0 by shuffles (same pairs, same
// operand order). Needs blockDim.x >= 32 and a shared buffer of 256 x 6
// double-floats.
template <int kAhead = 4>
__device__ __forceinline__ void reduce_pose_partials(const float *p, int K, double *out6, df (*s_red)[6]) {
    for (int s = threadIdx.x; s < kRedSlots; s += blockDim.x) {
        df acc[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] = {0.f, 0.f};
        for (int j = s; j < K; j += kAhead * kRedSlots) {
            float2 v[kAhead][6];
#pragma unroll
            for (int r = 0; r < kAhead; ++r) {
                const int jj = j + r * kRedSlots;
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    v[r][k] = jj < K ? __ldcg(reinterpret_cast<const float2 *>(p) + (size_t)jj * 6 + k)
                                     : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < kAhead; ++r)
                if (j + r * kRedSlots < K)
#pragma unroll
                    for (int k = 0; k < 6; ++k) acc[k] = df_add(acc[k], df{v[r][k].x, v[r][k].y});
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) s_red[s][k] = acc[k];
    }
    __syncthreads();
    for (int stride = kRedSlots / 2; stride >= 32; stride >>= 1) {
        for (int s = threadIdx.x; s < stride; s += blockDim.x)
#pragma unroll
            for (int k = 0; k < 6; ++k) s_red[s][k] = df_add(s_red[s][k], s_red[s + stride][k]);
        __syncthreads();
    }
    if (threadIdx.x < 32) {
        df h[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = s_red[threadIdx.x][k];
#pragma unroll
        for (int stride = 16; stride > 0; stride >>= 1)
#pragma unroll
            for (int k = 0; k < 6; ++k)
                h[k] = df_add(h[k], df{__shfl_down_sync(0xffffffffu, h[k].hi, stride),
                                       __shfl_down_sync(0xffffffffu, h[k].lo, stride)});
        // lane 0 holds the tree's root; hand it to lanes 0-5, one component each
        double r = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float hi = __shfl_sync(0xffffffffu, h[k].hi, 0), lo = __shfl_sync(0xffffffffu, h[k].lo, 0);
            if (threadIdx.x == k) r = (double)hi + (double)lo;
        }
        if (threadIdx.x < 6) out6[threadIdx.x] = r;
    }
    __syncthreads();
}

// Per-CTA double-float sum of six per-thread FP32 values (fixed tree); thread 0
// writes the partial (hi, lo pairs) to out12. s_w: [n_warps][6] double-floats.
__device__ __forceinline__ void cta_pose_partial(const float acc[6], float *out12, df (*s_w)[6]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int slot;
    const df v = df_warp_sum6(acc, slot);
    if ((lane & 3) == 0 && slot < 6) s_w[warp][slot] = v;
    __syncthreads();
    if (threadIdx.x < 6) {
        df s = {0.f, 0.f};
        for (int w = 0; w < nw; ++w) s = df_add(s, s_w[w][threadIdx.x]);
        reinterpret_cast<float2 *>(out12)[threadIdx.x] = make_float2(s.hi, s.lo);
    }
}

// Threadfence-reduction tail: after every CTA of frame f has written its
// partial, the last one to arrive (ticket = n_ctas - 1) reduces them in fixed
// order into pose_grad[6]. counter must be zero before the launch.
__device__ __forceinline__ void last_cta_pose_reduce(const float *partials_f, int K, int n_ctas, unsigned *counter,
                                                     double *pose_grad, df (*s_red)[6], int *s_flag) {
    __threadfence();
    __syncthreads();
    // atomicInc wraps the counter back to 0 at the last arrival, so it is
    // ready for the next launch without a memset
    if (threadIdx.x == 0) *s_flag = (atomicInc(counter, (unsigned)(n_ctas - 1)) == (unsigned)(n_ctas - 1));
    __syncthreads();
    if (*s_flag) {
        __threadfence();
        reduce_pose_partials(partials_f, K, pose_grad, s_red);
    }
}

}  // namespace gs
