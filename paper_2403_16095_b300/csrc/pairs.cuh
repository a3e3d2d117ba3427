// Pair expansion of tile binning, shared by the binning kernels and by the
// projection when it counts pairs itself: the tile rect of a record's pixel
// rect, the warp-balanced walk over the (record, tile) pairs of a warp's
// records, and the warp-aggregated claim of tile-counter slots.
#pragma once

#include "gs_internal.cuh"

namespace gs {

// tile rect of a record's inclusive pixel rect (clipped to the frame's tiles)
struct TileRect {
    int x0, y0, x1, y1;
};
__device__ __forceinline__ TileRect tile_rect(const int4 &rc, int ts, const FrameDesc &fd) {
    TileRect t;
    t.x0 = max(rc.x, 0) / ts;
    t.y0 = max(rc.y, 0) / ts;
    t.x1 = min(rc.z / ts, fd.tiles_x - 1);
    t.y1 = min(rc.w / ts, fd.tiles_y - 1);
    return t;
}

// One record per lane; its (record, tile) pairs are spread over the warp's
// lanes (warp prefix sum of the per-record tile counts, then lane l handles
// pairs l, l + 32, ...), so one large footprint does not serialise its warp.
struct PairSrc {
    bool valid;
    TileRect t;
    int tile_off, tiles_x;
    uint32_t payload;  // per-record value handed to the pair callback (depth bits)
};

// Walks every pair of the warp's records, 32 at a time: calls
// f(valid, owner_lane, global_tile, owner_payload) on all 32 lanes together
// (valid = the lane holds a pair in this step), so that f may use warp
// collectives; all shuffles happen with the whole warp converged.
template <class F>
__device__ __forceinline__ void warp_for_each_pair(const PairSrc &s, F &&f) {
    const int lane = threadIdx.x & 31;
    const int w = s.valid ? s.t.x1 - s.t.x0 + 1 : 0;
    const int cnt = s.valid ? w * (s.t.y1 - s.t.y0 + 1) : 0;
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        // owner = first lane whose inclusive prefix exceeds p (binary search)
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int probe = __shfl_sync(0xffffffffu, incl, lo + step - 1);
            if (probe <= p) lo += step;
        }
        const int owner = lo;
        const int o_incl = __shfl_sync(0xffffffffu, incl, owner);
        const int o_cnt = __shfl_sync(0xffffffffu, cnt, owner);
        const int o_w = __shfl_sync(0xffffffffu, w, owner);
        const int o_x0 = __shfl_sync(0xffffffffu, s.t.x0, owner);
        const int o_y0 = __shfl_sync(0xffffffffu, s.t.y0, owner);
        const int o_off = __shfl_sync(0xffffffffu, s.tile_off, owner);
        const int o_tx = __shfl_sync(0xffffffffu, s.tiles_x, owner);
        const uint32_t o_pl = __shfl_sync(0xffffffffu, s.payload, owner);
        const bool valid = p < total;
        int gt = -1;
        if (valid) {
            const int j = p - (o_incl - o_cnt);
            const int ty = o_y0 + j / o_w, tx = o_x0 + j % o_w;
            gt = o_off + ty * o_tx + tx;
        }
        f(valid, owner, gt, o_pl);
    }
}

// Warp-aggregated claim of one slot per valid lane in the counter of its tile
// (tile t's counter at tc.p[t tc.stride]): lanes with the same tile share one
// atomic (issued by the lowest of them). Returns the lane's slot when want_slot
// (the atomic's old value + its rank among its peers), else 0 and the atomic
// needs no return value. Records of a warp are often neighbours in space
// (Morton-ordered storage), so most of a warp's pairs tend to fall on a few
// tiles.
template <bool WANT_SLOT>
__device__ __forceinline__ uint32_t warp_claim(bool valid, int gt, TileCtr tc) {
    const int lane = threadIdx.x & 31;
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? gt : -1);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) {
        uint32_t *ctr = tc.p + (size_t)gt * (size_t)tc.stride;
        if (WANT_SLOT)
            base = atomicAdd(ctr, (uint32_t)__popc(peers));
        else
            atomicAdd(ctr, (uint32_t)__popc(peers));
    }
    if (!WANT_SLOT) return 0u;
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

}  // namespace gs
