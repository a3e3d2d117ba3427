// Tile binning: the "pre-sort of all visible Gaussians from near to far" of
// CG-SLAM Sec. 3.1, done per tile, as an MSD radix sort of the 64-bit keys
// (global tile id << 32 | float bits of depth) with the record index as the
// final tie-break:
//
//   k_bin_clear   zeroes the tile counters (a line apart in the workspace for
//                 calls of up to 4,096 tiles, else the end words of `ranges`;
//                 tile_counters) and the call's scalars.
//   k_tile_count  MSD digit = the tile id: one atomic increment per
//                 (record, overlapped tile) into the tile's counter; pairs are
//                 spread over the lanes of a warp so large footprints do not
//                 serialise, and lanes on the same tile share one atomic
//                 (pairs.cuh). gs_project_bin does this count in the
//                 projection kernel instead and skips this pass.
//   k_tile_scan   exclusive scan of the counters -> each tile's final
//                 [start, end) in `ranges`, the fill's cursor (= start), the
//                 total pair count P and the capacity check; optionally
//                 the launch order of the blend kernels: tiles by descending
//                 list length (a counting sort on lengths / 4), so that the
//                 longest tiles, which bound the blend kernels, start first.
//   k_tile_fill   each pair claims a slot in its tile's bucket (the cursor's
//                 atomic) and stores the low key (depth bits << 32 | record).
//   k_tile_sort   sorts each bucket's low keys: buckets under 256 keys by one
//                 warp in registers; up to 512 keys by a CTA bitonic network
//                 in registers and shared memory; larger ones by two stable LSD
//                 passes over the depth quantised to 16 bits over the bucket's
//                 depth range (in shared memory up to 2048 keys, ping-ponging
//                 in global memory beyond), after which each run of equal
//                 quantised depth is put in full-key order (runs longer than 32
//                 keys: a full LSD sort over the record-index digits, then the
//                 depth digits; digits constant over the bucket are skipped).
//                 Low keys are
//                 unique within a bucket, so the order of the atomic fill does
//                 not matter: the output is bit-exact, the same as a stable sort
//                 of the 64-bit keys emitted in record order, and independent of
//                 the launch configuration.
#include <climits>

#include "gs_internal.cuh"
#include "pairs.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kPassUnroll = 4;  // 32-key groups per step of a radix pass (loads issued together)
constexpr int kRadixMinKeys = 512;   // CTA lists above this (up to kSmemKeys) take the shared-memory radix sort
constexpr int kSmemKeys = 2048;  // bucket size sorted entirely in shared memory
constexpr int kBallotSmemTiles = 2048;  // larger batches: ballot peers in the shared-memory passes too

__device__ __forceinline__ bool status_ok(const int32_t *status) { return status[0] == 0; }

// The loads of one record that the pair expansion needs. On large batches
// k_tile_count and k_tile_fill give each thread kRecLarge records and issue
// the loads of all of them together -- first the visibility counts, then the
// rect (and depth) of the visible ones: the kernels are bound by memory
// latency, and this takes two round trips per kRecLarge records instead of two
// per record. A thread's records are a grid apart (record b kThreads + t +
// j gridDim kThreads), so that every CTA samples the whole batch: with records
// in spatial order the visible ones sit in contiguous ranges, and contiguous
// chunks per CTA would hand all of the expansion work to a few CTAs. Small
// batches keep one record per thread so that the grid still fills the GPU.
constexpr int kRecLarge = 8;
// records per SM (x 2,048 threads x kRecLarge / 2) from which a batch takes kRecLarge per thread
constexpr int kLargeBatchPerSm = 2048 * kRecLarge / 2;
struct RecLoad {
    int touched;
    int4 rc;
    uint32_t zb;  // depth bits (fill only)
};

template <int R, bool Z>
__device__ __forceinline__ void load_records(const float *__restrict__ rec, const int *__restrict__ touched,
                                             int base, int stride, int M, RecLoad (&L)[R]) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const long long i = (long long)base + (long long)j * stride;
        L[j].touched = i < M ? touched[i] : 0;
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const size_t i = (size_t)base + (size_t)j * stride;
        if (L[j].touched > 0) {
            L[j].rc = *reinterpret_cast<const int4 *>(rec + i * kRecFloats + R_X0);
            if (Z) L[j].zb = __float_as_uint(rec[i * kRecFloats + R_Z]);
        }
    }
}

__device__ __forceinline__ PairSrc pair_source(const RecLoad &L, int i, int n_per_frame, const FrameTable &ft) {
    PairSrc p{};
    p.valid = L.touched > 0;
    if (p.valid) {
        const FrameDesc &fd = ft.f[i / n_per_frame];
        p.t = tile_rect(L.rc, ft.tile, fd);
        p.tile_off = fd.tile_off;
        p.tiles_x = fd.tiles_x;
        p.payload = L.zb;
    }
    return p;
}

template <int R>
__global__ void __launch_bounds__(kThreads)
    k_tile_count(const float *__restrict__ rec, const int *__restrict__ touched, int M, int n_per_frame, FrameTable ft,
                 TileCtr tc, const int32_t *__restrict__ status) {
    dep_wait();
    if (!status_ok(status)) return;
    const int base = blockIdx.x * kThreads + threadIdx.x, stride = gridDim.x * kThreads;
    RecLoad L[R];
    load_records<R, false>(rec, touched, base, stride, M, L);
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const PairSrc src = pair_source(L[j], base + j * stride, n_per_frame, ft);
        if (!__any_sync(0xffffffffu, src.valid)) continue;
        warp_for_each_pair(src, [&](bool valid, int, int gt, uint32_t) { warp_claim<false>(valid, gt, tc); });
    }
}

// Zeroes the per-tile counters and the scalars of the call before the count: a
// kernel rather than memsets, so that the chain of launches stays kernel to
// kernel.
__global__ void __launch_bounds__(kThreads) k_bin_clear(TileCtr tc, int n_tiles, int *__restrict__ misc) {
    dep_wait();
    const int stride = gridDim.x * kThreads;
    for (int t = blockIdx.x * kThreads + threadIdx.x; t < n_tiles; t += stride) tc.p[(size_t)t * tc.stride] = 0u;
    if (blockIdx.x == 0 && threadIdx.x < 16) misc[threadIdx.x] = 0;
}

// One CTA: exclusive scan of the per-tile counts into the final ranges
// [start, end) and the fill's cursors (counter = start; the fill advances it
// to end). Where the counters are the ranges' end words (tile_counters), the
// cursor is written after the end, so that the fill starts from start.
constexpr int kOrderBuckets = kScanThreads;  // list length / 4, clipped
constexpr int kWarpSortKeys = 256;           // shorter lists are sorted by one warp

__device__ __forceinline__ int order_bucket(uint32_t len) { return (int)min(len >> 2, (uint32_t)kOrderBuckets - 1); }

__global__ void __launch_bounds__(kScanThreads)
    k_tile_scan(uint32_t *ranges, TileCtr tc, int n_tiles, int capacity, int32_t *__restrict__ status,
                int *__restrict__ misc, uint32_t *__restrict__ order) {
    dep_wait();
    __shared__ long long s_w[kScanThreads / 32];
    __shared__ uint32_t s_hist[kOrderBuckets];
    __shared__ uint32_t s_bw[kScanThreads / 32];
    if (!status_ok(status)) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (order) s_hist[t] = 0;
    __syncthreads();
    const int per = (n_tiles + kScanThreads - 1) / kScanThreads;
    const int lo = min(n_tiles, t * per), hi = min(n_tiles, lo + per);
    long long local = 0;
    for (int k = lo; k < hi; ++k) {
        const uint32_t c = tc.p[(size_t)k * tc.stride];
        local += c;
        if (order) atomicAdd(&s_hist[order_bucket(c)], 1u);
    }
    long long x = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    long long run = x - local, total = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        run += (w < warp) ? s_w[w] : 0;
        total += s_w[w];
    }
    if (order) {
        // descending bucket order: thread t owns bucket B = last - t; its first
        // slot is the number of tiles in heavier buckets (CTA exclusive scan)
        __syncthreads();
        const uint32_t h = s_hist[kOrderBuckets - 1 - t];
        uint32_t xs = h;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xs, off);
            if (lane >= off) xs += y;
        }
        if (lane == 31) s_bw[warp] = xs;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; ++w) pre += s_bw[w];
        s_hist[kOrderBuckets - 1 - t] = pre + xs - h;  // cursor of that bucket
        __syncthreads();
        // tiles of kWarpSortKeys or more entries: the first misc[1] of the order
        if (t == 0) misc[1] = (int)s_hist[kWarpSortKeys / 4 - 1];
        __syncthreads();  // read before the scatter below advances the cursors
    }
    for (int k = lo; k < hi; ++k) {
        uint32_t *ctr = tc.p + (size_t)k * tc.stride;
        const uint32_t c = *ctr;
        const uint32_t start = (uint32_t)(run > UINT_MAX ? UINT_MAX : run);
        run += c;
        ranges[2 * (size_t)k] = start;
        ranges[2 * (size_t)k + 1] = (uint32_t)(run > UINT_MAX ? UINT_MAX : run);
        *ctr = start;  // after the end word, which it may alias
        if (order) order[atomicAdd(&s_hist[order_bucket(c)], 1u)] = (uint32_t)k;
    }
    if (t == 0) {
        status[1] = (int32_t)(total > INT_MAX ? INT_MAX : total);
        if (total > capacity) status[0] = GS_ERR_CAPACITY;
        misc[0] = (int)(total > capacity ? capacity : total);
    }
}

template <int R>
__global__ void __launch_bounds__(kThreads)
    k_tile_fill(const float *__restrict__ rec, const int *__restrict__ touched, int M, int n_per_frame, FrameTable ft,
                TileCtr tc, uint64_t *__restrict__ low_keys, int capacity, const int32_t *__restrict__ status) {
    dep_wait();
    if (!status_ok(status)) return;
    const int base = blockIdx.x * kThreads + threadIdx.x, stride = gridDim.x * kThreads;
    RecLoad L[R];
    load_records<R, true>(rec, touched, base, stride, M, L);
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int i = base + j * stride;
        const PairSrc src = pair_source(L[j], i, n_per_frame, ft);
        if (!__any_sync(0xffffffffu, src.valid)) continue;
        warp_for_each_pair(src, [&](bool valid, int owner, int gt, uint32_t o_zb) {
            const uint32_t slot = warp_claim<true>(valid, gt, tc);
            const uint32_t o_i = (uint32_t)(i - (threadIdx.x & 31) + owner);
            if (valid && slot < (uint32_t)capacity) low_keys[slot] = ((uint64_t)o_zb << 32) | o_i;
        });
    }
}

// Exclusive scan over one value per thread of the CTA; returns the prefix.
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) pre += (w < warp) ? s_warp[w] : 0u;
    __syncthreads();
    return pre + x - v;
}

// 8-bit digits of a key for the LSD passes: the key's own bits at `shift`, or
// a byte of its depth quantised to 16 bits over the bucket's depth range,
// q = ((z - lo) mul) >> 32 with z the depth bits (high word), which is
// monotone in z (positive FP32 depths order as their bits).
struct BitDigit {
    int shift;
    __device__ __forceinline__ uint32_t operator()(uint64_t k) const { return (uint32_t)(k >> shift) & (kRadix - 1); }
};
struct DepthQ {
    uint32_t lo, mul;
    __device__ __forceinline__ uint32_t q(uint64_t k) const {
        return (uint32_t)(((uint64_t)((uint32_t)(k >> 32) - lo) * mul) >> 32);
    }
};
struct QDigit {
    DepthQ dq;
    int shift;
    __device__ __forceinline__ uint32_t operator()(uint64_t k) const { return (dq.q(k) >> shift) & (kRadix - 1); }
};

// The lanes of the warp whose 8-bit digit d equals this lane's, among the lanes
// with `active`, from eight ballots over the digit's bits. The radix passes of
// lists in global memory use it in place of __match_any_sync: ncu showed the
// sort kernel's ADU pipe 70% busy on the mapping window, with the match
// instruction as the suspect; with the ballots there, the mapping window went from
// 2,506 to 2,532 keyframe-iterations/s, the uneven batch from 2,103 to 2,126
// frames/s and 5M tracking from 575 to 577 iterations/s (same box, two runs
// each). Lists in shared memory use it in batches of more than
// kBallotSmemTiles tiles (launch_bin_tiles): there too it measured faster
// (mapping 2,548, uneven 2,135, 5M 584), but a 640x480 tracking frame's
// binning, whose long lists all sit in shared memory, was 1.6 us slower.
__device__ __forceinline__ uint32_t peers8(uint32_t d, bool active) {
    uint32_t m = __ballot_sync(0xffffffffu, active);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t v = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        m &= ((d >> b) & 1u) ? v : ~v;
    }
    return m;
}

// One stable LSD pass of the CTA over n keys: src -> dst by the 8-bit digit
// dig(key). Warp w owns the contiguous segment [w seg, (w + 1) seg) of src: it
// counts its segment's digits into its own histogram row, one CTA scan turns
// the rows (digit-major, warp-minor) into output cursors, and each warp then
// scatters its segment in order with warp barriers only. Returns false (dst
// untouched, src still current) when all n keys share the digit.
template <bool kBallotPeers, class Dig>
__device__ __forceinline__ bool cta_radix_pass(const uint64_t *src, uint64_t *dst, int n, Dig dig,
                                               uint32_t (*s_wh)[kRadix], uint32_t *s_warp) {
    static_assert(kThreads == kRadix, "one digit per thread in the scan");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s_wh[w][tid] = 0;
    __syncthreads();
    const int seg = (((n + kWarps - 1) / kWarps) + 31) & ~31;
    const int lo = min(n, warp * seg), hi = min(n, lo + seg);
    const uint32_t lt_mask = (1u << lane) - 1u;
    // kPassUnroll groups of 32 keys per step: their loads are issued together
    // (the passes are bound by the latency of these L2 reads), then the groups
    // are taken in index order
    for (int base = lo; base < hi; base += 32 * kPassUnroll) {
        uint32_t dg[kPassUnroll];
#pragma unroll
        for (int u = 0; u < kPassUnroll; ++u) {
            const int i = base + 32 * u + lane;
            dg[u] = i < hi ? dig(src[i]) : (uint32_t)kRadix;
        }
#pragma unroll
        for (int u = 0; u < kPassUnroll; ++u) {
            const uint32_t d = dg[u];
            const uint32_t peers = kBallotPeers ? peers8(d, d < (uint32_t)kRadix) : __match_any_sync(0xffffffffu, d);
            if (d < (uint32_t)kRadix && (peers & lt_mask) == 0) s_wh[warp][d] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) tot += s_wh[w][tid];
    if (__syncthreads_or(tot == (uint32_t)n)) return false;
    uint32_t r = cta_excl_scan(tot, s_warp);
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {  // column tid only: no barrier needed before it
        const uint32_t c = s_wh[w][tid];
        s_wh[w][tid] = r;
        r += c;
    }
    __syncthreads();
    for (int base = lo; base < hi; base += 32 * kPassUnroll) {
        uint64_t kg[kPassUnroll];
#pragma unroll
        for (int u = 0; u < kPassUnroll; ++u) {
            const int i = base + 32 * u + lane;
            kg[u] = i < hi ? src[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kPassUnroll; ++u) {
            const bool active = base + 32 * u + lane < hi;
            const uint64_t key = kg[u];
            const uint32_t d = active ? dig(key) : (uint32_t)kRadix;
            const uint32_t peers = kBallotPeers ? peers8(d, active) : __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & lt_mask);
            const uint32_t off = active ? s_wh[warp][d] : 0u;
            if (active) dst[off + rank] = key;
            __syncwarp();
            if (active && rank == 0) s_wh[warp][d] = off + __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    return true;
}

// Keys sorted by a run key rk(key) that is monotone in the full key (the
// quantised depth): put every run of equal rk in full-key order (depth bits,
// then record), the run's first position doing an insertion sort of the run in
// place. Runs are disjoint and other threads read only the run keys of a run,
// which the sort does not change. Returns true for the whole CTA when some run
// is longer than kMaxTieRun (left for a full sort instead).
constexpr int kMaxTieRun = 32;
template <class RunKey>
__device__ __forceinline__ bool cta_fix_runs(uint64_t *a, int n, RunKey rk) {
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        const uint32_t z = rk(a[i]);
        if (i + 1 >= n || rk(a[i + 1]) != z) continue;
        if (i > 0 && rk(a[i - 1]) == z) continue;  // not the first of its run
        int j = i + 2;
        while (j < n && j - i <= kMaxTieRun && rk(a[j]) == z) ++j;
        if (j - i > kMaxTieRun) {
            bad = 1;
            continue;
        }
        for (int p = i + 1; p < j; ++p) {
            const uint64_t k = a[p];
            int q = p - 1;
            while (q >= i && a[q] > k) {
                a[q + 1] = a[q];
                --q;
            }
            a[q + 1] = k;
        }
    }
    return __syncthreads_or(bad) != 0;
}

// Minimum and maximum of the depth bits (high words) of a[0, n), CTA-wide.
__device__ __forceinline__ void cta_depth_range(const uint64_t *a, int n, uint32_t (*s_mm)[kWarps], uint32_t &lo,
                                                uint32_t &hi) {
    uint32_t mn = 0xffffffffu, mx = 0u;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        const uint32_t z = (uint32_t)(a[i] >> 32);
        mn = min(mn, z);
        mx = max(mx, z);
    }
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_mm[0][warp] = mn;
        s_mm[1][warp] = mx;
    }
    __syncthreads();
    lo = s_mm[0][0];
    hi = s_mm[1][0];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) {
        lo = min(lo, s_mm[0][w]);
        hi = max(hi, s_mm[1][w]);
    }
    __syncthreads();
}

struct QRun {
    DepthQ dq;
    __device__ __forceinline__ uint32_t operator()(uint64_t k) const { return dq.q(k); }
};

// Sorts a bucket of n > kRadixMinKeys low keys by the full key (depth bits,
// then record), a[0, n) with b[0, n) as the other buffer, and returns the one
// that holds the result. Two stable LSD passes over the depth quantised to 16
// bits over the bucket's range (DepthQ, mul = 65535 2^32 / (hi - lo)) order the
// keys by quantised depth; each run of equal quantised depth is then put in
// full-key order in place. Quantised depth is monotone in the key, so this is
// the full-key order, in 2 passes where the 32 depth bits take 4. A run longer
// than kMaxTieRun (a tile whose depths crowd into a few quanta, or many equal
// depths) sends the bucket to a full LSD sort over the record-index and depth
// digits.
template <bool kBallotPeers>
__device__ uint64_t *cta_sort_bucket(uint64_t *a, uint64_t *b, int n, int rec_bits, uint32_t (*s_wh)[kRadix],
                                     uint32_t *s_warp, uint32_t (*s_mm)[kWarps]) {
    uint32_t lo, hi;
    cta_depth_range(a, n, s_mm, lo, hi);
    const uint32_t mul =
        hi > lo ? (uint32_t)min((unsigned long long)0xffffffffu, (65535ull << 32) / (unsigned long long)(hi - lo)) : 0u;
    const DepthQ dq{lo, mul};
    for (int shift = 0; shift < 16; shift += kRadixBits) {
        if (cta_radix_pass<kBallotPeers>(a, b, n, QDigit{dq, shift}, s_wh, s_warp)) {
            uint64_t *t = a;
            a = b;
            b = t;
        }
    }
    if (cta_fix_runs(a, n, QRun{dq})) {
        for (int shift = 0; shift < 64; shift += kRadixBits) {
            if (shift >= rec_bits && shift < 32) continue;
            if (cta_radix_pass<kBallotPeers>(a, b, n, BitDigit{shift}, s_wh, s_warp)) {
                uint64_t *t = a;
                a = b;
                b = t;
            }
        }
    }
    return a;
}

// ---------------------------------------------------------------------------
// Bitonic sort of n <= 256 K keys by one CTA of kThreads threads with the keys
// in registers: thread t holds positions t K .. t K + K - 1 (padding = the
// all-ones key, which sorts last). A stage with stride below K stays in the
// thread, one below 32 K is a warp shuffle, and only strides of 32 K or more go
// through shared memory -- the sort is bound by shared-memory bandwidth when
// every stage goes through it. Leaves the sorted keys in s_a[0, n).
template <int K>
__device__ void cta_sort_regs(const uint64_t *keys, int n, uint64_t *s_a) {
    constexpr int NP = kThreads * K;
    const int t = threadIdx.x;
    uint64_t x[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int p = t * K + j;
        x[j] = p < n ? keys[p] : ~0ull;
    }
    // The stage loops stay rolled: fully unrolled, the networks were straight-
    // line code ~2% faster on batches of long lists, but several times larger,
    // and a launch from a cold instruction cache took 24 instead of 13 us.
    for (int size = 2; size <= NP; size <<= 1) {
        for (int stride = size >> 1; stride >= K; stride >>= 1) {
            if (stride >= 32 * K) {  // partner in another warp: exchange through shared
                // memory, position q at s_a[(q % K) kThreads + q / K] (consecutive
                // threads on consecutive words: no bank conflicts)
#pragma unroll
                for (int j = 0; j < K; ++j) s_a[j * kThreads + t] = x[j];
                __syncthreads();
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int p = t * K + j;
                    const int q = p ^ stride;
                    const uint64_t y = s_a[(q % K) * kThreads + q / K];
                    const bool keep_min = ((p & stride) == 0) == ((p & size) == 0);
                    x[j] = keep_min ? (y < x[j] ? y : x[j]) : (y > x[j] ? y : x[j]);
                }
                __syncthreads();
            } else if (stride >= K) {  // partner in another lane of the warp
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int p = t * K + j;
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, x[j], stride / K);
                    const bool keep_min = ((p & stride) == 0) == ((p & size) == 0);
                    x[j] = keep_min ? (y < x[j] ? y : x[j]) : (y > x[j] ? y : x[j]);
                }
            }
        }
        // strides below K: both elements in this thread (compile-time indices)
#pragma unroll
        for (int stride = K / 2; stride > 0; stride >>= 1) {
            if (stride >= size) continue;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if (j & stride) continue;
                const uint64_t a = x[j], b = x[j + stride];
                const bool up = ((t * K + j) & size) == 0;
                if ((a > b) == up) {
                    x[j] = b;
                    x[j + stride] = a;
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) s_a[t * K + j] = x[j];
    __syncthreads();
}

// Bitonic sort of n <= 32 K keys by one warp with the keys in registers: lane
// l holds positions l K .. l K + K - 1 (padding = the all-ones key). Strides
// below K stay in the thread, the others are shuffles; no shared memory. The
// sorted keys go to values[s + i] (record index) and, if keys_out, to
// keys_out[s + i] (tile << 32 | depth bits).
template <int K>
__device__ void warp_sort_regs(const uint64_t *__restrict__ keys, int n, uint32_t *__restrict__ values,
                               uint64_t *__restrict__ keys_out, uint32_t s, uint32_t tile) {
    constexpr int NP = 32 * K;
    const int lane = threadIdx.x & 31;
    uint64_t x[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int p = lane * K + j;
        x[j] = p < n ? keys[p] : ~0ull;
    }
#pragma unroll
    for (int size = 2; size <= NP; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride >= K; stride >>= 1) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int p = lane * K + j;
                const uint64_t y = __shfl_xor_sync(0xffffffffu, x[j], stride / K);
                const bool keep_min = ((p & stride) == 0) == ((p & size) == 0);
                x[j] = keep_min ? (y < x[j] ? y : x[j]) : (y > x[j] ? y : x[j]);
            }
        }
#pragma unroll
        for (int stride = K / 2; stride > 0; stride >>= 1) {
            if (stride >= size) continue;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if (j & stride) continue;
                const uint64_t a = x[j], b = x[j + stride];
                const bool up = ((lane * K + j) & size) == 0;
                if ((a > b) == up) {
                    x[j] = b;
                    x[j + stride] = a;
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int p = lane * K + j;
        if (p < n) {
            values[s + p] = (uint32_t)x[j];
            if (keys_out) keys_out[s + p] = ((uint64_t)tile << 32) | (x[j] >> 32);
        }
    }
}

// k_tile_sort: heaviest tiles first when the launch order is given. With the
// order, tiles of fewer than kWarpSortKeys entries (most of them) are sorted one
// per warp, 8 per CTA, in registers (warp_sort_regs); the others take one CTA each.
// Bitonic networks (low keys are unique within a bucket, so the result is the
// same as a stable radix sort). A CTA sorts its bucket with the keys in
// registers (cta_sort_regs); buckets of more than kSmemKeys keys take the LSD
// radix sort over the depth digits and the equal-depth fix-up, ping-ponging in
// global memory.
template <bool kBallotSmem>
__global__ void __launch_bounds__(kThreads, 4)
    k_tile_sort(uint64_t *low_keys, uint64_t *tmp, const uint32_t *__restrict__ ranges,
                const uint32_t *__restrict__ order, const int *__restrict__ misc, int n_tiles,
                uint32_t *__restrict__ values, uint64_t *__restrict__ keys_out, int rec_bits,
                const int32_t *__restrict__ status) {
    dep_wait();
    __shared__ uint64_t s_a[kSmemKeys], s_b[kSmemKeys];
    __shared__ uint32_t s_wh[kWarps][kRadix];
    __shared__ uint32_t s_warp[kWarps];
    __shared__ uint32_t s_mm[2][kWarps];
    if (!status_ok(status)) return;
    const int tid = threadIdx.x;
    const int n_large = order ? misc[1] : n_tiles;
    if ((int)blockIdx.x >= n_large) {  // one short tile per warp
        const int warp = tid >> 5;
        const int ti = n_large + ((int)blockIdx.x - n_large) * kWarps + warp;
        if (ti >= n_tiles) return;
        const int tile = (int)order[ti];
        const uint32_t s = ranges[2 * (size_t)tile], e = ranges[2 * (size_t)tile + 1];
        const int n = (int)(e - s);
        if (n <= 0) return;  // n is the same on the whole warp
        if (n <= 32) warp_sort_regs<1>(low_keys + s, n, values, keys_out, s, (uint32_t)tile);
        else if (n <= 64) warp_sort_regs<2>(low_keys + s, n, values, keys_out, s, (uint32_t)tile);
        else if (n <= 128) warp_sort_regs<4>(low_keys + s, n, values, keys_out, s, (uint32_t)tile);
        else warp_sort_regs<8>(low_keys + s, n, values, keys_out, s, (uint32_t)tile);
        return;
    }
    const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    const uint32_t s = ranges[2 * (size_t)tile], e = ranges[2 * (size_t)tile + 1];
    const int n = (int)(e - s);
    if (n <= 0) return;
    if (n > kRadixMinKeys && n <= kSmemKeys) {
        // LSD radix over the quantised depth in shared memory (2 passes of ~25
        // instructions per key against ~6 per key for each of the 45-66 stages
        // of a bitonic network), then the run fix-up. From 513 keys (with the
        // 4 passes over the depth bits of the build before):
        // above 1,024 only, tracking at 640x480 / 300k measured 0.6 us per
        // iteration slower (6,269 / 6,271 against 6,277 / 6,285 iterations/s,
        // same box); from 257 keys, slower again (6,240 / 6,258)
        for (int i = tid; i < n; i += kThreads) s_a[i] = low_keys[s + i];
        __syncthreads();
        const uint64_t *a = cta_sort_bucket<kBallotSmem>(s_a, s_b, n, rec_bits, s_wh, s_warp, s_mm);
        for (int i = tid; i < n; i += kThreads) {
            const uint64_t k = a[i];
            values[s + i] = (uint32_t)k;
            if (keys_out) keys_out[s + i] = ((uint64_t)tile << 32) | (k >> 32);
        }
        return;
    }
    if (n <= kSmemKeys) {
        int np = kThreads;
        while (np < n) np <<= 1;
        static_assert(kRadixMinKeys <= 2 * kThreads, "bitonic lists fit 2 keys per thread");
        if (np == kThreads)  // n <= kRadixMinKeys here
            cta_sort_regs<1>(low_keys + s, n, s_a);
        else
            cta_sort_regs<2>(low_keys + s, n, s_a);
        // cta_sort_regs leaves the sorted keys in s_a[0, n)
        for (int i = tid; i < n; i += kThreads) {
            const uint64_t k = s_a[i];
            values[s + i] = (uint32_t)k;
            if (keys_out) keys_out[s + i] = ((uint64_t)tile << 32) | (k >> 32);
        }
        return;
    }
    // large buckets ping-pong between their own slots and the same slots of tmp
    const uint64_t *a = cta_sort_bucket<true>(low_keys + s, tmp + s, n, rec_bits, s_wh, s_warp, s_mm);
    for (int i = tid; i < n; i += kThreads) {
        const uint64_t k = a[i];
        values[s + i] = (uint32_t)k;
        if (keys_out) keys_out[s + i] = ((uint64_t)tile << 32) | (k >> 32);
    }
}

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
    size_t low, tmp, misc, total;
};

WsLayout layout(int capacity) {
    WsLayout L;
    size_t o = 0;
    L.low = o; o += align256(sizeof(uint64_t) * (size_t)capacity);
    L.tmp = o; o += align256(sizeof(uint64_t) * (size_t)capacity);
    L.misc = o; o += align256(sizeof(int) * 16);
    L.total = o;
    return L;
}

int bit_width(unsigned x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

}  // namespace

size_t bin_workspace_bytes(int n_records, int capacity) {
    (void)n_records;
    return layout(capacity).total;
}

// Every (record, tile) pair adds to its tile's counter with an atomic, in the
// count (or the counting projection) and again in the fill, and the atomics on
// one line are executed one after another by the L2 slice that holds it.
// Packed next to each other (the end words of `ranges`), the ~1,200 counters
// of a 640x480 frame take 75 lines, and ncu showed one L2 slice's atomic unit
// busy for half of the fill while the average slice was at 2%. So the
// counters of a call with at most kCtrSpreadTiles tiles get a 128-byte line
// each (kCtrStride words apart) in the sort's ping-pong buffer, which is
// unused until the sort, when it has room for them: tracking at 640x480 /
// 300k measured 6,213 -> 6,267 iterations/s (same box, two runs each; 256
// words apart the same, 6,267). Batches of more tiles keep them in `ranges`:
// their counters already span hundreds of lines, and the 8-frame mapping
// window measured 2,418 -> 2,406 keyframe-iterations/s spread out.
constexpr int kCtrStride = 32;
constexpr int kCtrSpreadTiles = 4096;

TileCtr tile_counters(uint32_t *ranges, const FrameTable &ft, int capacity, void *ws) {
    const WsLayout L = layout(capacity);
    if (ft.total_tiles <= kCtrSpreadTiles &&
        (size_t)ft.total_tiles * kCtrStride * sizeof(uint32_t) <= sizeof(uint64_t) * (size_t)capacity)
        return TileCtr{reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + L.tmp), kCtrStride};
    return TileCtr{ranges + 1, 2};
}

cudaError_t launch_bin_clear(uint32_t *ranges, const FrameTable &ft, int capacity, void *ws, cudaStream_t s) {
    int *misc = reinterpret_cast<int *>(static_cast<char *>(ws) + layout(capacity).misc);
    const int n = ft.total_tiles;
    const int clear_grid = n > 0 ? min((n + kThreads - 1) / kThreads, 4 * device_sm_count()) : 1;
    return launch_chained(k_bin_clear, dim3(clear_grid), dim3(kThreads), 0, s, tile_counters(ranges, ft, capacity, ws),
                          n, misc);
}

cudaError_t launch_bin_tiles(const float *rec, const int *touched, int n_records, int n_per_frame,
                             const FrameTable &ft, int capacity, uint32_t *values, uint64_t *keys_out,
                             uint32_t *ranges, uint32_t *order, int32_t *status, void *ws, cudaStream_t s,
                             bool counted) {
    const WsLayout L = layout(capacity);
    char *w = static_cast<char *>(ws);
    uint64_t *low = reinterpret_cast<uint64_t *>(w + L.low);
    uint64_t *tmp = reinterpret_cast<uint64_t *>(w + L.tmp);
    int *misc = reinterpret_cast<int *>(w + L.misc);
    const TileCtr tc = tile_counters(ranges, ft, capacity, ws);
    // low key = depth bits << 32 | record index; only the index bits that can be set are sorted
    const int rec_bits = bit_width((unsigned)(n_records > 0 ? n_records - 1 : 0));
    cudaError_t err;
    if (!counted && (err = launch_bin_clear(ranges, ft, capacity, ws, s)) != cudaSuccess) return err;
    if (ft.total_tiles == 0) return cudaSuccess;
    const bool large = (long long)n_records >= (long long)kLargeBatchPerSm * device_sm_count();
    const int per_cta = kThreads * (large ? kRecLarge : 1);
    const int grid = n_records > 0 ? (int)(((size_t)n_records + per_cta - 1) / per_cta) : 1;
    auto count = large ? k_tile_count<kRecLarge> : k_tile_count<1>;
    auto fill = large ? k_tile_fill<kRecLarge> : k_tile_fill<1>;
    if (!counted && (err = launch_chained(count, dim3(grid), dim3(kThreads), 0, s, rec, touched, n_records, n_per_frame,
                                          ft, tc, status)) != cudaSuccess)
        return err;
    if ((err = launch_chained(k_tile_scan, dim3(1), dim3(kScanThreads), 0, s, ranges, tc, ft.total_tiles, capacity,
                              status, misc, order)) != cudaSuccess)
        return err;
    if ((err = launch_chained(fill, dim3(grid), dim3(kThreads), 0, s, rec, touched, n_records, n_per_frame, ft, tc, low,
                              capacity, status)) != cudaSuccess)
        return err;
    // Batches of more than kBallotSmemTiles tiles (multi-frame windows, the
    // 1200x680 frames) take ballot peers in the shared-memory passes too: with
    // them, mapping measured 2,532 -> 2,548 keyframe-iterations/s, uneven
    // 2,126 -> 2,135 frames/s and 5M tracking 577 -> 584 iterations/s, while the
    // 1,200-tile tracking frame lost 1.6 us of binning per iteration (peers8).
    auto sort = ft.total_tiles > kBallotSmemTiles ? k_tile_sort<true> : k_tile_sort<false>;
    if ((err = launch_chained(sort, dim3(ft.total_tiles), dim3(kThreads), 0, s, low, tmp, ranges, order, misc,
                              ft.total_tiles, values, keys_out, rec_bits, status)) != cudaSuccess)
        return err;
    return cudaGetLastError();
}

}  // namespace gs
