// Tile binning: the "pre-sort of all visible Gaussians from near to far" of
// CG-SLAM Sec. 3.1, done per tile.
//
//   k_count / k_scan_top   exclusive scan of tiles_touched over the records
//                          (fixed grid of 4 CTAs per SM, each owning a contiguous
//                          slice), total pair count P and the capacity check.
//   k_emit                 one (key, record) pair per overlapped tile,
//                          key = (global tile id << 32) | float bits of depth.
//   k_radix_hist / k_radix_scan / k_radix_scatter
//                          one stable LSD pass per 8-bit digit over only the key
//                          bits that can be non-zero (32 depth bits + the bits of
//                          the largest tile id). Each pass: per-CTA digit counts
//                          (digit-major, so one flat exclusive scan yields every
//                          CTA's output offsets), then a scatter whose in-CTA
//                          ranks come from __match_any_sync peer groups processed
//                          in input order -- the order of equal keys is preserved,
//                          so the output is bit-exact regardless of the grid.
//   k_ranges               [start, end) of every tile from the sorted keys.
#include <climits>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kScanTopThreads = 1024;
static_assert(kScanBlocks <= kScanTopThreads, "top-level scan handles one value per thread");
static_assert((kRadix * kSortBlocks) % (kScanTopThreads * 4) == 0, "digit scan uses uint4 chunks");

__device__ __forceinline__ void slice(long long total, int b, int nb, long long &lo, long long &hi) {
    lo = total * b / nb;
    hi = total * (b + 1) / nb;
}

// Exclusive block scan of one int per thread (256 threads); returns the block total.
__device__ __forceinline__ int block_excl_scan(int v, int &total, int *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    int wpre = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const int s = s_warp[w];
        wpre += (w < warp) ? s : 0;
        total += s;
    }
    __syncthreads();
    return wpre + x - v;
}

__global__ void __launch_bounds__(kThreads)
    k_count(const int *__restrict__ touched, int M, long long *__restrict__ sums, const int32_t *__restrict__ status) {
    __shared__ long long s_w[kWarps];
    if (status[0] != 0) return;
    long long lo, hi;
    slice(M, blockIdx.x, gridDim.x, lo, hi);
    long long acc = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += kThreads) acc += touched[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < kWarps; ++w) t += s_w[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanTopThreads)
    k_scan_top(long long *__restrict__ sums, int nb, int capacity, int32_t *__restrict__ status,
               int *__restrict__ misc) {
    __shared__ long long s_w[kScanTopThreads / 32];
    if (status[0] != 0) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long v = t < nb ? sums[t] : 0;
    long long x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    long long wpre = 0, total = 0;
    for (int w = 0; w < kScanTopThreads / 32; ++w) {
        wpre += (w < warp) ? s_w[w] : 0;
        total += s_w[w];
    }
    if (t < nb) sums[t] = wpre + x - v;
    if (t == 0) {
        status[1] = (int32_t)(total > INT_MAX ? INT_MAX : total);
        if (total > capacity) status[0] = GS_ERR_CAPACITY;
        misc[0] = (int)(total > capacity ? capacity : total);
    }
}

__global__ void __launch_bounds__(kThreads)
    k_emit(const float *__restrict__ rec, const int *__restrict__ touched, int M, int n_per_frame, FrameTable ft,
           const long long *__restrict__ offs, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
           const int32_t *__restrict__ status) {
    __shared__ int s_warp[kWarps];
    if (status[0] != 0) return;
    long long lo, hi;
    slice(M, blockIdx.x, gridDim.x, lo, hi);
    long long run = offs[blockIdx.x];
    const int ts = ft.tile;
    for (long long base = lo; base < hi; base += kThreads) {
        const long long i = base + threadIdx.x;
        const int t = i < hi ? touched[i] : 0;
        int total;
        const int ex = block_excl_scan(t, total, s_warp);
        if (t > 0) {
            const int f = (int)(i / n_per_frame);
            const FrameDesc &fd = ft.f[f];
            const float *R = rec + (size_t)i * kRecFloats;
            const int4 rc = *reinterpret_cast<const int4 *>(R + R_X0);
            const uint32_t zb = __float_as_uint(R[R_Z]);
            long long o = run + ex;
            const long long o_end = o + t;  // never write more than this record's scanned count
            const int ty1 = min(rc.w / ts, fd.tiles_y - 1), tx1 = min(rc.z / ts, fd.tiles_x - 1);
            for (int ty = max(rc.y, 0) / ts; ty <= ty1; ++ty)
                for (int tx = max(rc.x, 0) / ts; tx <= tx1 && o < o_end; ++tx) {
                    const uint32_t tile = (uint32_t)(fd.tile_off + ty * fd.tiles_x + tx);
                    keys[o] = ((uint64_t)tile << 32) | zb;
                    vals[o] = (uint32_t)i;
                    ++o;
                }
        }
        run += total;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_radix_hist(const uint64_t *__restrict__ keys, int shift, uint32_t *__restrict__ hist,
                 const int *__restrict__ misc, const int32_t *__restrict__ status) {
    __shared__ uint32_t h[kRadix];
    if (status[0] != 0) return;
    long long lo, hi;
    slice(misc[0], blockIdx.x, gridDim.x, lo, hi);
    h[threadIdx.x] = 0;
    __syncthreads();
    for (long long i = lo + threadIdx.x; i < hi; i += kThreads)
        atomicAdd(&h[(uint32_t)(keys[i] >> shift) & (kRadix - 1)], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of the digit-major [256][NB] count matrix, in place.
__global__ void __launch_bounds__(kScanTopThreads)
    k_radix_scan(uint32_t *__restrict__ hist, int n, const int32_t *__restrict__ status) {
    __shared__ uint32_t s_w[kScanTopThreads / 32];
    if (status[0] != 0) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = n / kScanTopThreads;  // multiple of 4
    uint4 *p = reinterpret_cast<uint4 *>(hist + (size_t)t * per);
    uint32_t local = 0;
    for (int q = 0; q < per / 4; ++q) {
        const uint4 v = p[q];
        local += v.x + v.y + v.z + v.w;
    }
    uint32_t x = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    uint32_t run = x - local;
    for (int w = 0; w < warp; ++w) run += s_w[w];
    for (int q = 0; q < per / 4; ++q) {
        uint4 v = p[q];
        uint4 o;
        o.x = run; run += v.x;
        o.y = run; run += v.y;
        o.z = run; run += v.z;
        o.w = run; run += v.w;
        p[q] = o;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                    uint32_t *__restrict__ vout, int shift, const uint32_t *__restrict__ hist,
                    const int *__restrict__ misc, const int32_t *__restrict__ status) {
    __shared__ uint32_t run[kRadix];
    __shared__ uint32_t wh[kWarps][kRadix];
    if (status[0] != 0) return;
    long long lo, hi;
    slice(misc[0], blockIdx.x, gridDim.x, lo, hi);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = hist[(size_t)tid * gridDim.x + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (long long base = lo; base < hi; base += kThreads) {
        const long long i = base + tid;
        const bool active = i < hi;
        const uint64_t key = active ? kin[i] : 0ull;
        const uint32_t val = active ? vin[i] : 0u;
        const uint32_t d = active ? ((uint32_t)(key >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        __syncthreads();  // previous chunk finished reading wh
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wh[w][tid] = 0;
        __syncthreads();
        if (active && rank == 0) wh[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t r = run[tid];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = wh[w][tid];
                wh[w][tid] = r;
                r += c;
            }
            run[tid] = r;
        }
        __syncthreads();
        if (active) {
            const uint32_t pos = wh[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
    }
}

__global__ void __launch_bounds__(kThreads)
    k_ranges(const uint64_t *__restrict__ keys, uint32_t *__restrict__ ranges, const int *__restrict__ misc,
             const int32_t *__restrict__ status) {
    if (status[0] != 0) return;
    const long long P = misc[0];
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < P; i += (long long)gridDim.x * kThreads) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[2 * (size_t)t] = (uint32_t)i;
        if (i == P - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[2 * (size_t)t + 1] = (uint32_t)(i + 1);
    }
}

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
    size_t keys_a, keys_b, vals_b, hist, sums, misc, total;
};

WsLayout layout(int capacity) {
    WsLayout L;
    size_t o = 0;
    L.keys_a = o; o += align256(sizeof(uint64_t) * (size_t)capacity);
    L.keys_b = o; o += align256(sizeof(uint64_t) * (size_t)capacity);
    L.vals_b = o; o += align256(sizeof(uint32_t) * (size_t)capacity);
    L.hist = o; o += align256(sizeof(uint32_t) * (size_t)kRadix * kSortBlocks);
    L.sums = o; o += align256(sizeof(long long) * (size_t)kScanBlocks);
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

cudaError_t launch_bin_tiles(const float *rec, const int *touched, int n_records, int n_per_frame,
                             const FrameTable &ft, int capacity, uint32_t *values, uint64_t *keys_out,
                             uint32_t *ranges, int32_t *status, void *ws, cudaStream_t s) {
    const WsLayout L = layout(capacity);
    char *w = static_cast<char *>(ws);
    uint64_t *K[2] = {keys_out ? keys_out : reinterpret_cast<uint64_t *>(w + L.keys_a),
                      reinterpret_cast<uint64_t *>(w + L.keys_b)};
    uint32_t *V[2] = {values, reinterpret_cast<uint32_t *>(w + L.vals_b)};
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + L.hist);
    long long *sums = reinterpret_cast<long long *>(w + L.sums);
    int *misc = reinterpret_cast<int *>(w + L.misc);

    const int key_bits = 32 + bit_width((unsigned)(ft.total_tiles > 0 ? ft.total_tiles - 1 : 0));
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    const int e = passes & 1;

    cudaError_t err;
    if ((err = cudaMemsetAsync(misc, 0, sizeof(int) * 16, s)) != cudaSuccess) return err;
    k_count<<<kScanBlocks, kThreads, 0, s>>>(touched, n_records, sums, status);
    k_scan_top<<<1, kScanTopThreads, 0, s>>>(sums, kScanBlocks, capacity, status, misc);
    k_emit<<<kScanBlocks, kThreads, 0, s>>>(rec, touched, n_records, n_per_frame, ft, sums, K[e], V[e], status);
    for (int p = 0; p < passes; ++p) {
        const int src = (e + p) & 1, dst = (e + p + 1) & 1;
        const int shift = p * kRadixBits;
        k_radix_hist<<<kSortBlocks, kThreads, 0, s>>>(K[src], shift, hist, misc, status);
        k_radix_scan<<<1, kScanTopThreads, 0, s>>>(hist, kRadix * kSortBlocks, status);
        k_radix_scatter<<<kSortBlocks, kThreads, 0, s>>>(K[src], V[src], K[dst], V[dst], shift, hist, misc, status);
    }
    if ((err = cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)ft.total_tiles, s)) != cudaSuccess)
        return err;
    k_ranges<<<kScanBlocks, kThreads, 0, s>>>(K[0], ranges, misc, status);
    return cudaGetLastError();
}

}  // namespace gs
