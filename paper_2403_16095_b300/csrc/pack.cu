// 16-bit storage of the Gaussians: BF16 attributes, and means as 16-bit
// fixed-point offsets inside a per-chunk FP32 box; plus the spatial order that
// makes those boxes small.
//
// A plain BF16 mean at 5-10 m from the origin is quantised in steps of 2-4 cm,
// coarser than the Gaussians themselves (a few cm); a BF16 offset from a chunk
// anchor is only as fine as 2^-8 of the offset, and a Morton-ordered chunk that
// straddles two octants can span the whole scene. A 16-bit fixed-point offset
// over the chunk's own bounding box has a uniform step of extent / 65535: about
// 1 um for a compact chunk, below 0.1 mm even for a chunk spanning 10 m.
//
// k_bbox_partial / k_morton   per-block min/max of the means, reduced again by
//                             every block of the second kernel (a few hundred
//                             entries), then a 30-bit Morton code per Gaussian:
//                             q = min(1023, floor((m - lo) * (1024 / (hi - lo))))
//                             per axis in FP32 round-to-nearest, bits
//                             interleaved x, y, z from the lowest bit up. Key =
//                             code << 32 | index.
// k_radix_hist / k_radix_scan / k_radix_scatter
//                             a stable LSD radix sort of the keys over the code
//                             bits (8-bit digits, four passes): per-block digit
//                             histograms, one exclusive scan in digit-major
//                             order, then each block scatters its items in
//                             order. Deterministic: perm = the index order of
//                             the sorted keys (ties by index).
// k_pack_bf16                 one CTA per chunk: the chunk's bounding box gives
//                             lo and step = (hi - lo) / 65535 per axis (FP32);
//                             q = rint((m - lo) / step) in [0, 65535]; the
//                             other attributes are rounded to BF16 (nearest,
//                             ties to even); 32 bytes per Gaussian.
#include <cuda_bf16.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                       // items per thread in the radix passes
constexpr int kTileItems = kThreads * kItems;  // items per block
constexpr int kBoxBlocks = 296;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// CTA-wide min (k < 3) / max (k >= 3) of six values; every thread gets the result.
__device__ void cta_minmax6(float v[6], float (*s)[6]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = k < 3 ? warp_min(v[k]) : warp_max(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) s[warp][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float r = s[0][k];
        for (int w = 1; w < kWarps; ++w) r = k < 3 ? fminf(r, s[w][k]) : fmaxf(r, s[w][k]);
        v[k] = r;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
    k_bbox_partial(const float *__restrict__ means, int n, float *__restrict__ part, const int32_t *__restrict__ status) {
    __shared__ float s[kWarps][6];
    if (status[0] != 0) return;
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float m = means[3 * (size_t)i + k];
            v[k] = fminf(v[k], m);
            v[3 + k] = fmaxf(v[3 + k], m);
        }
    cta_minmax6(v, s);
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = v[threadIdx.x];
}

// spreads the low 10 bits of v to every third bit
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t quant10(float m, float lo, float scale) {
    if (!(scale > 0.f)) return 0u;  // degenerate axis (all equal)
    const float q = __fmul_rn(__fsub_rn(m, lo), scale);
    return q >= 1023.f ? 1023u : (uint32_t)q;  // q >= 0: truncation is floor
}

__global__ void __launch_bounds__(kThreads)
    k_morton(const float *__restrict__ means, int n, const float *__restrict__ part, int n_part,
             uint64_t *__restrict__ keys, const int32_t *__restrict__ status) {
    __shared__ float s[kWarps][6];
    if (status[0] != 0) return;
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int j = threadIdx.x; j < n_part; j += kThreads)
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = k < 3 ? fminf(v[k], part[6 * j + k]) : fmaxf(v[k], part[6 * j + k]);
    cta_minmax6(v, s);
    float sc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ext = __fsub_rn(v[3 + k], v[k]);
        sc[k] = ext > 0.f ? __fdiv_rn(1024.f, ext) : 0.f;
    }
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const size_t b = 3 * (size_t)i;
        const uint32_t code = spread3(quant10(means[b], v[0], sc[0])) | (spread3(quant10(means[b + 1], v[1], sc[1])) << 1) |
                              (spread3(quant10(means[b + 2], v[2], sc[2])) << 2);
        keys[i] = ((uint64_t)code << 32) | (uint32_t)i;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_radix_hist(const uint64_t *__restrict__ src, int n, int shift, uint32_t *__restrict__ hist, int nb,
                 const int32_t *__restrict__ status) {
    __shared__ uint32_t s_cnt[256];
    if (status[0] != 0) return;
    s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kTileItems;
    for (int r = 0; r < kItems; ++r) {
        const int i = base + r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_cnt[(uint32_t)(src[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = s_cnt[threadIdx.x];
}

// exclusive scan of `total` counters in place by one CTA: thread t owns a
// contiguous segment, segment sums are scanned across the CTA
__global__ void __launch_bounds__(kScanThreads)
    k_radix_scan(uint32_t *__restrict__ hist, int total, const int32_t *__restrict__ status) {
    __shared__ uint32_t s_warp[kScanThreads / 32];
    if (status[0] != 0) return;
    const int seg = (total + kScanThreads - 1) / kScanThreads;
    const int b = threadIdx.x * seg, e = min(total, b + seg);
    uint32_t sum = 0;
    for (int i = b; i < e; ++i) sum += hist[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre += s_warp[w];
    uint32_t run = pre + x - sum;
    for (int i = b; i < e; ++i) {
        const uint32_t c = hist[i];
        hist[i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_radix_scatter(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, int n, int shift,
                    const uint32_t *__restrict__ hist, int nb, const int32_t *__restrict__ status) {
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_wh[kWarps][256];
    if (status[0] != 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_off[tid] = hist[(size_t)tid * nb + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int base = blockIdx.x * kTileItems;
    for (int r = 0; r < kItems; ++r) {
        const int i = base + r * kThreads + tid;
        const bool active = i < n;
        const uint64_t key = active ? src[i] : 0ull;
        const uint32_t d = active ? ((uint32_t)(key >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        __syncthreads();  // previous round done with s_wh / s_off
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s_wh[w][tid] = 0;
        __syncthreads();
        if (active && rank == 0) s_wh[warp][d] = __popc(peers);
        __syncthreads();
        {  // digit tid: per-warp start offsets in warp order, then advance
            uint32_t o = s_off[tid];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = s_wh[w][tid];
                s_wh[w][tid] = o;
                o += c;
            }
            s_off[tid] = o;
        }
        __syncthreads();
        if (active) dst[s_wh[warp][d] + rank] = key;
    }
}

__global__ void k_keys_to_perm(const uint64_t *__restrict__ keys, int n, uint32_t *__restrict__ perm,
                               const int32_t *__restrict__ status) {
    if (status[0] != 0) return;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) perm[i] = (uint32_t)keys[i];
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) { return bf16_bits(lo) | (bf16_bits(hi) << 16); }

__device__ __forceinline__ uint32_t quant16(float m, float lo, float step) {
    if (!(step > 0.f)) return 0u;
    const float t = __fdiv_rn(__fsub_rn(m, lo), step);
    const int q = __float2int_rn(t);  // nearest, ties to even
    return (uint32_t)min(65535, max(0, q));
}

__global__ void __launch_bounds__(kThreads)
    k_pack_bf16(GaussPtrs g, int n, const uint32_t *__restrict__ perm, float4 *__restrict__ anchors,
                uint4 *__restrict__ packed, const int32_t *__restrict__ status) {
    static_assert(GS_BF16_CHUNK == kThreads, "one thread per Gaussian of a chunk");
    __shared__ float s[kWarps][6];
    if (status[0] != 0) return;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const bool valid = j < n;
    const int i = valid ? (perm ? (int)perm[j] : j) : 0;
    float m[3] = {0.f, 0.f, 0.f};
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    if (valid)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            m[k] = g.means[3 * (size_t)i + k];
            v[k] = v[3 + k] = m[k];
        }
    cta_minmax6(v, s);
    float st[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) st[k] = __fdiv_rn(__fsub_rn(v[3 + k], v[k]), 65535.f);
    if (threadIdx.x == 0) {
        anchors[2 * blockIdx.x] = make_float4(v[0], v[1], v[2], st[0]);
        anchors[2 * blockIdx.x + 1] = make_float4(st[1], st[2], 0.f, 0.f);
    }
    if (!valid) return;
    const float *ls = g.log_scales + 3 * (size_t)i;
    const float4 q = reinterpret_cast<const float4 *>(g.quats)[i];
    const float *c = g.colors + 3 * (size_t)i;
    uint4 A, B;
    A.x = quant16(m[0], v[0], st[0]) | (quant16(m[1], v[1], st[1]) << 16);
    A.y = quant16(m[2], v[2], st[2]) | (bf16_bits(ls[0]) << 16);
    A.z = pack2(ls[1], ls[2]);
    A.w = pack2(q.x, q.y);
    B.x = pack2(q.z, q.w);
    B.y = pack2(g.opacity_logit[i], c[0]);
    B.z = pack2(c[1], c[2]);
    B.w = pack2(g.nu[i], 0.f);
    packed[2 * (size_t)j] = A;
    packed[2 * (size_t)j + 1] = B;
}

int blocks_for(long long items, int cap) {
    const long long b = (items + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct OrderWs {
    size_t a, b, hist, part, total;
};
OrderWs order_layout(int n) {
    OrderWs L;
    const size_t nb = ((size_t)n + kTileItems - 1) / kTileItems;
    size_t o = 0;
    L.a = o; o += align256(sizeof(uint64_t) * (size_t)n);
    L.b = o; o += align256(sizeof(uint64_t) * (size_t)n);
    L.hist = o; o += align256(sizeof(uint32_t) * 256 * (nb > 0 ? nb : 1));
    L.part = o; o += align256(sizeof(float) * 6 * kBoxBlocks);
    L.total = o;
    return L;
}

}  // namespace

size_t spatial_order_workspace_bytes(int n) { return order_layout(n).total; }

cudaError_t launch_spatial_order(const float *means, int n, uint32_t *perm, void *ws, const int32_t *status,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const OrderWs L = order_layout(n);
    char *w = static_cast<char *>(ws);
    uint64_t *a = reinterpret_cast<uint64_t *>(w + L.a);
    uint64_t *b = reinterpret_cast<uint64_t *>(w + L.b);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + L.hist);
    float *part = reinterpret_cast<float *>(w + L.part);
    const int nbox = blocks_for(n, kBoxBlocks);
    k_bbox_partial<<<nbox, kThreads, 0, s>>>(means, n, part, status);
    k_morton<<<blocks_for(n, 8 * device_sm_count()), kThreads, 0, s>>>(means, n, part, nbox, a, status);
    const int nb = (n + kTileItems - 1) / kTileItems;
    for (int shift = 32; shift < 64; shift += 8) {  // the 30 code bits; ties keep index order
        k_radix_hist<<<nb, kThreads, 0, s>>>(a, n, shift, hist, nb, status);
        k_radix_scan<<<1, kScanThreads, 0, s>>>(hist, 256 * nb, status);
        k_radix_scatter<<<nb, kThreads, 0, s>>>(a, b, n, shift, hist, nb, status);
        uint64_t *t = a;
        a = b;
        b = t;
    }
    k_keys_to_perm<<<blocks_for(n, 8 * device_sm_count()), kThreads, 0, s>>>(a, n, perm, status);
    return cudaGetLastError();
}

cudaError_t launch_pack_bf16(const GaussPtrs &g, int n, const uint32_t *perm, float *anchors, uint16_t *packed,
                             const int32_t *status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int chunks = (n + GS_BF16_CHUNK - 1) / GS_BF16_CHUNK;
    k_pack_bf16<<<chunks, kThreads, 0, s>>>(g, n, perm, reinterpret_cast<float4 *>(anchors),
                                            reinterpret_cast<uint4 *>(packed), status);
    return cudaGetLastError();
}

}  // namespace gs
