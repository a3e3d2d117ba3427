// EWA projection of 3D Gaussians (CG-SLAM Eq. 1-2) and its adjoint.
//
// k_project      one thread per (frame, Gaussian): activation, camera transform,
//                Jacobian with x/z, y/z clamp, dilated 2D covariance, conic,
//                centre, radius, pixel rect, tiles touched; in POSE mode also the
//                6x6 forward-mode derivative of (mean2d, conic, z) w.r.t. a left
//                se(3) perturbation of the pose.
// k_project_bwd  one thread per Gaussian, looping over frames: chains the
//                accumulated per-record 2D gradients to mean, log-scale,
//                quaternion, opacity logit, colour and nu (summed over frames,
//                no atomics) and writes one FP64 pose partial per (frame, CTA).
#include "gs_internal.cuh"
#include "pairs.cuh"
#include "dfloat.cuh"

namespace gs {
namespace {

constexpr int kProjThreads = 256;

// Parameter sources. Each has a per-Gaussian handle (`Rec`) and accessors that
// the projection calls in the same order for both storages.
//   F32Src   the FP32 arrays of gs_gaussians; the geometry inputs (quaternion,
//            mean, log-scales) are loaded up front in one round trip, opacity,
//            colour and nu lazily, so a culled Gaussian costs 40 of its 60
//            bytes. (Loading the log-scales only after the near-plane test cost
//            a second round trip: mapping projection 0.148 against 0.159 ms;
//            loading all 60 bytes up front, 0.171 ms.)
//   BF16Src  the packed 32-byte record of gs_gaussians_bf16, fetched whole (one
//            sector), plus its chunk's FP32 box: mean = lo + step * q (FP32
//            multiply, then add, each rounded); BF16 -> FP32 is exact (the bits
//            shifted up).
struct F32Src {
    GaussPtrs g;
    struct Rec {
        float4 q;
        float m[3], ls[3];
        int i;
    };
    __device__ __forceinline__ Rec fetch(int i) const {
        Rec r;
        r.i = i;
        r.q = __ldg(reinterpret_cast<const float4 *>(g.quats) + i);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            r.m[k] = __ldg(g.means + 3 * i + k);
            r.ls[k] = __ldg(g.log_scales + 3 * i + k);
        }
        return r;
    }
    __device__ __forceinline__ float4 quat(const Rec &r) const { return r.q; }
    __device__ __forceinline__ float mean(const Rec &r, int k) const { return r.m[k]; }
    __device__ __forceinline__ float log_scale(const Rec &r, int k) const { return r.ls[k]; }
    __device__ __forceinline__ float opacity_logit(const Rec &r) const { return __ldg(g.opacity_logit + r.i); }
    __device__ __forceinline__ float color(const Rec &r, int k) const { return __ldg(g.colors + 3 * r.i + k); }
    __device__ __forceinline__ float nu(const Rec &r) const { return __ldg(g.nu + r.i); }
};

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

struct BF16Src {
    const float4 *anchors;  // [ceil(n / GS_BF16_CHUNK)][2]: (lo xyz, step x), (step y, z, 0, 0)
    const uint4 *packed;    // [n][2]; h[16] = q xyz (uint16), then BF16 log-scale xyz, quat
                            // wxyz, logit, rgb, nu, 0; word k of the record holds h[2k]
                            // (low half) and h[2k+1] (high half)
    struct Rec {
        float4 box0, box1;
        uint4 a, b;
    };
    __device__ __forceinline__ Rec fetch(int i) const {
        Rec r;
        r.box0 = __ldg(anchors + 2 * (i / GS_BF16_CHUNK));
        r.box1 = __ldg(anchors + 2 * (i / GS_BF16_CHUNK) + 1);
        r.a = __ldg(packed + 2 * (size_t)i);
        r.b = __ldg(packed + 2 * (size_t)i + 1);
        return r;
    }
    __device__ __forceinline__ float4 quat(const Rec &r) const {
        return make_float4(bf_lo(r.a.w), bf_hi(r.a.w), bf_lo(r.b.x), bf_hi(r.b.x));
    }
    __device__ __forceinline__ float mean(const Rec &r, int k) const {
        const uint32_t q = k == 0 ? (r.a.x & 0xffffu) : (k == 1 ? (r.a.x >> 16) : (r.a.y & 0xffffu));
        const float lo = k == 0 ? r.box0.x : (k == 1 ? r.box0.y : r.box0.z);
        const float st = k == 0 ? r.box0.w : (k == 1 ? r.box1.x : r.box1.y);
        return __fadd_rn(lo, __fmul_rn(st, (float)q));
    }
    __device__ __forceinline__ float log_scale(const Rec &r, int k) const {
        return k == 0 ? bf_hi(r.a.y) : (k == 1 ? bf_lo(r.a.z) : bf_hi(r.a.z));
    }
    __device__ __forceinline__ float opacity_logit(const Rec &r) const { return bf_lo(r.b.y); }
    __device__ __forceinline__ float color(const Rec &r, int k) const {
        return k == 0 ? bf_hi(r.b.y) : (k == 1 ? bf_lo(r.b.z) : bf_hi(r.b.z));
    }
    __device__ __forceinline__ float nu(const Rec &r) const { return bf_lo(r.b.w); }
};

// Camera-space quantities of one Gaussian that both directions need.
struct Geo {
    float R[3][3];   // rotation of the normalised quaternion
    float qn[4];     // normalised quaternion (w,x,y,z)
    float qinv;      // 1/|q|
    float s[3];      // scales
    float WM[3][3];  // R_cw * R * diag(s)
    float V[3][3];   // camera-space covariance R_cw Sigma R_cw^T
    float p[3];      // camera-space centre
    float iz;        // 1/z
    float u, v;      // x/z, y/z (unclamped)
    float uc, vc;    // clamped values used in J
    bool clx, cly;
    float J00, J02, J11, J12;
    float a, b, c;   // dilated 2D covariance
    float A, B, C;   // conic
};

__device__ __forceinline__ void load_pose(const float *__restrict__ T, float W[3][3], float t[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        W[r][0] = __ldg(T + 4 * r + 0);
        W[r][1] = __ldg(T + 4 * r + 1);
        W[r][2] = __ldg(T + 4 * r + 2);
        t[r] = __ldg(T + 4 * r + 3);
    }
}

// Returns false if the Gaussian is culled before the 2D covariance step
// (zero quaternion, behind the near plane, nu cull, non-positive determinant).
template <class Src>
__device__ __forceinline__ bool geometry(const Src &src, const typename Src::Rec &G, const FrameDesc &fd,
                                         const float W[3][3], const float t[3], float jclamp, float nu_cull, Geo &o) {
    const float4 q = src.quat(G);
    const float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    const float mx = src.mean(G, 0), my = src.mean(G, 1), mz = src.mean(G, 2);
#pragma unroll
    for (int r = 0; r < 3; ++r) o.p[r] = fmaf(W[r][0], mx, fmaf(W[r][1], my, fmaf(W[r][2], mz, t[r])));
    if (!(n2 > 0.f)) return false;
    if (!(o.p[2] > fd.znear)) return false;
    if (nu_cull > 0.f && src.nu(G) > nu_cull) return false;

    o.qinv = rsqrtf(n2);
    const float w = q.x * o.qinv, x = q.y * o.qinv, y = q.z * o.qinv, z = q.w * o.qinv;
    o.qn[0] = w; o.qn[1] = x; o.qn[2] = y; o.qn[3] = z;
    o.R[0][0] = 1.f - 2.f * (y * y + z * z); o.R[0][1] = 2.f * (x * y - w * z); o.R[0][2] = 2.f * (x * z + w * y);
    o.R[1][0] = 2.f * (x * y + w * z); o.R[1][1] = 1.f - 2.f * (x * x + z * z); o.R[1][2] = 2.f * (y * z - w * x);
    o.R[2][0] = 2.f * (x * z - w * y); o.R[2][1] = 2.f * (y * z + w * x); o.R[2][2] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
    for (int k = 0; k < 3; ++k) o.s[k] = expf(src.log_scale(G, k));
    // WM = W R diag(s); V = WM WM^T is symmetric by construction
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            o.WM[r][k] = (W[r][0] * o.R[0][k] + W[r][1] * o.R[1][k] + W[r][2] * o.R[2][k]) * o.s[k];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) {
            const float v = o.WM[r][0] * o.WM[c][0] + o.WM[r][1] * o.WM[c][1] + o.WM[r][2] * o.WM[c][2];
            o.V[r][c] = v;
            o.V[c][r] = v;
        }
    o.iz = 1.f / o.p[2];
    o.u = o.p[0] * o.iz;
    o.v = o.p[1] * o.iz;
    o.uc = o.u;
    o.vc = o.v;
    o.clx = o.cly = false;
    if (jclamp > 0.f) {
        const float lx = jclamp * 0.5f * fd.W / fd.fx, ly = jclamp * 0.5f * fd.H / fd.fy;
        if (o.u < -lx) { o.uc = -lx; o.clx = true; }
        if (o.u > lx) { o.uc = lx; o.clx = true; }
        if (o.v < -ly) { o.vc = -ly; o.cly = true; }
        if (o.v > ly) { o.vc = ly; o.cly = true; }
    }
    o.J00 = fd.fx * o.iz;
    o.J02 = -fd.fx * o.uc * o.iz;
    o.J11 = fd.fy * o.iz;
    o.J12 = -fd.fy * o.vc * o.iz;
    // Sigma_2d = J V J^T (J has structural zeros J01 = J10 = 0) + 0.3 I
    const float P00 = o.V[0][0] * o.J00 + o.V[0][2] * o.J02, P01 = o.V[0][1] * o.J11 + o.V[0][2] * o.J12;
    const float P11 = o.V[1][1] * o.J11 + o.V[1][2] * o.J12;
    const float P20 = o.V[2][0] * o.J00 + o.V[2][2] * o.J02, P21 = o.V[2][1] * o.J11 + o.V[2][2] * o.J12;
    o.a = o.J00 * P00 + o.J02 * P20 + 0.3f;
    o.b = o.J00 * P01 + o.J02 * P21;
    o.c = o.J11 * P11 + o.J12 * P21 + 0.3f;
    const float det = o.a * o.c - o.b * o.b;
    if (!(det > 0.f)) return false;
    const float idet = 1.f / det;
    o.A = o.c * idet;
    o.B = -o.b * idet;
    o.C = o.a * idet;
    return true;
}

// A culled record gets only its empty rect (16 B of the 64): at 5M Gaussians
// most records are culled, and nothing reads their other fields.
__device__ __forceinline__ void write_culled(float *rec, int *touched, size_t r) {
    reinterpret_cast<int4 *>(rec + r * kRecFloats)[3] = make_int4(1, 1, 0, 0);
    touched[r] = 0;
}

// COUNT: the projection also counts the (record, tile) pairs of the visible
// records into the binning's tile counters (zeroed before the launch),
// with the same warp-balanced walk and warp-aggregated atomics as
// k_tile_count, so that the binning can skip its count pass. Every lane then
// stays to the end of the walk (no early return).
// Held to 64 registers (4 CTAs per SM; the Jacobian builds spill ~32 bytes):
// the kernel is bound by memory latency, and the extra CTA per SM measured
// 0.3% faster per tracking iteration and 0.5% at 5M Gaussians than 68-72
// registers at 3 CTAs per SM.
template <bool JAC, bool COUNT, class Src>
__global__ void __launch_bounds__(kProjThreads, 4)
    k_project(Src src, int n, FrameTable ft, const float *__restrict__ T_cw, float jclamp, float nu_cull,
              float *__restrict__ rec, int *__restrict__ touched, float *__restrict__ jac,
              TileCtr tc, const int32_t *__restrict__ status) {
    dep_wait();
    if (status[0] != 0) return;
    // frame fastest: the CTAs of one block of Gaussians for every frame are
    // launched together, so a batch's frames read the block's parameters from
    // DRAM once and from L2 after that (uneven 16-frame batch 2,006 -> 2,035
    // frames/s, mapping window 2,440 -> 2,454 keyframe-iterations/s, same box,
    // two runs each)
    const unsigned nf = (unsigned)ft.n;
    const int f = nf == 1u ? 0 : (int)(blockIdx.x % nf);
    const int i = (int)(nf == 1u ? blockIdx.x : blockIdx.x / nf) * kProjThreads + threadIdx.x;
    if (!COUNT && i >= n) return;
    const FrameDesc &fd = ft.f[f];
    const size_t r = (size_t)f * n + i;
    Geo o;
    typename Src::Rec G{};
    bool vis = false;
    float mx = 0.f, my = 0.f, rad = 0.f;
    int ix0 = 1, iy0 = 1, ix1 = 0, iy1 = 0;
    if (i < n) {
        float W[3][3], t[3];
        load_pose(T_cw + 12 * f, W, t);
        G = src.fetch(i);
        if (geometry(src, G, fd, W, t, jclamp, nu_cull, o)) {
            mx = fmaf(fd.fx, o.u, fd.cx);
            my = fmaf(fd.fy, o.v, fd.cy);
            const float half = 0.5f * (o.a - o.c);
            const float lam = 0.5f * (o.a + o.c) + sqrtf(fmaxf(half * half + o.b * o.b, 0.f));
            rad = ceilf(3.f * sqrtf(lam));
            const float x0 = fmaxf(0.f, ceilf(mx - 0.5f - rad)), x1 = fminf((float)(fd.W - 1), floorf(mx - 0.5f + rad));
            const float y0 = fmaxf(0.f, ceilf(my - 0.5f - rad)), y1 = fminf((float)(fd.H - 1), floorf(my - 0.5f + rad));
            if (x0 <= x1 && y0 <= y1) {
                vis = true;
                ix0 = (int)x0;
                ix1 = (int)x1;
                iy0 = (int)y0;
                iy1 = (int)y1;
            }
        }
        if (!vis) write_culled(rec, touched, r);
    }
    if (COUNT) {
        PairSrc ps{};
        ps.valid = vis;
        if (vis) {
            ps.t = tile_rect(make_int4(ix0, iy0, ix1, iy1), ft.tile, fd);
            ps.tile_off = fd.tile_off;
            ps.tiles_x = fd.tiles_x;
        }
        if (__any_sync(0xffffffffu, ps.valid))
            warp_for_each_pair(ps, [&](bool valid, int, int gt, uint32_t) { warp_claim<false>(valid, gt, tc); });
    }
    if (!vis) return;
    const int ts = ft.tile;
    touched[r] = (ix1 / ts - ix0 / ts + 1) * (iy1 / ts - iy0 / ts + 1);

    const float opac = 1.f / (1.f + expf(-src.opacity_logit(G)));
    float4 *out = reinterpret_cast<float4 *>(rec + r * kRecFloats);
    out[0] = make_float4(mx, my, o.A, o.B);
    out[1] = make_float4(o.C, opac, o.p[2], src.nu(G));
    out[2] = make_float4(src.color(G, 0), src.color(G, 1), src.color(G, 2), rad);
    reinterpret_cast<int4 *>(out)[3] = make_int4(ix0, iy0, ix1, iy1);

    if (JAC) {
        // Forward-mode derivative along each of the six directions of the left
        // perturbation: dp = rho (translation) or e_k x p (rotation), and for
        // rotations dV = [e_k]_x V - V [e_k]_x. Output row-major [theta][xi],
        // theta = (mx, my, A, B, C, z).
        const float fx = fd.fx, fy = fd.fy, iz = o.iz, iz2 = iz * iz;
        float J[6][6];
        // terms of dSigma_2d that come from dJ: E = dJ * P with P = V J^T
        const float P00 = o.V[0][0] * o.J00 + o.V[0][2] * o.J02, P01 = o.V[0][1] * o.J11 + o.V[0][2] * o.J12;
        const float P10 = o.V[1][0] * o.J00 + o.V[1][2] * o.J02, P11 = o.V[1][1] * o.J11 + o.V[1][2] * o.J12;
        const float P20 = o.V[2][0] * o.J00 + o.V[2][2] * o.J02, P21 = o.V[2][1] * o.J11 + o.V[2][2] * o.J12;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float dp[3];
            float dV[3][3];
            if (k < 3) {
                dp[0] = (k == 0); dp[1] = (k == 1); dp[2] = (k == 2);
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) dV[a][b] = 0.f;
            } else {
                const int e = k - 3;
                // e x p
                dp[0] = (e == 1) ? o.p[2] : (e == 2 ? -o.p[1] : 0.f);
                dp[1] = (e == 2) ? o.p[0] : (e == 0 ? -o.p[2] : 0.f);
                dp[2] = (e == 0) ? o.p[1] : (e == 1 ? -o.p[0] : 0.f);
                // K = [e]_x ; dV = K V - V K
                float K[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
                if (e == 0) { K[1][2] = -1.f; K[2][1] = 1.f; }
                if (e == 1) { K[0][2] = 1.f; K[2][0] = -1.f; }
                if (e == 2) { K[0][1] = -1.f; K[1][0] = 1.f; }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
                        dV[a][b] = K[a][0] * o.V[0][b] + K[a][1] * o.V[1][b] + K[a][2] * o.V[2][b] -
                                   (o.V[a][0] * K[0][b] + o.V[a][1] * K[1][b] + o.V[a][2] * K[2][b]);
            }
            const float dz = dp[2];
            const float dJ00 = -fx * dz * iz2, dJ11 = -fy * dz * iz2;
            const float dJ02 = o.clx ? fx * o.uc * dz * iz2 : fx * iz2 * (2.f * o.u * dz - dp[0]);
            const float dJ12 = o.cly ? fy * o.vc * dz * iz2 : fy * iz2 * (2.f * o.v * dz - dp[1]);
            const float E00 = dJ00 * P00 + dJ02 * P20, E01 = dJ00 * P01 + dJ02 * P21;
            const float E10 = dJ11 * P10 + dJ12 * P20, E11 = dJ11 * P11 + dJ12 * P21;
            // J dV J^T
            const float Q00 = o.J00 * o.J00 * dV[0][0] + 2.f * o.J00 * o.J02 * dV[0][2] + o.J02 * o.J02 * dV[2][2];
            const float Q01 = o.J00 * o.J11 * dV[0][1] + o.J00 * o.J12 * dV[0][2] + o.J02 * o.J11 * dV[2][1] +
                              o.J02 * o.J12 * dV[2][2];
            const float Q11 = o.J11 * o.J11 * dV[1][1] + 2.f * o.J11 * o.J12 * dV[1][2] + o.J12 * o.J12 * dV[2][2];
            const float S00 = 2.f * E00 + Q00, S01 = E01 + E10 + Q01, S11 = 2.f * E11 + Q11;
            // d(conic) = -M dSigma M, M = [[A, B], [B, C]]
            const float m00 = o.A * S00 + o.B * S01, m01 = o.A * S01 + o.B * S11;
            const float m10 = o.B * S00 + o.C * S01, m11 = o.B * S01 + o.C * S11;
            J[0][k] = fx * (dp[0] - o.u * dz) * iz;
            J[1][k] = fy * (dp[1] - o.v * dz) * iz;
            J[2][k] = -(m00 * o.A + m01 * o.B);
            J[3][k] = -(m00 * o.B + m01 * o.C);
            J[4][k] = -(m10 * o.B + m11 * o.C);
            J[5][k] = dz;
        }
        float4 *jo = reinterpret_cast<float4 *>(jac + r * kJacFloats);
#pragma unroll
        for (int q4 = 0; q4 < 9; ++q4) {
            const int e = 4 * q4;
            jo[q4] = make_float4(J[e / 6][e % 6], J[(e + 1) / 6][(e + 1) % 6], J[(e + 2) / 6][(e + 2) % 6],
                                 J[(e + 3) / 6][(e + 3) % 6]);
        }
    }
}

// ------------------------------------------------------------ adjoint
__global__ void __launch_bounds__(kProjThreads)
    k_project_bwd(GaussPtrs g, int n, FrameTable ft, const float *__restrict__ T_cw, float jclamp,
                  const int *__restrict__ touched, const float *__restrict__ grad2d, gs_grads out,
                  float *__restrict__ pose_partials, int per_frame, double *__restrict__ pose_grad,
                  unsigned *__restrict__ counters, const int32_t *__restrict__ status) {
    if (status[0] != 0) return;
    const int i = blockIdx.x * kProjThreads + threadIdx.x;
    const bool valid_i = i < n;
    float g_mean[3] = {0.f, 0.f, 0.f}, g_ls[3] = {0.f, 0.f, 0.f}, g_q[4] = {0.f, 0.f, 0.f, 0.f};
    float g_op = 0.f, g_col[3] = {0.f, 0.f, 0.f}, g_nu = 0.f;
    constexpr int NW = kProjThreads / 32;
    __shared__ df s_pf[GS_MAX_FRAMES][NW][6];  // per frame, per warp: pose sums
    __shared__ df s_red[kRedSlots][6];
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // frames in which this Gaussian was visible (tiles_touched > 0, i.e. a
    // non-empty rect): the counts of all frames are loaded up front, side by
    // side, rather than one round trip per frame. A warp's 32 counts of a frame
    // share one 128-byte line, where the records' rects took one 32-byte
    // sector per record (with the opacity below: mapping backward 1.768 ->
    // 1.737 ms, uneven 3.941 -> 3.816 ms, same box, two runs each).
    uint64_t live_mask = 0;
    if (valid_i) {
#pragma unroll 8
        for (int f = 0; f < ft.n; ++f)
            if (touched[(size_t)f * n + i] > 0) live_mask |= 1ull << f;
    }
    // sigmoid of the opacity logit, as the projection computed it for the
    // records (same expression), once per Gaussian instead of a record load per
    // frame
    const float opac = live_mask ? 1.f / (1.f + expf(-g.opacity_logit[i])) : 0.f;

    for (int f = 0; f < ft.n; ++f) {
        const FrameDesc &fd = ft.f[f];
        float pc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const size_t r = (size_t)f * n + i;
        const bool live = ((live_mask >> f) & 1ull) != 0;
        if (live) {
            float W[3][3], t[3];
            load_pose(T_cw + 12 * f, W, t);
            Geo o;
            const F32Src src{g};
            geometry(src, src.fetch(i), fd, W, t, jclamp, -1.f, o);  // same arithmetic as the forward
            const float *ga = grad2d + r * kGrad2d;
            const float gmx = ga[G_MX], gmy = ga[G_MY], gA = ga[G_CA], gB = ga[G_CB], gC = ga[G_CC];
            const float gz_dir = ga[G_Z];
            g_col[0] += ga[G_R]; g_col[1] += ga[G_G]; g_col[2] += ga[G_B];
            g_nu += ga[G_NU];
            g_op += ga[G_OP] * opac * (1.f - opac);

            // conic -> Sigma_2d: H2 = -M Gm M with Gm = [[gA, gB/2], [gB/2, gC]]
            const float hB = 0.5f * gB;
            const float n00 = o.A * gA + o.B * hB, n01 = o.A * hB + o.B * gC;
            const float n10 = o.B * gA + o.C * hB, n11 = o.B * hB + o.C * gC;
            const float H00 = -(n00 * o.A + n01 * o.B), H01 = -(n00 * o.B + n01 * o.C);
            const float H11 = -(n10 * o.B + n11 * o.C);
            // Sigma_2d = J V J^T: dL/dV = J^T H J, dL/dJ = 2 H J V
            float JV[2][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                JV[0][c] = o.J00 * o.V[0][c] + o.J02 * o.V[2][c];
                JV[1][c] = o.J11 * o.V[1][c] + o.J12 * o.V[2][c];
            }
            const float gJ00 = 2.f * (H00 * JV[0][0] + H01 * JV[1][0]);
            const float gJ02 = 2.f * (H00 * JV[0][2] + H01 * JV[1][2]);
            const float gJ11 = 2.f * (H01 * JV[0][1] + H11 * JV[1][1]);
            const float gJ12 = 2.f * (H01 * JV[0][2] + H11 * JV[1][2]);
            float Jm[2][3] = {{o.J00, 0.f, o.J02}, {0.f, o.J11, o.J12}};
            float HV[3][3];  // dL/dV = J^T H J (symmetric)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    HV[a][b] = Jm[0][a] * (H00 * Jm[0][b] + H01 * Jm[1][b]) + Jm[1][a] * (H01 * Jm[0][b] + H11 * Jm[1][b]);
            // camera-space centre
            const float fx = fd.fx, fy = fd.fy, iz = o.iz, iz2 = iz * iz;
            float gp0 = gmx * fx * iz, gp1 = gmy * fy * iz;
            float gp2 = gz_dir - gmx * fx * o.u * iz - gmy * fy * o.v * iz;
            gp2 += -(gJ00 * fx + gJ11 * fy) * iz2;
            if (o.clx) gp2 += gJ02 * fx * o.uc * iz2;
            else { gp0 += -gJ02 * fx * iz2; gp2 += gJ02 * 2.f * fx * o.u * iz2; }
            if (o.cly) gp2 += gJ12 * fy * o.vc * iz2;
            else { gp1 += -gJ12 * fy * iz2; gp2 += gJ12 * 2.f * fy * o.v * iz2; }
            // world mean: p = W X + t
#pragma unroll
            for (int k = 0; k < 3; ++k) g_mean[k] += W[0][k] * gp0 + W[1][k] * gp1 + W[2][k] * gp2;
            // V = (W M)(W M)^T with M = R diag(s): dL/d(WM) = 2 HV WM; dL/dM = W^T (that)
            float gWM[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    gWM[a][k] = 2.f * (HV[a][0] * o.WM[0][k] + HV[a][1] * o.WM[1][k] + HV[a][2] * o.WM[2][k]);
            float gM[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int k = 0; k < 3; ++k) gM[a][k] = W[0][a] * gWM[0][k] + W[1][a] * gWM[1][k] + W[2][a] * gWM[2][k];
            float gR[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int k = 0; k < 3; ++k) gR[a][k] = gM[a][k] * o.s[k];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                g_ls[k] += (gM[0][k] * o.R[0][k] + gM[1][k] * o.R[1][k] + gM[2][k] * o.R[2][k]) * o.s[k];
            const float w = o.qn[0], x = o.qn[1], y = o.qn[2], z = o.qn[3];
            const float gw = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
            const float gx = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] - w * gR[1][2] +
                                    z * gR[2][0] + w * gR[2][1] - 2.f * x * gR[2][2]);
            const float gy = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                                    w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
            const float gzq = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] -
                                     2.f * z * gR[1][1] + y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
            const float dot = gw * w + gx * x + gy * y + gzq * z;
            g_q[0] += (gw - w * dot) * o.qinv;
            g_q[1] += (gx - x * dot) * o.qinv;
            g_q[2] += (gy - y * dot) * o.qinv;
            g_q[3] += (gzq - z * dot) * o.qinv;
            // pose (left perturbation): rho = dL/dp, phi = p x dL/dp + 2 (Z12, Z20, Z01), Z = V H - H V
            pc[0] = gp0; pc[1] = gp1; pc[2] = gp2;
            pc[3] = o.p[1] * gp2 - o.p[2] * gp1;
            pc[4] = o.p[2] * gp0 - o.p[0] * gp2;
            pc[5] = o.p[0] * gp1 - o.p[1] * gp0;
            float Z[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    Z[a][b] = (o.V[a][0] * HV[0][b] + o.V[a][1] * HV[1][b] + o.V[a][2] * HV[2][b]) -
                              (HV[a][0] * o.V[0][b] + HV[a][1] * o.V[1][b] + HV[a][2] * o.V[2][b]);
            pc[3] += 2.f * Z[1][2];
            pc[4] += 2.f * Z[2][0];
            pc[5] += 2.f * Z[0][1];
        }
        // this warp's pose sum for frame f (double-float, fixed halving order);
        // the CTA combines the warps once, after the frame loop, so the loop
        // has no CTA barrier
        if (__any_sync(0xffffffffu, live)) {
            int slot;
            const df v = df_warp_sum6(pc, slot);
            if ((lane & 3) == 0 && slot < 6) s_pf[f][warp][slot] = v;
        } else if (lane < 6) {
            s_pf[f][warp][lane] = df{0.f, 0.f};
        }
    }
    // per-CTA pose partial of every frame (warps summed in order: the same
    // values as a per-frame CTA tree), then the last CTA reduces all frames
    __syncthreads();
    for (int e = threadIdx.x; e < ft.n * 6; e += kProjThreads) {
        const int f = e / 6, k = e % 6;
        df sum = {0.f, 0.f};
        for (int w = 0; w < NW; ++w) sum = df_add(sum, s_pf[f][w][k]);
        reinterpret_cast<float2 *>(pose_partials + ((size_t)f * per_frame + blockIdx.x) * 12)[k] =
            make_float2(sum.hi, sum.lo);
    }
    if (pose_grad) {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_flag = (atomicInc(counters, gridDim.x - 1) == gridDim.x - 1);  // wraps to 0
        __syncthreads();
        if (s_flag) {
            __threadfence();
            for (int f = 0; f < ft.n; ++f) {
                reduce_pose_partials(pose_partials + (size_t)f * per_frame * 12, per_frame, pose_grad + 6 * f, s_red);
                __syncthreads();  // s_red is reused by the next frame
            }
        }
    }
    if (!valid_i) return;
    if (out.means) for (int k = 0; k < 3; ++k) out.means[3 * i + k] = g_mean[k];
    if (out.log_scales) for (int k = 0; k < 3; ++k) out.log_scales[3 * i + k] = g_ls[k];
    if (out.quats) for (int k = 0; k < 4; ++k) out.quats[4 * i + k] = g_q[k];
    if (out.opacity_logit) out.opacity_logit[i] = g_op;
    if (out.colors) for (int k = 0; k < 3; ++k) out.colors[3 * i + k] = g_col[k];
    if (out.nu) out.nu[i] = g_nu;
}

}  // namespace

template <class Src>
cudaError_t launch_src(const Src &src, int n, const FrameTable &ft, const float *T_cw, float jclamp, float nu_cull,
                       int mode, float *rec, int *touched, float *jac, TileCtr tc, const int32_t *status,
                       cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)((n + kProjThreads - 1) / kProjThreads) * (unsigned)ft.n);
    const dim3 block(kProjThreads);
    const bool jacob = mode == GS_MODE_POSE;
    if (tc.p)
        return jacob ? launch_chained(k_project<true, true, Src>, grid, block, 0, s, src, n, ft, T_cw, jclamp, nu_cull,
                                      rec, touched, jac, tc, status)
                     : launch_chained(k_project<false, true, Src>, grid, block, 0, s, src, n, ft, T_cw, jclamp, nu_cull,
                                      rec, touched, jac, tc, status);
    return jacob ? launch_chained(k_project<true, false, Src>, grid, block, 0, s, src, n, ft, T_cw, jclamp, nu_cull,
                                  rec, touched, jac, tc, status)
                 : launch_chained(k_project<false, false, Src>, grid, block, 0, s, src, n, ft, T_cw, jclamp, nu_cull,
                                  rec, touched, jac, tc, status);
}

cudaError_t launch_project(const GaussPtrs &g, int n, const FrameTable &ft, const float *T_cw, float jclamp,
                           float nu_cull, int mode, float *rec, int *touched, float *jac, TileCtr tile_counts,
                           const int32_t *status, cudaStream_t s) {
    return launch_src(F32Src{g}, n, ft, T_cw, jclamp, nu_cull, mode, rec, touched, jac, tile_counts, status, s);
}

cudaError_t launch_project_bf16(const float *anchors, const uint16_t *packed, int n, const FrameTable &ft,
                                const float *T_cw, float jclamp, float nu_cull, int mode, float *rec, int *touched,
                                float *jac, TileCtr tile_counts, const int32_t *status, cudaStream_t s) {
    const BF16Src src{reinterpret_cast<const float4 *>(anchors), reinterpret_cast<const uint4 *>(packed)};
    return launch_src(src, n, ft, T_cw, jclamp, nu_cull, mode, rec, touched, jac, tile_counts, status, s);
}

cudaError_t launch_project_bwd(const GaussPtrs &g, int n, const FrameTable &ft, const float *T_cw, float jclamp,
                               const int *touched, const float *grad2d, gs_grads grads, float *pose_partials,
                               int per_frame, double *pose_grad, unsigned *counters, const int32_t *status,
                               cudaStream_t s) {
    dim3 grid(per_frame);  // ceil(n / 256), at least one CTA so the frame's pose gradient is written
    k_project_bwd<<<grid, kProjThreads, 0, s>>>(g, n, ft, T_cw, jclamp, touched, grad2d, grads, pose_partials,
                                                per_frame, pose_grad, counters, status);
    return cudaGetLastError();
}

}  // namespace gs
