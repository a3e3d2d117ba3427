// Per-pixel blending arithmetic shared by the forward and backward kernels.
//
// Both passes must take bit-identical decisions (footprint, alpha threshold,
// clamp, stop), so q, G and alpha are computed here with explicitly rounded
// operations that the compiler cannot contract differently per call site.
#pragma once

#include <cuda_runtime.h>

namespace gs {

constexpr float kTMin = 1e-4f;          // stop before T would drop below this
constexpr float kAlphaMin = 1.f / 255.f; // entries below are skipped
constexpr float kAlphaMax = 0.99f;      // alpha clamp
constexpr float kQMax = 9.f;            // footprint: q <= 9 (3 sigma)

// a = (mx, my, A, B), b = (C, opacity, z, nu). Returns false if the Gaussian does
// not contribute (q > 9 or alpha < 1/255); otherwise G = exp(-q/2),
// sg = opacity * G and alpha = min(0.99, sg). The exponential is taken for
// every lane, with no exit at q > 9, so that a warp's lanes stay on one path
// (a NaN q fails the q test whatever alpha becomes).
//
// A Gaussian is in a pixel's list iff the pixel lies in its rect and q <= 9.
// The blend kernels test only q <= 9 on the entries of the pixel's tile list:
// the rect contains the q <= 9 ellipse, since over a pixel offset (dx, dy)
// q >= dx^2 / S_xx >= dx^2 / lambda_max for the dilated 2D covariance S (and
// likewise in y), while the rect's half-width r = ceil(3 sqrt(lambda_max)).
// In FP32 the two tests can disagree only where q is within ~1e-6 (relative)
// of 9 and r within as much of 3 sqrt(S_xx), a threshold decision like the
// FP32 footprint test itself.
__device__ __forceinline__ bool eval_alpha(float pxc, float pyc, const float4 &a, const float4 &b, float &dx,
                                           float &dy, float &G, float &sg, float &alpha) {
    dx = __fsub_rn(pxc, a.x);
    dy = __fsub_rn(pyc, a.y);
    const float cross = __fmul_rn(__fmul_rn(2.f, a.w), __fmul_rn(dx, dy));
    const float q = __fmaf_rn(__fmul_rn(a.z, dx), dx, __fmaf_rn(__fmul_rn(b.x, dy), dy, cross));
    G = __expf(__fmul_rn(-0.5f, q));
    sg = __fmul_rn(b.y, G);
    alpha = fminf(kAlphaMax, sg);
    return (q <= kQMax) & (alpha >= kAlphaMin);
}

// Conservative test: can the Gaussian (a, b, rect rc) be blended by any pixel
// of the warp's 8x4 block whose pixel centres span [wx0+.5, wx0+7.5] x
// [wy0+.5, wy0+3.5]? False only if the block misses the pixel rect, or if the
// minimum of q over the block rectangle exceeds 9 by a slack that bounds the
// FP32 rounding of both this evaluation and the per-pixel one (relative to the
// magnitudes of the three terms of q, which can cancel for long, thin
// footprints). q is convex, so with the centre outside the block its minimum
// lies on an edge: each edge is minimised in closed form and clamped. Culled
// entries would be rejected by every pixel of the block, so per-pixel results
// are unchanged.
__device__ __forceinline__ float q_slack(float A, float B, float C, float dx, float dy) {
    const float t1 = A * dx * dx, t2 = 2.f * B * dx * dy, t3 = C * dy * dy;
    return (t1 + t2 + t3) - 1e-5f * (fabsf(t1) + fabsf(t2) + fabsf(t3));
}
__device__ __forceinline__ bool warp_block_may_hit(const float4 &a, const float4 &b, const int4 &rc, int wx0,
                                                   int wy0) {
    if (rc.x > wx0 + 7 || rc.z < wx0 || rc.y > wy0 + 3 || rc.w < wy0) return false;
    const float x0 = (float)wx0 + 0.5f - a.x, x1 = x0 + 7.f;  // block corners relative to the centre
    const float y0 = (float)wy0 + 0.5f - a.y, y1 = y0 + 3.f;
    if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return true;
    const float A = a.z, B = a.w, C = b.x;
    // the reciprocals only place the minimiser on an edge: a relative error e
    // there changes q by O(e^2), far inside the slack below
    const float iA = __fdividef(1.f, A), iC = __fdividef(1.f, C);
    float qmin = 1e30f;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dx = e ? x1 : x0;  // vertical edge, dy free in [y0, y1]
        const float dy = fminf(fmaxf(-B * dx * iC, y0), y1);
        qmin = fminf(qmin, q_slack(A, B, C, dx, dy));
        const float ey = e ? y1 : y0;  // horizontal edge, dx free in [x0, x1]
        const float ex = fminf(fmaxf(-B * ey * iA, x0), x1);
        qmin = fminf(qmin, q_slack(A, B, C, ex, ey));
    }
    return !(qmin > kQMax + 1e-3f);  // NaN-safe: keep on doubt
}

// Backward of one blended entry under the colour + depth loss (adjoint of
// Eq. 3-6, walking the list back to front). On entry T is the transmittance
// behind the entry and GS the sum of w_i (g . f_i) over the entries behind it;
// on return T is the transmittance in front of it and GS includes it. th gets
// the loss gradient of the entry's (mean2d.x, mean2d.y, A, B, C, z), w its
// blend weight and dal dL/dalpha. Every operation is explicitly rounded, so
// that the tracking pass and the separate backward produce the same bits.
__device__ __forceinline__ void entry_grad_cd(float alpha, float sg, float dx, float dy, const float4 &a,
                                              const float4 &b, const float4 &c, float gc0, float gc1, float gc2,
                                              float gD, float &T, float &GS, float (&th)[6], float &w, float &dal) {
    const float one_m = __fsub_rn(1.f, alpha);
    const float inv = __fdividef(1.f, one_m);
    T = __fmul_rn(T, inv);
    w = __fmul_rn(alpha, T);
    const float dot = __fmaf_rn(gD, b.z, __fmaf_rn(gc2, c.z, __fmaf_rn(gc1, c.y, __fmul_rn(gc0, c.x))));
    dal = __fmaf_rn(T, dot, -__fmul_rn(inv, GS));
    GS = __fmaf_rn(w, dot, GS);
    const float dpow = sg >= kAlphaMax ? 0.f : __fmul_rn(dal, alpha);
    const float hp = __fmul_rn(-0.5f, dpow);
    th[0] = __fmul_rn(dpow, __fmaf_rn(a.z, dx, __fmul_rn(a.w, dy)));
    th[1] = __fmul_rn(dpow, __fmaf_rn(a.w, dx, __fmul_rn(b.x, dy)));
    th[2] = __fmul_rn(hp, __fmul_rn(dx, dx));
    th[3] = __fmul_rn(-dpow, __fmul_rn(dx, dy));
    th[4] = __fmul_rn(hp, __fmul_rn(dy, dy));
    th[5] = __fmul_rn(w, gD);
}

// acc[c] += th[r] * J[6r + c] for the 6x6 pose Jacobian J of one record
// (row-major [theta = mean2d.x, mean2d.y, A, B, C, z][xi = rho, phi], nine
// float4 in shared memory), in element order. Each pair of neighbouring
// columns (2m, 2m + 1) lies in one row, so the pairs are contracted with the
// packed two-lane FP32 FMA of sm_100+ (fma.rn.f32x2): 18 instructions instead
// of 36, each lane rounded exactly as fmaf, so the sums are the same bits.
__device__ __forceinline__ void fma_x2(float &d0, float &d1, float a, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %2};\n\t"
        "mov.b64 rb, {%3, %4};\n\t"
        "mov.b64 rd, {%0, %1};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rd;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void pose_contract(float (&acc)[6], const float (&th)[6], const float4 *J) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float4 jq = J[q];
        const int e = 4 * q;  // elements e .. e + 3: two column pairs, each within row e / 6 resp. (e + 2) / 6
        fma_x2(acc[e % 6], acc[(e + 1) % 6], th[e / 6], jq.x, jq.y);
        fma_x2(acc[(e + 2) % 6], acc[(e + 3) % 6], th[(e + 2) / 6], jq.z, jq.w);
    }
}

}  // namespace gs
