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

// inclusive pixel rect test: x0 <= px <= x1 and y0 <= py <= y1
__device__ __forceinline__ bool in_rect(int px, int py, int4 rc) {
    return (unsigned)(px - rc.x) <= (unsigned)(rc.z - rc.x) && (unsigned)(py - rc.y) <= (unsigned)(rc.w - rc.y);
}

// a = (mx, my, A, B), b = (C, opacity, z, nu). Returns false if the Gaussian does
// not contribute (q > 9 or alpha < 1/255); otherwise G = exp(-q/2),
// sg = opacity * G and alpha = min(0.99, sg).
__device__ __forceinline__ bool eval_alpha(float pxc, float pyc, const float4 &a, const float4 &b, float &dx,
                                           float &dy, float &G, float &sg, float &alpha) {
    dx = __fsub_rn(pxc, a.x);
    dy = __fsub_rn(pyc, a.y);
    const float cross = __fmul_rn(__fmul_rn(2.f, a.w), __fmul_rn(dx, dy));
    const float q = __fmaf_rn(__fmul_rn(a.z, dx), dx, __fmaf_rn(__fmul_rn(b.x, dy), dy, cross));
    if (!(q <= kQMax)) return false;
    G = __expf(__fmul_rn(-0.5f, q));
    sg = __fmul_rn(b.y, G);
    alpha = fminf(kAlphaMax, sg);
    return alpha >= kAlphaMin;
}

}  // namespace gs
