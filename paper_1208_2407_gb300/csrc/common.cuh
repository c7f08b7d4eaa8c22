// Device helpers shared by the kernels of libtrotter.so (sm_103a).
//
// Rotation convention (Sec. 2, the block exponential M with hopping -J):
//   a' = cos(t) a + i sin(t) b,  b' = i sin(t) a + cos(t) b.
// The kernels apply it in one of two forms, never with cos(t) itself:
//  - the versine form a' = a - g a + i s b, g = 1 - cos(t) = 2 sin^2(t/2),
//    s = sin(t), with (g, s) computed in FP64 and rounded once, so that the
//    per-sweep unitarity defect of the rounded coefficients is O(ulp * t)
//    rather than O(ulp): (1 - g)^2 + s^2 - 1 stays ~1e-10 in FP32;
//  - the lifting form (three shears with tan(t/2) and sin(t), each of
//    determinant 1) where both members of a pair are at hand and |t| <= pi/2.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ts {

// a <- a - g a + i s b   (one member of a pair; b is the partner's old value)
template <typename T>
__device__ __forceinline__ void rot1(T &ar, T &ai, T br, T bi, T g, T s)
{
    T nr = fma(-s, bi, fma(-g, ar, ar));
    T ni = fma(s, br, fma(-g, ai, ai));
    ar = nr;
    ai = ni;
}

// both members of a pair
template <typename T>
__device__ __forceinline__ void rot2(T &ar, T &ai, T &br, T &bi, T g, T s)
{
    T ar0 = ar, ai0 = ai;
    rot1(ar, ai, br, bi, g, s);
    rot1(br, bi, ar0, ai0, g, s);
}

// Both members of a pair in lifting form: the rotation a' = c a + i s b,
// b' = i s a + c b is two real plane rotations, of (a_re, b_im) and of
// (b_re, a_im), each applied as three shears x -= t y; y += s x; x -= t y
// with t = tan(theta/2), s = sin(theta) (6 FMA per pair, determinant 1).
__device__ __forceinline__ void rot_lift(float &ar, float &ai, float &br, float &bi, float t,
                                         float s)
{
    ar = fmaf(-t, bi, ar);
    br = fmaf(-t, ai, br);
    bi = fmaf(s, ar, bi);
    ai = fmaf(s, br, ai);
    ar = fmaf(-t, bi, ar);
    br = fmaf(-t, ai, br);
}

// The same in FP64.
__device__ __forceinline__ void rot_lift(double &ar, double &ai, double &br, double &bi, double t,
                                         double s)
{
    ar = fma(-t, bi, ar);
    br = fma(-t, ai, br);
    bi = fma(s, ar, bi);
    ai = fma(s, br, ai);
    ar = fma(-t, bi, ar);
    br = fma(-t, ai, br);
}

// A pair rotation in lifting form (c = tan(theta/2)) or versine form
// (c = 1 - cos(theta)); s = sin(theta) in both.
template <bool LIFT, typename T>
__device__ __forceinline__ void rot_pair(T &ar, T &ai, T &br, T &bi, T c, T s)
{
    if constexpr (LIFT)
        rot_lift(ar, ai, br, bi, c, s);
    else
        rot2(ar, ai, br, bi, c, s);
}

// psi <- psi * exp(-i phi) with g = 1 - cos(phi), s = sin(phi):
//   (r + i m)((1 - g) - i s) = (r - g r + s m) + i (m - g m - s r)
template <typename T>
__device__ __forceinline__ void phase1(T &r, T &m, T g, T s)
{
    T nr = fma(s, m, fma(-g, r, r));
    T nm = fma(-s, r, fma(-g, m, m));
    r = nr;
    m = nm;
}

// Versine coefficients of an angle phi computed on the device in FP32:
// g = 1 - cos phi = 2 sin^2 h and s = sin phi = 2 sin h cos h, h = phi / 2.
// Both are unchanged when h moves by a multiple of pi (sin h and cos h change
// sign together), so h is reduced to r = h - k pi, |r| <= pi/2, by a
// Cody-Waite split of pi into three floats (the first two have 12 significant
// bits, so k times them is exact for |k| < 2^12; beyond that the reduction
// error stays below the rounding error of phi itself).  sin r and cos r come
// from their Taylor series through r^13 and r^14 (truncation below 7e-10);
// for |h| <= 0.4 no reduction is needed and the series stop at r^7 and r^8
// (truncation below 2e-9 relative).  g and s share sin r and cos r, so the
// unitarity defect (1 - g)^2 + s^2 - 1 = -4 sin^2 r (1 - sin^2 r - cos^2 r)
// is O(ulp * phi^2) for small angles.
__device__ __forceinline__ void versine_short(float h, float &g, float &s)
{
    const float t = h * h;
    const float sh = h * fmaf(t, fmaf(t, fmaf(t, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
    const float ch = fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f),
                             -0.5f), 1.0f);
    g = 2.0f * sh * sh;
    s = 2.0f * sh * ch;
}

// Kept out of line: large angles are rare, and inlining this path at every
// use made the fused kernel's code outgrow the instruction cache.  Returns
// (g, s) in registers.
static __device__ __noinline__ float2 versine_reduced2(float h)
{
    const float k = rintf(h * 0.318309886f);             // 1/pi
    float r = fmaf(-k, 3.140625f, h);                      // pi = A + B + C
    r = fmaf(-k, 0x1.fb4p-11f, r);
    r = fmaf(-k, 0x1.4442d2p-23f, r);
    const float t = r * r;
    float ps = fmaf(t, -1.0f / 6227020800.0f, 1.0f / 39916800.0f);
    ps = fmaf(t, ps, -1.0f / 362880.0f);
    ps = fmaf(t, ps, 1.0f / 5040.0f);
    ps = fmaf(t, ps, -1.0f / 120.0f);
    ps = fmaf(t, ps, 1.0f / 6.0f);
    const float sh = fmaf(-r * t, ps, r);                 // r - r^3/6 + ...
    float pc = fmaf(t, -1.0f / 87178291200.0f, 1.0f / 479001600.0f);
    pc = fmaf(t, pc, -1.0f / 3628800.0f);
    pc = fmaf(t, pc, 1.0f / 40320.0f);
    pc = fmaf(t, pc, -1.0f / 720.0f);
    pc = fmaf(t, pc, 1.0f / 24.0f);
    pc = fmaf(t, pc, -0.5f);
    const float ch = fmaf(t, pc, 1.0f);
    return make_float2(2.0f * sh * sh, 2.0f * sh * ch);
}

__device__ __forceinline__ void versine_reduced(float h, float &g, float &s)
{
    const float2 r = versine_reduced2(h);
    g = r.x;
    s = r.y;
}

__device__ __forceinline__ void angle_versine(float phi, float &g, float &s)
{
    const float h = 0.5f * phi;
    if (fabsf(h) <= 0.4f)
        versine_short(h, g, s);
    else
        versine_reduced(h, g, s);
}

// The same in FP64 (plain path of FP64 grids).
__device__ __forceinline__ void angle_versine(double phi, double &g, double &s)
{
    const double sh = sin(0.5 * phi);
    g = 2.0 * sh * sh;
    s = sin(phi);
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace ts
