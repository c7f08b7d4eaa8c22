// Device helpers shared by the kernels of libtrotter.so (sm_103a).
//
// Rotation convention (Sec. 2, the block exponential M with hopping -J):
//   a' = cos(t) a + i sin(t) b,  b' = i sin(t) a + cos(t) b.
// Every kernel applies it in the versine form
//   a' = a - g a + i s b,  g = 1 - cos(t) = 2 sin^2(t/2),  s = sin(t),
// with (g, s) computed in FP64 and rounded once, so that the per-sweep
// unitarity defect of the rounded coefficients is O(ulp * t) rather than
// O(ulp): the error of (1 - g)^2 + s^2 - 1 stays ~1e-10 in FP32.
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
// g = 1 - cos phi = 2 sin^2 h, s = sin phi = 2 sin h cos h with h = phi/2.
// For |h| <= 0.4, sin h and cos h come from their Taylor series through h^7
// and h^8 (truncation below 2e-9 relative, under half an FP32 ulp); larger
// angles call sincosf.  g and s share sin h and cos h, so
// (1 - g)^2 + s^2 - 1 = -4 sin^2 h (1 - sin^2 h - cos^2 h) stays at
// O(ulp * phi^2): the unitarity defect shrinks with the angle.
__device__ __forceinline__ void angle_versine(float phi, float &g, float &s)
{
    const float h = 0.5f * phi;
    float sh, ch;
    if (fabsf(h) <= 0.4f) {
        const float h2 = h * h;
        sh = h * fmaf(h2, fmaf(h2, fmaf(h2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
        ch = fmaf(h2, fmaf(h2, fmaf(h2, fmaf(h2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f),
                           -0.5f), 1.0f);
    } else {
        sincosf(h, &sh, &ch);
    }
    g = 2.0f * sh * sh;
    s = 2.0f * sh * ch;
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
