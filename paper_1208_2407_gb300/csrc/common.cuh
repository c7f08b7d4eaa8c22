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

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace ts
