// Double-float ("float-float") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the classical
// error-free transformations:
//   - two_sum (Knuth): s + e == a + b exactly, s = fl(a + b);
//   - fast_two_sum (Dekker): the same when |a| >= |b|;
//   - two_prod via FMA: p + e == a * b exactly, p = fl(a * b).
// On GB300 the FP64 unit runs at ~1/67 of the FP32 rate, so the reductions
// and the table preparation of FP32 grids use these instead of doubles.
#pragma once

#include <cuda_runtime.h>

namespace ts {

struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_make(float hi, float lo = 0.f) { return FF{hi, lo}; }

__device__ __forceinline__ FF two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return FF{s, e};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b)
{
    const float s = a + b;
    const float e = b - (s - a);
    return FF{s, e};
}

__device__ __forceinline__ FF two_prod(float a, float b)
{
    const float p = a * b;
    return FF{p, fmaf(a, b, -p)};
}

// a + b, both double-float
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    FF s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}

// a + b, b a float
__device__ __forceinline__ FF ff_add_f(FF a, float b)
{
    FF s = two_sum(a.hi, b);
    s.lo += a.lo;
    return fast_two_sum(s.hi, s.lo);
}

// a * b, b a float
__device__ __forceinline__ FF ff_mul_f(FF a, float b)
{
    FF p = two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// a * b, both double-float
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    FF p = two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

}  // namespace ts
