// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 executes FP32 at ~58x its FP64 rate, so the FFT arithmetic of the
// FP64-accuracy mu_ex path runs in this format on the FP32 pipes.  Error-free
// transformations (Knuth's two-sum, Dekker's fast two-sum, the FMA-based exact
// product) give the classic double-float add and multiply; the add is the
// normwise ("sloppy") variant, whose error is bounded relative to |a| + |b| --
// the bound that FFT error analysis uses.  Nothing here relies on
// reassociation; the code is compiled without fast-math.
#pragma once

#include <cuda_runtime.h>

namespace pnp {

struct __align__(8) dd {
    float hi, lo;
    __host__ __device__ constexpr dd() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    // split of a double into the nearest float and the float nearest the rest
    __host__ __device__ constexpr dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ constexpr dd(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) dd2 {
    dd x, y;
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return dd(s, e);
}

__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return dd(s, e);
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    const float t = s.lo + (a.lo + b.lo);
    return dd_fast_two_sum(s.hi, t);
}

__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dd_fast_two_sum(p, e);
}

__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }
__device__ __forceinline__ dd &operator*=(dd &a, dd b) { return a = a * b; }

}  // namespace pnp
