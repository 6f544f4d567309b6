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

// Packed (re, im) sums: the IEEE operations of operator+ applied to the real
// and the imaginary part side by side, two FP32 values per instruction (the
// packed FP32x2 arithmetic of compute capability 10.x), so the results are
// bitwise those of the scalar code.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

__device__ __forceinline__ dd2 dd2_add(dd2 a, dd2 b) {
    const float2 ah = make_float2(a.x.hi, a.y.hi), bh = make_float2(b.x.hi, b.y.hi);
    const float2 al = make_float2(a.x.lo, a.y.lo), bl = make_float2(b.x.lo, b.y.lo);
    // two-sum of the high parts
    const float2 s = f2_add(ah, bh);
    const float2 bb = f2_sub(s, ah);
    const float2 e = f2_add(f2_sub(ah, f2_sub(s, bb)), f2_sub(bh, bb));
    // the low parts, then the fast two-sum
    const float2 t = f2_add(e, f2_add(al, bl));
    const float2 r = f2_add(s, t);
    const float2 l = f2_sub(t, f2_sub(r, s));
    return dd2{dd(r.x, l.x), dd(r.y, l.y)};
}
__device__ __forceinline__ dd2 dd2_sub(dd2 a, dd2 b) { return dd2_add(a, dd2{-b.x, -b.y}); }


__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }
__device__ __forceinline__ dd &operator*=(dd &a, dd b) { return a = a * b; }

}  // namespace pnp
