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


// a / b: the FP32 quotient of the high parts, corrected once by the
// remainder a - q b taken in double-float (about 2^-47 relative)
__device__ __forceinline__ dd dd_div(dd a, dd b) {
    const float q1 = a.hi / b.hi;
    const dd r = a - b * dd(q1, 0.f);
    const float q2 = r.hi / b.hi;
    return dd_fast_two_sum(q1, q2);
}

// ln(1 - u) for 1 - u > 2^-100, on the FP32 pipes.  With x = 1 - u = 2^e m,
// m in [1/sqrt2, sqrt2): ln x = e ln2 + 2 atanh(r), r = (m - 1) / (m + 1),
// |r| <= 0.1716, and atanh(r) = r (1 + r^2/3 + r^4/5 + ... + r^18/19): the
// first term left out is below 2^-54 of the sum.  For u <= 0.29 (e = 0)
// r = -u / (2 - u) is formed from u itself, so a small u keeps its relative
// precision (1 - u would round its low bits away).
__device__ __forceinline__ dd dd_log1m(dd u) {
    constexpr dd kLn2(0.6931471805599453094172321);
    const dd one(1.f, 0.f);
    dd num, den;
    int e = 0;
    if (u.hi <= 0.29f) {
        num = -u;
        den = dd(2.f, 0.f) - u;
    } else {
        const dd x = one - u;
        e = ((__float_as_int(x.hi) >> 23) & 0xff) - 126;       // x.hi / 2^e in [1/2, 1)
        const float sc = __int_as_float((127 - e) << 23);          // 2^-e, exact
        dd m(x.hi * sc, x.lo * sc);
        if (m.hi < 0.70710678f) {
            m = dd(2.f * m.hi, 2.f * m.lo);
            e -= 1;
        }
        num = m - one;
        den = m + one;
    }
    const dd r = dd_div(num, den);
    const dd z = r * r;
    dd p(1.0 / 19.0);
    p = p * z + dd(1.0 / 17.0);
    p = p * z + dd(1.0 / 15.0);
    p = p * z + dd(1.0 / 13.0);
    p = p * z + dd(1.0 / 11.0);
    p = p * z + dd(1.0 / 9.0);
    p = p * z + dd(1.0 / 7.0);
    p = p * z + dd(1.0 / 5.0);
    p = p * z + dd(1.0 / 3.0);
    p = p * z + one;
    const dd at = r * p;
    return dd(2.f * at.hi, 2.f * at.lo) + dd((float)e, 0.f) * kLn2;
}

__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }
__device__ __forceinline__ dd &operator*=(dd &a, dd b) { return a = a * b; }

}  // namespace pnp
