// Register-resident two-factor FFT of length L = N1 * N2 (N1, N2 in
// {2, 3, 4, 5, 6, 8, 16}, compile time).
//
// One line is handled by a group of G = max(N1, N2) threads; lane t of the
// group keeps its values in registers.  Forward transform of natural-order
// input x[n], n = n1 + N1 n2:
//   pass A (lane t = n1 < N1):  v[k2] = DFT_N2 over n2 of x[t + N1 n2],
//                               v[k2] *= W_L^(t k2), store to the exchange buffer
//   pass B (lane t = k2 < N2):  u[k1] = DFT_N1 over n1 of buf[n1][t]
//   => lane t holds X[t + N2 k1], k1 < N1.
// The inverse runs the same steps backwards with conjugate roots, taking
// X[t + N2 k1] in lane t and returning x[t + N1 n2] in lane t, so a forward
// transform, a pointwise product and an inverse need no extra reordering.
// W_L^m for m = t * j are precomputed per lane from the FP64-built table.
#pragma once

#include "fft_smem.cuh"

namespace pnp {

// root-of-unity constants (mathematical values, rounded to T)
constexpr double kC8 = 0.70710678118654752440;   // cos(pi/4)
constexpr double kC16 = 0.92387953251128675613;  // cos(pi/8)
constexpr double kS16 = 0.38268343236508977173;  // sin(pi/8)
constexpr double kS3 = 0.86602540378443864676;   // sin(2pi/3)
constexpr double kC5a = 0.30901699437494742410;  // cos(2pi/5)
constexpr double kC5b = -0.80901699437494742410; // cos(4pi/5)
constexpr double kS5a = 0.95105651629515357212;  // sin(2pi/5)
constexpr double kS5b = 0.58778525229247312917;  // sin(4pi/5)

template <typename C> __device__ __forceinline__ C mulc(C a, double re, double im) {
    using T = decltype(a.x);
    return C{a.x * (T)re - a.y * (T)im, a.x * (T)im + a.y * (T)re};
}

// in-register DFTs of size R, in place, natural order in and out; forward
// uses exp(-2 pi i / R), INV its conjugate
template <bool INV, typename C> __device__ __forceinline__ void rdft2(C *v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <bool INV, typename C> __device__ __forceinline__ void rdft3(C *v) {
    using T = decltype(v[0].x);
    C t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C m = C{v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y};
    C r = rot<INV>(cscale(d, (T)kS3));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}

// complex sums of the radix-4 butterflies: PK selects, for double-float,
// the packed FP32x2 form (two FP32 additions per instruction, the scalar
// bits).  Only the 256-point x and y transforms take it: taken by every
// double-float kernel it stretched that unit's compile from 2 to 10.5 min.
template <bool PK, typename C> __device__ __forceinline__ C bsum(C a, C b) {
    if constexpr (PK && std::is_same<C, dd2>::value) return dd2_add(a, b);
    else return cadd(a, b);
}
template <bool PK, typename C> __device__ __forceinline__ C bdif(C a, C b) {
    if constexpr (PK && std::is_same<C, dd2>::value) return dd2_sub(a, b);
    else return csub(a, b);
}

template <bool INV, typename C, bool PK = false> __device__ __forceinline__ void rdft4(C *v) {
    C t0 = bsum<PK>(v[0], v[2]), t1 = bdif<PK>(v[0], v[2]);
    C t2 = bsum<PK>(v[1], v[3]), t3 = rot<INV>(bdif<PK>(v[1], v[3]));
    v[0] = bsum<PK>(t0, t2);
    v[2] = bdif<PK>(t0, t2);
    v[1] = bsum<PK>(t1, t3);
    v[3] = bdif<PK>(t1, t3);
}

template <bool INV, typename C> __device__ __forceinline__ void rdft5(C *v) {
    using T = decltype(v[0].x);
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    C a1 = C{v[0].x + (T)kC5a * t1.x + (T)kC5b * t2.x, v[0].y + (T)kC5a * t1.y + (T)kC5b * t2.y};
    C a2 = C{v[0].x + (T)kC5b * t1.x + (T)kC5a * t2.x, v[0].y + (T)kC5b * t1.y + (T)kC5a * t2.y};
    C b1 = rot<INV>(C{(T)kS5a * d1.x + (T)kS5b * d2.x, (T)kS5a * d1.y + (T)kS5b * d2.y});
    C b2 = rot<INV>(C{(T)kS5b * d1.x - (T)kS5a * d2.x, (T)kS5b * d1.y - (T)kS5a * d2.y});
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

// 8 = 2 x 4: even/odd halves, combined with W8^k
template <bool INV, typename C> __device__ __forceinline__ void rdft8(C *v) {
    using T = decltype(v[0].x);
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    rdft4<INV>(e);
    rdft4<INV>(o);
    const double sg = INV ? 1.0 : -1.0;
    C w1 = mulc(o[1], kC8, sg * kC8);
    C w2 = rot<INV>(o[2]);
    C w3 = mulc(o[3], -kC8, sg * kC8);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);
    v[5] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);
    v[6] = csub(e[2], w2);
    v[3] = cadd(e[3], w3);
    v[7] = csub(e[3], w3);
    (void)sizeof(T);
}

// 6 = 2 x 3 (Good-Thomas would need no twiddles; the plain split keeps the
// same shape as radix 16): n = n1 + 2 n2, k = k2 + 3 k1
template <bool INV, typename C> __device__ __forceinline__ void rdft6(C *v) {
    C a0[3] = {v[0], v[2], v[4]};
    C a1[3] = {v[1], v[3], v[5]};
    rdft3<INV>(a0);
    rdft3<INV>(a1);
    const double sg = INV ? 1.0 : -1.0;
    // W6^k2 for the odd half: 1, (1/2, -+sqrt3/2), (-1/2, -+sqrt3/2)
    a1[1] = mulc(a1[1], 0.5, sg * kS3);
    a1[2] = mulc(a1[2], -0.5, sg * kS3);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
        v[k2] = cadd(a0[k2], a1[k2]);
        v[k2 + 3] = csub(a0[k2], a1[k2]);
    }
}

// radix-4 butterflies for zero padding: inputs 2 and 3 zero, or only
// outputs 0 and 1 wanted; the values rdft4 gives there (adding an exact zero
// changes nothing)
template <bool INV, typename C, bool PK = false> __device__ __forceinline__ void rdft4_in2(C *v) {
    const C a = v[0], b = v[1], rb = rot<INV>(b);
    v[0] = bsum<PK>(a, b);
    v[2] = bdif<PK>(a, b);
    v[1] = bsum<PK>(a, rb);
    v[3] = bdif<PK>(a, rb);
}
template <bool INV, typename C, bool PK = false> __device__ __forceinline__ void rdft4_out2(C *v) {
    const C t0 = bsum<PK>(v[0], v[2]), t1 = bdif<PK>(v[0], v[2]);
    const C t2 = bsum<PK>(v[1], v[3]), t3 = rot<INV>(bdif<PK>(v[1], v[3]));
    v[0] = bsum<PK>(t0, t2);
    v[1] = bsum<PK>(t1, t3);
}

// 16 = 4 x 4: n = n1 + 4 n2, k = k2 + 4 k1.  IN8: inputs 8..15 are zero
// (n2 >= 2); OUT8: only outputs 0..7 are wanted (k1 < 2; the others are left
// undefined).
template <bool INV, typename C, bool IN8 = false, bool OUT8 = false, bool PK = false>
__device__ __forceinline__ void rdft16(C *v) {
    C a[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) a[n1][n2] = v[n1 + 4 * n2];
        if constexpr (IN8)
            rdft4_in2<INV, C, PK>(a[n1]);
        else
            rdft4<INV, C, PK>(a[n1]);
    }
    const double sg = INV ? 1.0 : -1.0;
    // W16^(n1 k2): exponents 1, 2, 3 (n1 = 1), 2, 4, 6 (n1 = 2), 3, 6, 9 (n1 = 3)
    a[1][1] = mulc(a[1][1], kC16, sg * kS16);
    a[1][2] = mulc(a[1][2], kC8, sg * kC8);
    a[1][3] = mulc(a[1][3], kS16, sg * kC16);
    a[2][1] = mulc(a[2][1], kC8, sg * kC8);
    a[2][2] = rot<INV>(a[2][2]);
    a[2][3] = mulc(a[2][3], -kC8, sg * kC8);
    a[3][1] = mulc(a[3][1], kS16, sg * kC16);
    a[3][2] = mulc(a[3][2], -kC8, sg * kC8);
    a[3][3] = mulc(a[3][3], -kC16, -sg * kS16);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        C b[4] = {a[0][k2], a[1][k2], a[2][k2], a[3][k2]};
        if constexpr (OUT8) {
            rdft4_out2<INV, C, PK>(b);
            v[k2] = b[0];
            v[k2 + 4] = b[1];
        } else {
            rdft4<INV, C, PK>(b);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = b[k1];
        }
    }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void rdftR(C *v) {
    if constexpr (R == 2) rdft2<INV>(v);
    else if constexpr (R == 3) rdft3<INV>(v);
    else if constexpr (R == 4) rdft4<INV>(v);
    else if constexpr (R == 5) rdft5<INV>(v);
    else if constexpr (R == 6) rdft6<INV>(v);
    else if constexpr (R == 8) rdft8<INV>(v);
    else if constexpr (R == 16) rdft16<INV>(v);
}

template <int N1, int N2> struct Shape {
    static constexpr int L = N1 * N2;
    static constexpr int G = N1 > N2 ? N1 : N2;   // lanes per line
    static constexpr int EX = N1 * (N2 + 1);       // exchange buffer (padded) per line
};

// Per-lane twiddles W_L^(t j) for j < G (mod L), from the table tw[m] = exp(-2 pi i m / L).
template <int N1, int N2, typename C> struct LaneTw {
    C w[Shape<N1, N2>::G];
    __device__ __forceinline__ void load(const C *__restrict__ tw, int t) {
        constexpr int L = N1 * N2;
#pragma unroll
        for (int j = 0; j < Shape<N1, N2>::G; ++j) w[j] = ldgc(&tw[(t * j) % L]);
    }
    __device__ __forceinline__ C operator[](int j) const { return w[j]; }
};

// The same values in a shared-memory table [j][lane] (one per CTA), for
// kernels whose register budget is better spent elsewhere.
template <int N1, int N2, typename C> struct SmemTw {
    const C *tab;
    int t;
    static constexpr int G = Shape<N1, N2>::G;
    static constexpr int WORDS = G * G;
    // every thread of the block calls fill; a __syncthreads must follow
    static __device__ __forceinline__ void fill(C *tab, const C *__restrict__ tw) {
        constexpr int L = N1 * N2;
        for (int k = threadIdx.x; k < G * G; k += blockDim.x) {
            const int j = k / G, lane = k % G;
            tab[k] = ldgc(&tw[(lane * j) % L]);
        }
    }
    __device__ __forceinline__ C operator[](int j) const { return tab[j * G + t]; }
};

// forward: lane t < N1 gives x[t + N1 n2] in v[n2] (n2 < N2); on return lane
// t < N2 holds X[t + N2 k1] in v[k1] (k1 < N1).  ex = this line's exchange
// buffer, element a at ex[a * xs] (xs = number of interleaved lines).  half:
// x[j] = 0 for j >= L / 2 (a zero-extended line of at most L / 2 points),
// which prunes the first radix-16 stage (FP32 and FP64; double-float keeps
// the full stage: the second copy of it costs spills at its 128-register
// budget, 0.46 -> 0.49 ms for ten fields).  Contains two __syncthreads (every
// thread of the block must call).
template <int N1, int N2, bool PK = false, typename C, typename TW>
__device__ __forceinline__ void fwd2(C (&v)[Shape<N1, N2>::G], const TW &tw, C *ex, int t, int xs,
                                     bool half = false) {
    constexpr int S = N2 + 1;
    if (t < N1) {
        if constexpr (N2 == 16 && !std::is_same<C, dd2>::value) {
            if (half)
                rdft16<false, C, true, false>(v);
            else
                rdft16<false>(v);
        } else if constexpr (N2 == 16) {
            rdft16<false, C, false, false, PK>(v);
        } else {
            rdftR<N2, false>(v);
        }
#pragma unroll
        for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], tw[k2]);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) ex[(t * S + k2) * xs] = v[k2];
    }
    __syncthreads();
    if (t < N2) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = ex[(n1 * S + t) * xs];
        if constexpr (N1 == 16)
            rdft16<false, C, false, false, PK>(v);
        else
            rdftR<N1, false>(v);
    }
    __syncthreads();
}

// inverse (unnormalised): lane t < N2 gives X[t + N2 k1] in v[k1]; on return
// lane t < N1 holds x[t + N1 n2] in v[n2].  half: only x[j], j < L / 2, is
// wanted (v[n2] for n2 >= N2 / 2 may be left undefined; FP32 and FP64 prune
// the last radix-16 stage).
template <int N1, int N2, bool PK = false, typename C, typename TW>
__device__ __forceinline__ void inv2(C (&v)[Shape<N1, N2>::G], const TW &tw, C *ex, int t, int xs,
                                     bool half = false) {
    constexpr int S = N2 + 1;
    if (t < N2) {
        if constexpr (N1 == 16)
            rdft16<true, C, false, false, PK>(v);
        else
            rdftR<N1, true>(v);
#pragma unroll
        for (int n1 = 1; n1 < N1; ++n1) v[n1] = cmul(v[n1], cconj(tw[n1]));
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) ex[(n1 * S + t) * xs] = v[n1];
    }
    __syncthreads();
    if (t < N1) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = ex[(t * S + k2) * xs];
        if constexpr (N2 == 16 && !std::is_same<C, dd2>::value) {
            if (half)
                rdft16<true, C, false, true>(v);
            else
                rdft16<true>(v);
        } else if constexpr (N2 == 16) {
            rdft16<true, C, false, false, PK>(v);
        } else {
            rdftR<N2, true>(v);
        }
    }
    __syncthreads();
}

}  // namespace pnp
