// Batched mixed-radix Stockham FFT in shared memory.
//
// A CTA transforms NL lines of length L held element-major in shared memory
// (element j of line l at a[j * NL + l], so consecutive threads touch
// consecutive lines and bank conflicts stay low).  Each stage of radix R reads
// R strided values, applies the twiddles exp(-+2 pi i k r / (Ns R)) from a
// global table of exp(-2 pi i m / L) (built on the host in FP64), does the
// radix-R DFT in registers and writes the autosorted output to the other
// buffer; after the last stage the result is in natural order.
#pragma once

#include <cuda_runtime.h>

#include "ddouble.cuh"
#include "pnp_internal.h"

namespace pnp {

template <typename T> struct vec2;
template <> struct vec2<double> { using type = double2; };
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<dd> { using type = dd2; };

// read-only cached loads of scalars and complex values of every precision
template <typename T> __device__ __forceinline__ T ldgt(const T *p) { return __ldg(p); }
template <> __device__ __forceinline__ dd ldgt<dd>(const dd *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return dd(v.x, v.y);
}
template <typename C> __device__ __forceinline__ C ldgc(const C *p) { return __ldg(p); }
template <> __device__ __forceinline__ dd2 ldgc<dd2>(const dd2 *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return dd2{dd(v.x, v.y), dd(v.z, v.w)};
}

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return C{a.x * s, a.y * s}; }
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot(C a) {
    return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void small_dft(C (&v)[R], const C *__restrict__ tw, int L) {
    if constexpr (R == 2) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = rot<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if constexpr (R == 3) {
        // W = exp(-+2 pi i / 3): X1,2 = a - (b+c)/2 -+ i (sqrt3/2)(b - c)
        C w = tw[L / 3];                      // (-1/2, -sqrt3/2)
        auto s3 = -w.y;                       // sqrt(3)/2
        C t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        C m = C{v[0].x + w.x * t.x, v[0].y + w.x * t.y};
        C r = rot<INV>(cscale(d, s3));        // -+ i s3 d
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    } else if constexpr (R == 5) {
        C w1 = tw[L / 5], w2 = tw[(2 * L) / 5];
        auto c1 = w1.x, s1 = -w1.y, c2 = w2.x, s2 = -w2.y;
        C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        C d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
        C a1 = C{v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y};
        C a2 = C{v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y};
        C b1 = rot<INV>(C{s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y});
        C b2 = rot<INV>(C{s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y});
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void fft_stage(const C *__restrict__ a, C *__restrict__ b, int NL, int L, int Ns,
                                          const C *__restrict__ tw) {
    const int LR = L / R, step = L / (Ns * R);
    const int total = NL * LR;
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        const int l = it % NL, j = it / NL, k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C x = a[(j + r * LR) * NL + l];
            if (r > 0 && k > 0) {
                C w = ldgc(&tw[k * r * step]);
                if (INV) w.y = -w.y;
                x = cmul(x, w);
            }
            v[r] = x;
        }
        small_dft<R, INV>(v, tw, L);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) b[(base + r * Ns) * NL + l] = v[r];
    }
}

// Transform NL lines in `a` using `b` as the ping-pong buffer.  Caller has
// synchronised after filling `a`.  Returns the buffer holding the result;
// ends with a __syncthreads().
template <bool INV, typename C>
__device__ C *fft_lines(C *a, C *b, int NL, const FftAxis &ax, const C *__restrict__ tw) {
    int Ns = 1;
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.radix[s];
        switch (R) {
            case 4: fft_stage<4, INV>(a, b, NL, ax.L, Ns, tw); break;
            case 2: fft_stage<2, INV>(a, b, NL, ax.L, Ns, tw); break;
            case 3: fft_stage<3, INV>(a, b, NL, ax.L, Ns, tw); break;
            default: fft_stage<5, INV>(a, b, NL, ax.L, Ns, tw); break;
        }
        __syncthreads();
        C *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// Same, but the result always ends in `a` (copies back when needed).
template <bool INV, typename C>
__device__ void fft_lines_inplace(C *a, C *b, int NL, const FftAxis &ax, const C *__restrict__ tw) {
    C *res = fft_lines<INV>(a, b, NL, ax, tw);
    if (res != a) {
        const int total = NL * ax.L;
        for (int i = threadIdx.x; i < total; i += blockDim.x) a[i] = res[i];
        __syncthreads();
    }
}

}  // namespace pnp
