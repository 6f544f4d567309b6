// z kernels for padded length Lz = 256 with up to three species and
// double-float values: 64 lanes per column, four radix-4 stages, per-lane
// accumulators in registers.
//
// The two-factor z kernels (mu_ex_reg.cuh) give a column 16 lanes of 16
// values and keep the s spectral accumulators of every column in shared
// memory, which caps residency at 8 (FP32) or 6 (double-float) warps per SM
// and costs a shared-memory read-modify-write per product.  Here a column has
// 64 lanes of 4 values: lane t holds x[t + 64 n1]; after the forward
// transform lane t = 16 k1 + 4 k2 + k3 holds X[k1 + 4 k2 + 16 k3 + 64 k4] in
// v[k4], and the inverse takes that layout back to natural order, so the
// spectral products need no reordering and each lane's s x 4 accumulators
// stay in registers.  Decimation in frequency: with n = n0 + 64 n1 and
// k = k1 + 4 k',
//   X[k1 + 4 k'] = sum_n0 W64^(n0 k') [ W256^(n0 k1) sum_n1 x[n0 + 64 n1] W4^(n1 k1) ],
// and the same split again on the inner 64- and 16-point transforms.  The
// three exchanges go through two padded shared-memory buffers per column.
// A CTA takes TX half-spectrum columns at the two rows (kyp, Ly - kyp), which
// read the same kernel-spectrum octant entries; thread = t * 2 TX + b * TX + c
// keeps consecutive kx in consecutive threads for coalesced column loads.
// Included by mu_ex_core.cuh only.
#pragma once

#include <type_traits>

#include "fft_reg.cuh"

namespace pnp {

constexpr int kZ4Len = 256;
constexpr int kZ4Lanes = 64;
constexpr int kZ4Buf = 320;        // 256 values + one pad slot per four
constexpr int kZ4MaxSpecies = 3;

// padded exchange index: stride-4 accesses land on the minimum number of
// shared-memory wavefronts
__device__ __forceinline__ int z4pad(int i) { return i + (i >> 2); }

// The radix-4 butterflies here keep scalar double-float sums: the packed
// FP32x2 form of the x and y lines (fft_reg.cuh) measured slower in these
// kernels (z MAC 1.57 -> 1.62 ms, z back 1.77 -> 1.79 ms at 128^3 -> 256^3),
// presumably because their 128-register budget leaves little room to keep
// real and imaginary parts paired.

// Columns of at most 128 rows (the zero-extended half of Lz = 256): a lane's
// input values n1 = 2, 3 are zero padding and only its output rows t and
// t + 64 are stored, so the first forward and the last inverse radix-4
// butterflies shrink.  Both give the values rdft4 gives (adding an exact zero
// changes nothing).
template <bool INV, typename C> __device__ __forceinline__ void z4_rdft4_in2(C (&v)[4]) {
    const C a = v[0], b = v[1], rb = rot<INV>(b);
    v[0] = cadd(a, b);
    v[2] = csub(a, b);
    v[1] = cadd(a, rb);
    v[3] = csub(a, rb);
}
template <bool INV, typename C> __device__ __forceinline__ void z4_rdft4_out2(C (&v)[4]) {
    const C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const C t2 = cadd(v[1], v[3]), t3 = rot<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[1] = cadd(t1, t3);
}

// lane t's frequency of value k4
__device__ __forceinline__ int z4_freq(int t, int k4) { return (t >> 4) + 4 * ((t >> 2) & 3) + 16 * (t & 3) + 64 * k4; }

// twiddles of lane t: [0..2] W256^(n0 k), [3..5] W64^(m0 k), [6..8] W16^(p0 k),
// k = 1..3, n0 = t, m0 = t mod 16, p0 = t mod 4.  Held in registers (FP32) or
// read from a per-CTA copy of the W256 table in shared memory (64-bit types).
template <typename C> struct Z4TwReg {
    C w[9];
    __device__ __forceinline__ void init(const C *__restrict__ tab, int t) {
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            w[k - 1] = ldgc(&tab[(t * k) & 255]);
            w[2 + k] = ldgc(&tab[(4 * (t & 15) * k) & 255]);
            w[5 + k] = ldgc(&tab[(16 * (t & 3) * k) & 255]);
        }
    }
    __device__ __forceinline__ C operator[](int j) const { return w[j]; }
};
template <typename C> struct Z4TwSmem {
    const C *tab;
    int e[3];
    __device__ __forceinline__ void init(const C *stab, int t) {
        tab = stab;
        e[0] = t;
        e[1] = 4 * (t & 15);
        e[2] = 16 * (t & 3);
    }
    __device__ __forceinline__ C operator[](int j) const { return tab[(e[j / 3] * (j % 3 + 1)) & 255]; }
};

// forward 256-point DFT (see the header comment for the layouts).  A, B: the
// column's exchange buffers, element i at [z4pad(i) * xs]; half: inputs
// x[t + 128], x[t + 192] are zero.  Starts with a barrier before its first
// write (the buffers may still be read by the previous transform); every
// thread of the block must call it.
template <typename C, typename TW>
__device__ __forceinline__ void z4_fwd(C (&v)[4], const TW &tw, C *A, C *B, int t, int xs, bool half) {
    if (half)
        z4_rdft4_in2<false>(v);
    else
        rdft4<false>(v);
#pragma unroll
    for (int k = 1; k < 4; ++k) v[k] = cmul(v[k], tw[k - 1]);
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) A[z4pad(k1 * 64 + t) * xs] = v[k1];
    __syncthreads();
    {
        const int k1 = t >> 4, m0 = t & 15;
#pragma unroll
        for (int m1 = 0; m1 < 4; ++m1) v[m1] = A[z4pad(k1 * 64 + m0 + 16 * m1) * xs];
        rdft4<false>(v);
#pragma unroll
        for (int k = 1; k < 4; ++k) v[k] = cmul(v[k], tw[2 + k]);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) B[z4pad(k1 * 64 + k2 * 16 + m0) * xs] = v[k2];
    }
    __syncthreads();
    {
        const int k1 = t >> 4, k2 = (t >> 2) & 3, p0 = t & 3;
#pragma unroll
        for (int p1 = 0; p1 < 4; ++p1) v[p1] = B[z4pad(k1 * 64 + k2 * 16 + p0 + 4 * p1) * xs];
        rdft4<false>(v);
#pragma unroll
        for (int k = 1; k < 4; ++k) v[k] = cmul(v[k], tw[5 + k]);
#pragma unroll
        for (int k3 = 0; k3 < 4; ++k3) A[z4pad(k1 * 64 + k2 * 16 + k3 * 4 + p0) * xs] = v[k3];
    }
    __syncthreads();
    {
        const int k1 = t >> 4, k2 = (t >> 2) & 3, k3 = t & 3;
#pragma unroll
        for (int p0 = 0; p0 < 4; ++p0) v[p0] = A[z4pad(k1 * 64 + k2 * 16 + k3 * 4 + p0) * xs];
        rdft4<false>(v);
    }
}

// inverse (unnormalised) of z4_fwd: the same stages backwards with conjugate
// twiddles; half: only rows t and t + 64 (v[0], v[1]) are produced
template <typename C, typename TW>
__device__ __forceinline__ void z4_inv(C (&v)[4], const TW &tw, C *A, C *B, int t, int xs, bool half) {
    {
        const int k1 = t >> 4, k2 = (t >> 2) & 3, k3 = t & 3;
        rdft4<true>(v);
        __syncthreads();
#pragma unroll
        for (int p0 = 0; p0 < 4; ++p0) A[z4pad(k1 * 64 + k2 * 16 + k3 * 4 + p0) * xs] = v[p0];
    }
    __syncthreads();
    {
        const int k1 = t >> 4, k2 = (t >> 2) & 3, p0 = t & 3;
#pragma unroll
        for (int k3 = 0; k3 < 4; ++k3) v[k3] = A[z4pad(k1 * 64 + k2 * 16 + k3 * 4 + p0) * xs];
#pragma unroll
        for (int k = 1; k < 4; ++k) v[k] = cmul(v[k], cconj(tw[5 + k]));
        rdft4<true>(v);
#pragma unroll
        for (int p1 = 0; p1 < 4; ++p1) B[z4pad(k1 * 64 + k2 * 16 + p0 + 4 * p1) * xs] = v[p1];
    }
    __syncthreads();
    {
        const int k1 = t >> 4, m0 = t & 15;
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k2] = B[z4pad(k1 * 64 + k2 * 16 + m0) * xs];
#pragma unroll
        for (int k = 1; k < 4; ++k) v[k] = cmul(v[k], cconj(tw[2 + k]));
        rdft4<true>(v);
#pragma unroll
        for (int m1 = 0; m1 < 4; ++m1) A[z4pad(k1 * 64 + m0 + 16 * m1) * xs] = v[m1];
    }
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k1] = A[z4pad(k1 * 64 + t) * xs];
#pragma unroll
    for (int k = 1; k < 4; ++k) v[k] = cmul(v[k], cconj(tw[k - 1]));
    if (half)
        z4_rdft4_out2<true>(v);
    else
        rdft4<true>(v);
}

// columns per CTA side: FP32 4 (512 threads), 64-bit types 2 (256 threads)
template <typename T> constexpr int z4_tx() { return std::is_same<T, float>::value ? 4 : 2; }

// dynamic shared memory of a z4 CTA: two exchange buffers per column and the
// twiddle table; the z back adds two prefetch stages of four values per lane
// and two kernel-spectrum stages of S x 4 values per lane and column pair
template <typename T> constexpr size_t z4_smem() {
    return (2 * (size_t)kZ4Buf * 2 * z4_tx<T>() + kZ4Len) * sizeof(typename vec2<T>::type);
}
template <typename T> constexpr size_t z4_stage_elems() { return (size_t)2 * 4 * kZ4Lanes * 2 * z4_tx<T>(); }
template <typename T> constexpr size_t z4_spec_elems() { return (size_t)2 * kZ4MaxSpecies * 4 * kZ4Lanes * z4_tx<T>(); }
template <typename T> constexpr size_t z4_smem_mac() { return z4_smem<T>() + z4_spec_elems<T>() * sizeof(T); }
template <typename T> constexpr size_t z4_smem_back() {
    return z4_smem<T>() + z4_stage_elems<T>() * sizeof(typename vec2<T>::type) + z4_spec_elems<T>() * sizeof(T);
}

// 16-byte asynchronous copy global -> shared (zero-fill when !valid; src must
// still be a valid address)
__device__ __forceinline__ void z4_cp16(void *smem, const void *gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 16 : 0));
}

// asynchronous copy of one 4- or 8-byte value global -> shared (zero-fill
// when !valid; src must still be a valid address)
template <typename T> __device__ __forceinline__ void z4_cp_scalar(T *smem, const T *gmem, bool valid) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte values");
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"((int)sizeof(T)),
                 "r"(valid ? (int)sizeof(T) : 0));
}

// per-lane set-up shared by both kernels
template <typename T> struct Z4Lane {
    using C = typename vec2<T>::type;
    using TW = typename std::conditional<std::is_same<T, float>::value, Z4TwReg<C>, Z4TwSmem<C>>::type;
    int c, b, t, lanes, kx, ky, fy;
    bool ok;
    C *bufA, *bufB;
    TW tw;
    int fz[4];
    bool hi[4];
    bool half;         // nz <= 128: rows >= 128 are zero padding
    __device__ __forceinline__ void init(const Dims &d, const C *__restrict__ twz, unsigned char *smem) {
        constexpr int TX = z4_tx<T>();
        half = d.nz <= kZ4Len / 2;
        lanes = 2 * TX;
        c = threadIdx.x % TX;
        b = (threadIdx.x / TX) & 1;
        t = threadIdx.x / lanes;
        const int kyp = blockIdx.y;
        kx = blockIdx.x * TX + c;
        ok = zcol(d, kyp, b, kx, ky);
        fy = kyp;        // both rows of the pair fold to kyp
        C *base = reinterpret_cast<C *>(smem);
        bufA = base + (b * TX + c);
        bufB = bufA + (size_t)kZ4Buf * lanes;
        C *tab = base + (size_t)2 * kZ4Buf * lanes;
        if constexpr (std::is_same<T, float>::value) {
            tw.init(twz, t);
        } else {
            for (int k = threadIdx.x; k < kZ4Len; k += blockDim.x) tab[k] = ldgc(&twz[k]);
            __syncthreads();
            tw.init(tab, t);
        }
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
            const int kz = z4_freq(t, k4);
            fz[k4] = kz <= kZ4Len / 2 ? kz : kZ4Len - kz;
            hi[k4] = kz > kZ4Len / 2;
        }
    }
    // x[t + 64 n1] of a column whose rows z < nz start at src (stride plane)
    __device__ __forceinline__ void load(C (&v)[4], const C *src, const Dims &d, size_t plane) const {
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) {
            const int zz = t + 64 * n1;
            v[n1] = (ok && zz < d.nz) ? src[(size_t)zz * plane] : C{0, 0};
        }
    }
    // asynchronous copy of this lane's four values of a column into its own
    // slots of a prefetch stage (read back by the same lane: no barrier)
    __device__ __forceinline__ void prefetch(C *stage, const C *src, const Dims &d, size_t plane) const {
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) {
            const int zz = t + 64 * n1;
            const bool in = ok && zz < d.nz;
            z4_cp16(stage + ((size_t)n1 * kZ4Lanes + t) * lanes + (b * z4_tx<T>() + c), in ? src + (size_t)zz * plane : src,
                    in);
        }
        asm volatile("cp.async.commit_group;\n" ::);
    }
    __device__ __forceinline__ void take(C (&v)[4], const C *stage) const {
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) v[n1] = stage[((size_t)n1 * kZ4Lanes + t) * lanes + (b * z4_tx<T>() + c)];
    }
    __device__ __forceinline__ void store(const C (&v)[4], C *dst, const Dims &d, size_t plane) const {
        if (!ok) return;
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) {
            const int zz = t + 64 * n1;
            if (zz < d.nz) dst[(size_t)zz * plane] = v[n1];
        }
    }
};

// Kernel-spectrum stage: K_type,i at lane t's four frequencies for column c
// at [((i * 4 + k4) * 64 + t) * TX + c] of buffer type & 1.  The pair's two
// rows read the same entries (either row's column exists iff kx < Wx); row b
// copies k4 = 2b, 2b + 1, one commit group per type.  A reader waits for the
// group and passes a barrier before its first read.
template <typename T, int S> constexpr size_t z4_spec_stride() { return (size_t)S * 4 * kZ4Lanes * z4_tx<T>(); }
template <typename T, int S>
__device__ __forceinline__ void z4_fetch_spec(T *gst, const T *__restrict__ spec, const Z4Lane<T> &ln, const Dims &d,
                                              int type) {
    constexpr int TX = z4_tx<T>();
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    const bool ok = ln.kx < d.Wx;
    T *dst = gst + (type & 1) * z4_spec_stride<T, S>();
#pragma unroll
    for (int i = 0; i < S; ++i) {
        const T *base = spec + (size_t)(i * kNumKernels + type) * oct + (size_t)ln.fy * d.Ox + ln.kx;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int k4 = 2 * ln.b + kk;
            z4_cp_scalar(&dst[((size_t)(i * 4 + k4) * kZ4Lanes + ln.t) * TX + ln.c],
                         ok ? &base[(size_t)ln.fz[k4] * d.Oy * d.Ox] : spec, ok);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
}
template <typename T, int S>
__device__ __forceinline__ T z4_spec_at(const T *gst, const Z4Lane<T> &ln, int type, int i, int k4) {
    return gst[(type & 1) * z4_spec_stride<T, S>() + ((size_t)(i * 4 + k4) * kZ4Lanes + ln.t) * z4_tx<T>() + ln.c];
}

// z MAC, L = 256: forward FFT of the S density columns (kept per lane in
// registers), the ten weighted-density spectra conj(K_alpha,i) rho_i summed
// over species, inverse FFT, rows z < nz.  grid (ceil(Wx/TX), Ly/2 + 1),
// block 128 TX.
template <typename T, int S>
__global__ void __launch_bounds__(512, 1) k_zmac_q4(const typename vec2<T>::type *__restrict__ Bs,
                                                    typename vec2<T>::type *__restrict__ B10, Dims d,
                                                    const typename vec2<T>::type *__restrict__ twz,
                                                    const T *__restrict__ spec, SpeciesConst sc) {
    using C = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Z4Lane<T> ln;
    ln.init(d, twz, smem_raw);
    const size_t plane = (size_t)d.Ly * d.Wx;
    C rs[S][4];
    C v[4];
    // kernel spectra staged one type ahead: type t + 1 is copied at the start
    // of type t (the inverse transforms of type t - 1 put barriers after every
    // thread's last read of that buffer) and published by a barrier at the
    // start of type t + 1
    T *gst = reinterpret_cast<T *>(smem_raw + z4_smem<T>());
    z4_fetch_spec<T, S>(gst, spec, ln, d, 0);
#pragma unroll
    for (int i = 0; i < S; ++i) {
        ln.load(v, Bs + (size_t)i * d.nz * plane + (size_t)ln.ky * d.Wx + ln.kx, d, plane);
        z4_fwd(v, ln.tw, ln.bufA, ln.bufB, ln.t, ln.lanes, ln.half);
#pragma unroll
        for (int k = 0; k < 4; ++k) rs[i][k] = v[k];
    }
    // output groups: shell {n0, n1, n2}, ball {n3}, vector x {n1x, n2x}, y, z
    for (int type = 0; type < kNumKernels; ++type) {
        const int nout = type == 0 ? 3 : (type == 1 ? 1 : 2);
        const bool flip_y = type == 3 && ln.ky > d.Ly / 2;
        if (type + 1 < kNumKernels) {
            z4_fetch_spec<T, S>(gst, spec, ln, d, type + 1);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();
        T g[S][4];
#pragma unroll
        for (int i = 0; i < S; ++i) {
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
                T gv = z4_spec_at<T, S>(gst, ln, type, i, k4);
                if (flip_y || (type == 4 && ln.hi[k4])) gv = -gv;
                g[i][k4] = gv;
            }
        }
        for (int o = 0; o < nout; ++o) {
            const int alpha = type == 0 ? o : (type == 1 ? 3 : (o == 0 ? 4 + type - 2 : 7 + type - 2));
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = C{0, 0};
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const T cf = alpha == 0 ? sc_c0<T>(sc, i)
                                        : ((alpha == 1 || (alpha >= 4 && alpha < 7)) ? sc_c1<T>(sc, i) : (T)1);
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const T gg = cf * g[i][k4];
                    const C x = rs[i][k4];
                    if (type <= 1) {
                        v[k4].x += gg * x.x;
                        v[k4].y += gg * x.y;
                    } else {             // conj(K) = +i S
                        v[k4].x -= gg * x.y;
                        v[k4].y += gg * x.x;
                    }
                }
            }
            z4_inv(v, ln.tw, ln.bufA, ln.bufB, ln.t, ln.lanes, ln.half);
            ln.store(v, B10 + (size_t)alpha * d.nz * plane + (size_t)ln.ky * d.Wx + ln.kx, d, plane);
        }
    }
}

// z back, L = 256: forward FFT of each Psi_alpha column, mu_i += K_alpha,i
// Psi_alpha into per-lane register accumulators, with MSA the pair kernels on
// the densities' y-spectra still in Bs (written over only at the end), then
// the inverse FFT of the S accumulators, rows z < nz.
template <typename T, int S, bool MSA>
__global__ void __launch_bounds__(512, 1) k_zback_q4(const typename vec2<T>::type *__restrict__ B10,
                                                     typename vec2<T>::type *__restrict__ Bs, Dims d,
                                                     const typename vec2<T>::type *__restrict__ twz,
                                                     const T *__restrict__ spec, SpeciesConst sc) {
    using C = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Z4Lane<T> ln;
    ln.init(d, twz, smem_raw);
    const size_t plane = (size_t)d.Ly * d.Wx;
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    C acc[S][4];
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[i][k] = C{0, 0};
    C v[4];
    // the ten Psi columns in the order (type, o) below; each lane prefetches
    // its values of the next column into its own slots of the other stage
    C *stage = reinterpret_cast<C *>(smem_raw) + z4_smem<T>() / sizeof(C);
    const size_t stage_stride = (size_t)4 * kZ4Lanes * ln.lanes;
    auto column = [&](int alpha) { return B10 + (size_t)alpha * d.nz * plane + (size_t)ln.ky * d.Wx + ln.kx; };
    // kernel spectra staged one type ahead: type t + 1 is copied after the
    // first forward transform of type t (whose barriers follow every
    // thread's last read of that buffer, type t - 1), completes with the next
    // column's wait and is published by the barriers of the next transform
    T *gst = reinterpret_cast<T *>(stage + 2 * stage_stride);
    ln.prefetch(stage, column(0), d, plane);
    z4_fetch_spec<T, S>(gst, spec, ln, d, 0);
    int seq = 0;
    // the column loop stays rolled: unrolled, its ten forward transforms
    // and products outgrow the instruction cache (ncu: 1.6 no-instruction
    // stalls per issue; 2.05 -> 1.83 ms at 128^3 -> 256^3 rolled)
#pragma unroll 1
    for (int type = 0; type < kNumKernels; ++type) {
        const int nin = type == 0 ? 3 : (type == 1 ? 1 : 2);
        const bool flip_y = type == 3 && ln.ky > d.Ly / 2;
#pragma unroll 1
        for (int o = 0; o < nin; ++o, ++seq) {
            const int alpha = type == 0 ? o : (type == 1 ? 3 : (o == 0 ? 4 + type - 2 : 7 + type - 2));
            if (seq + 1 < kNumWeighted) {
                const int t1 = o + 1 < nin ? type : type + 1, o1 = o + 1 < nin ? o + 1 : 0;
                const int a1 = t1 == 0 ? o1 : (t1 == 1 ? 3 : (o1 == 0 ? 4 + t1 - 2 : 7 + t1 - 2));
                ln.prefetch(stage + ((seq + 1) & 1) * stage_stride, column(a1), d, plane);
                asm volatile("cp.async.wait_group 1;\n" ::);
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::);
            }
            ln.take(v, stage + (seq & 1) * stage_stride);
            z4_fwd(v, ln.tw, ln.bufA, ln.bufB, ln.t, ln.lanes, ln.half);
            if (o == 0 && type + 1 < kNumKernels) z4_fetch_spec<T, S>(gst, spec, ln, d, type + 1);
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const T cf = alpha == 0 ? sc_c0<T>(sc, i)
                                        : ((alpha == 1 || (alpha >= 4 && alpha < 7)) ? sc_c1<T>(sc, i) : (T)1);
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    T g = z4_spec_at<T, S>(gst, ln, type, i, k4);
                    if (flip_y || (type == 4 && ln.hi[k4])) g = -g;
                    const T gg = cf * g;
                    const C x = v[k4];
                    if (type <= 1) {
                        acc[i][k4].x += gg * x.x;
                        acc[i][k4].y += gg * x.y;
                    } else {             // K = -i S
                        acc[i][k4].x += gg * x.y;
                        acc[i][k4].y -= gg * x.x;
                    }
                }
            }
        }
    }
    if constexpr (MSA) {
        // MSA correlations (Sec 2.3.4): mu_i -= sum_j C_ij rho_j, the stored
        // even spectra being -C_ij
#pragma unroll
        for (int j = 0; j < S; ++j) {
            ln.load(v, Bs + (size_t)j * d.nz * plane + (size_t)ln.ky * d.Wx + ln.kx, d, plane);
            z4_fwd(v, ln.tw, ln.bufA, ln.bufB, ln.t, ln.lanes, ln.half);
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const T *base = spec + (size_t)(S * kNumKernels + msa_pair(i, j, S)) * oct + (size_t)ln.fy * d.Ox +
                                ln.kx;
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const T gg = ln.ok ? ldgt(&base[(size_t)ln.fz[k4] * d.Oy * d.Ox]) : (T)0;
                    acc[i][k4].x += gg * v[k4].x;
                    acc[i][k4].y += gg * v[k4].y;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = acc[i][k];
        z4_inv(v, ln.tw, ln.bufA, ln.bufB, ln.t, ln.lanes, ln.half);
        ln.store(v, Bs + (size_t)i * d.nz * plane + (size_t)ln.ky * d.Wx + ln.kx, d, plane);
    }
}

}  // namespace pnp
