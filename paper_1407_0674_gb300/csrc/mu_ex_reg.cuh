// mu_ex pipeline kernels on the register-resident two-factor FFT
// (fft_reg.cuh).  Same passes, layouts and arithmetic as the shared-memory
// Stockham kernels in mu_ex.cu; used for every axis whose padded length has a
// two-factor shape (see fast_shape()).  Included by mu_ex.cu only.
#pragma once

#include <type_traits>

#include "fft_reg.cuh"

namespace pnp {

// R2C of two real lines packed as one complex line: given Z = FFT(a + i b)
// in natural order in `z`, write X = FFT(a), Y = FFT(b) for k < Wx.
template <typename C>
__device__ __forceinline__ void untangle_store(const C *z, int L, int Wx, int lane, int G, C *dst0, C *dst1) {
    using T = decltype(z[0].x);
    for (int k = lane; k < Wx; k += G) {
        const C zk = z[k];
        const C zm = z[(L - k) % L];
        dst0[k] = C{(T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)};
        if (dst1) dst1[k] = C{(T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x)};
    }
}

// Z_k = X_k + i Y_k for the half spectra X (line y0) and Y (line y0 + 1) of two
// real lines; k > L/2 from Hermitian symmetry.
template <typename C>
__device__ __forceinline__ C pack_two(const C *__restrict__ x0, const C *__restrict__ x1, int k, int L) {
    const bool up = k > L / 2;
    const int kk = up ? L - k : k;
    C X = x0[kk];
    C Y = x1 ? x1[kk] : C{0, 0};
    if (up) {
        X.y = -X.y;
        Y.y = -Y.y;
    }
    return C{X.x - Y.y, X.y + Y.x};
}

// resident 256-thread CTAs the x kernels are compiled for: two for
// double-float (at most 128 registers: 16 warps per SM instead of 8; the DF64
// x stages at 256 points take 1.32 -> 1.08 ms), none (the compiler's own
// choice) otherwise -- a minimum of one lets it raise the FP32 x inverse from
// 78 to 88 registers, two CTAs per SM instead of three
template <typename T> constexpr int xlines_min_blocks() { return std::is_same<T, dd>::value ? 2 : 0; }

// packed FP32x2 butterfly sums for the double-float 256-point x and y lines
template <typename T, int N1, int N2> constexpr bool lines_packed() {
    return std::is_same<T, dd>::value && N1 == 16 && N2 == 16;
}

// ---------------------------------------------------------------------------
// x forward (R2C, two real lines per complex FFT).  block P*G, grid (ceil(npairs/P), nz, F)
template <typename T, int N1, int N2, typename InT = double>
__global__ void __launch_bounds__(256, xlines_min_blocks<T>()) k_xfwd_r(const InT *__restrict__ in, size_t in_fstride,
                                                 typename vec2<T>::type *__restrict__ A, Dims d,
                                                 const typename vec2<T>::type *__restrict__ tw, int P) {
    using C = typename vec2<T>::type;
    constexpr int G = Shape<N1, N2>::G, EX = Shape<N1, N2>::EX, L = N1 * N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = threadIdx.x / G, t = threadIdx.x % G;
    C *ex = reinterpret_cast<C *>(smem_raw) + p * EX;
    const int z = blockIdx.y, f = blockIdx.z, y0 = 2 * (blockIdx.x * P + p);
    LaneTw<N1, N2, C> lt;
    lt.load(tw, t);
    C v[G];
    const InT *src = in + f * in_fstride + (size_t)z * d.ny * d.nx;
    if (t < N1) {
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
            const int x = t + N1 * n2;
            T re = 0, im = 0;
            if (x < d.nx && y0 < d.ny) {
                re = (T)src[(size_t)y0 * d.nx + x];
                if (y0 + 1 < d.ny) im = (T)src[(size_t)(y0 + 1) * d.nx + x];
            }
            v[n2] = C{re, im};
        }
    }
    fwd2<N1, N2, lines_packed<T, N1, N2>()>(v, lt, ex, t, 1, 2 * d.nx <= L);
    if (t < N2) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) ex[t + N2 * k1] = v[k1];
    }
    __syncthreads();
    if (y0 < d.ny) {
        C *dst = A + ((size_t)f * d.nz + z) * d.ny * d.Wx + (size_t)y0 * d.Wx;
        untangle_store(ex, L, d.Wx, t, G, dst, y0 + 1 < d.ny ? dst + d.Wx : (C *)nullptr);
    }
}

// x inverse (C2R) of F fields, write x < nx as FP64, optionally + coef * U
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(256, xlines_min_blocks<T>()) k_xinv_r(const typename vec2<T>::type *__restrict__ A,
                                                 double *__restrict__ out, size_t out_fstride, Dims d,
                                                 const typename vec2<T>::type *__restrict__ tw,
                                                 const double *__restrict__ U, SpeciesConst sc, int P,
                                                 const double *__restrict__ E) {
    using C = typename vec2<T>::type;
    constexpr int G = Shape<N1, N2>::G, EX = Shape<N1, N2>::EX, L = N1 * N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = threadIdx.x / G, t = threadIdx.x % G;
    C *ex = reinterpret_cast<C *>(smem_raw) + p * EX;
    const int z = blockIdx.y, f = blockIdx.z, y0 = 2 * (blockIdx.x * P + p);
    LaneTw<N1, N2, C> lt;
    lt.load(tw, t);
    C v[G];
    const C *src = A + ((size_t)f * d.nz + z) * d.ny * d.Wx + (size_t)y0 * d.Wx;
    if (t < N2) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1)
            v[k1] = y0 < d.ny ? pack_two(src, y0 + 1 < d.ny ? src + d.Wx : (const C *)nullptr, t + N2 * k1, L)
                              : C{0, 0};
    }
    inv2<N1, N2, lines_packed<T, N1, N2>()>(v, lt, ex, t, 1, 2 * d.nx <= L);
    if (t < N1 && y0 < d.ny) {
        double *dst = out + f * out_fstride + (size_t)z * d.ny * d.nx;
        const double coef = U ? sc.sh[f] : 0.0;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
            const int x = t + N1 * n2;
            if (x >= d.nx) continue;
            double u0 = 0, u1 = 0;
            if (U) {
                u0 = coef * U[((size_t)z * d.ny + y0) * d.nx + x];
                if (y0 + 1 < d.ny) u1 = coef * U[((size_t)z * d.ny + y0 + 1) * d.nx + x];
            }
            double r0 = (double)v[n2].x + u0, r1 = (double)v[n2].y + u1;
            if (E) {
                const double *e = E + f * out_fstride;
                r0 += e[((size_t)z * d.ny + y0) * d.nx + x];
                if (y0 + 1 < d.ny) r1 += e[((size_t)z * d.ny + y0 + 1) * d.nx + x];
            }
            dst[(size_t)y0 * d.nx + x] = r0;
            if (y0 + 1 < d.ny) dst[(size_t)(y0 + 1) * d.nx + x] = r1;
        }
    }
}

// x inverse (C2R) of F fields into real arrays of type OutT (x < nx), for the
// split form of the derivative stage
template <typename T, int N1, int N2, typename OutT>
__global__ void __launch_bounds__(256, xlines_min_blocks<T>()) k_xinv_raw_r(const typename vec2<T>::type *__restrict__ A,
                                                     OutT *__restrict__ out, Dims d,
                                                     const typename vec2<T>::type *__restrict__ tw, int P) {
    using C = typename vec2<T>::type;
    constexpr int G = Shape<N1, N2>::G, EX = Shape<N1, N2>::EX, L = N1 * N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = threadIdx.x / G, t = threadIdx.x % G;
    C *ex = reinterpret_cast<C *>(smem_raw) + p * EX;
    const int z = blockIdx.y, f = blockIdx.z, y0 = 2 * (blockIdx.x * P + p);
    LaneTw<N1, N2, C> lt;
    lt.load(tw, t);
    C v[G];
    const C *src = A + ((size_t)f * d.nz + z) * d.ny * d.Wx + (size_t)y0 * d.Wx;
    if (t < N2) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1)
            v[k1] = y0 < d.ny ? pack_two(src, y0 + 1 < d.ny ? src + d.Wx : (const C *)nullptr, t + N2 * k1, L)
                              : C{0, 0};
    }
    inv2<N1, N2, lines_packed<T, N1, N2>()>(v, lt, ex, t, 1, 2 * d.nx <= L);
    if (t < N1 && y0 < d.ny) {
        OutT *dst = out + ((size_t)f * d.nz + z) * d.ny * d.nx;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
            const int x = t + N1 * n2;
            if (x >= d.nx) continue;
            dst[(size_t)y0 * d.nx + x] = (OutT)v[n2].x;
            if (y0 + 1 < d.ny) dst[(size_t)(y0 + 1) * d.nx + x] = (OutT)v[n2].y;
        }
    }
}

// x fused: C2R of the ten n_alpha, FP64 dPhi/dn inside the domain, R2C of the
// ten Psi_alpha, in place in A.  Only the NQ = ceil(nx / N1) lane values that
// can hold x < nx are kept (Psi is zero beyond nx).
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(256) k_xfused_r(typename vec2<T>::type *__restrict__ A, Dims d,
                                                   const typename vec2<T>::type *__restrict__ tw,
                                                   int *__restrict__ flag, int P, int NQ) {
    using C = typename vec2<T>::type;
    constexpr int G = Shape<N1, N2>::G, EX = Shape<N1, N2>::EX, L = N1 * N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = threadIdx.x / G, t = threadIdx.x % G;
    C *slots = reinterpret_cast<C *>(smem_raw);                     // [10][NQ][P][N1]
    C *ex = slots + (size_t)kNumWeighted * NQ * P * N1 + p * EX;
    auto slot = [&](int a, int q) -> C & { return slots[((a * NQ + q) * P + p) * N1 + t]; };
    const int z = blockIdx.y, y0 = 2 * (blockIdx.x * P + p);
    const size_t fstride = (size_t)d.nz * d.ny * d.Wx;
    C *base = A + (size_t)z * d.ny * d.Wx + (size_t)y0 * d.Wx;
    const bool live = y0 < d.ny, two = y0 + 1 < d.ny;
    LaneTw<N1, N2, C> lt;
    lt.load(tw, t);
    C v[G];
    for (int a = 0; a < kNumWeighted; ++a) {
        if (t < N2) {
            const C *src = base + a * fstride;
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1)
                v[k1] = live ? pack_two(src, two ? src + d.Wx : (const C *)nullptr, t + N2 * k1, L) : C{0, 0};
        }
        inv2<N1, N2>(v, lt, ex, t, 1);
        if (t < N1) {
#pragma unroll
            for (int q = 0; q < N2; ++q)
                if (q < NQ) slot(a, q) = v[q];
        }
    }
    bool bad = false;
    if (t < N1) {
        for (int q = 0; q < NQ; ++q) {
            const int x = t + N1 * q;
            for (int h = 0; h < 2; ++h) {
                const int y = y0 + h;
                double n[kNumWeighted], psi[kNumWeighted];
#pragma unroll
                for (int a = 0; a < kNumWeighted; ++a) {
                    const C s = slot(a, q);
                    n[a] = (double)(h ? s.y : s.x);
                }
                if (x < d.nx && y < d.ny) {
                    if (!fmt_dphi(n, psi, d.fmt)) bad = true;
                } else {
#pragma unroll
                    for (int a = 0; a < kNumWeighted; ++a) psi[a] = 0.0;
                }
#pragma unroll
                for (int a = 0; a < kNumWeighted; ++a) {
                    C &s = slot(a, q);
                    if (h) s.y = (T)psi[a]; else s.x = (T)psi[a];
                }
            }
        }
    }
    if (bad) atomicOr(flag, kFlagPacking);
    for (int a = 0; a < kNumWeighted; ++a) {
        if (t < N1) {
#pragma unroll
            for (int q = 0; q < N2; ++q) v[q] = q < NQ ? slot(a, q) : C{0, 0};
        }
        fwd2<N1, N2>(v, lt, ex, t, 1);
        if (t < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) ex[t + N2 * k1] = v[k1];
        }
        __syncthreads();
        if (live) {
            C *dst = base + a * fstride;
            untangle_store(ex, L, d.Wx, t, G, dst, two ? dst + d.Wx : (C *)nullptr);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// y pass over TX half-spectrum columns; block TX*G with lane-major thread
// index (t * TX + c) so global accesses are contiguous over c.
template <typename T, bool INV, int N1, int N2>
__global__ void __launch_bounds__(256, xlines_min_blocks<T>()) k_ypass_r(const typename vec2<T>::type *__restrict__ in,
                                                  typename vec2<T>::type *__restrict__ out, Dims d, int rows_in,
                                                  int n_in, int rows_out, int n_out,
                                                  const typename vec2<T>::type *__restrict__ tw, int TX) {
    using C = typename vec2<T>::type;
    constexpr int G = Shape<N1, N2>::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x / TX, c = threadIdx.x % TX;
    C *ex = reinterpret_cast<C *>(smem_raw) + c;
    const int z = blockIdx.y, f = blockIdx.z, kx = blockIdx.x * TX + c;
    const bool ok = kx < d.Wx;
    const C *src = in + ((size_t)f * d.nz + z) * rows_in * d.Wx + kx;
    C *dst = out + ((size_t)f * d.nz + z) * rows_out * d.Wx + kx;
    LaneTw<N1, N2, C> lt;
    lt.load(tw, t);
    C v[G];
    if (!INV) {
        if (t < N1) {
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) {
                const int j = t + N1 * n2;
                v[n2] = (ok && j < n_in) ? src[(size_t)j * d.Wx] : C{0, 0};
            }
        }
        fwd2<N1, N2, lines_packed<T, N1, N2>()>(v, lt, ex, t, TX, 2 * n_in <= N1 * N2);
        if (t < N2 && ok) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
                const int j = t + N2 * k1;
                if (j < n_out) dst[(size_t)j * d.Wx] = v[k1];
            }
        }
    } else {
        if (t < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
                const int j = t + N2 * k1;
                v[k1] = (ok && j < n_in) ? src[(size_t)j * d.Wx] : C{0, 0};
            }
        }
        inv2<N1, N2, lines_packed<T, N1, N2>()>(v, lt, ex, t, TX, 2 * n_out <= N1 * N2);
        if (t < N1 && ok) {
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) {
                const int j = t + N1 * n2;
                if (j < n_out) dst[(size_t)j * d.Wx] = v[n2];
            }
        }
    }
}

}  // namespace pnp

namespace pnp {

// ---------------------------------------------------------------------------
// z kernels, paired-column form.  A CTA takes TX half-spectrum columns kx at
// the two rows ky' and Ly - ky' (which read the same kernel-spectrum octant
// entries), lanes (t, b, c) with c fastest.  The spectral products are grouped
// by kernel type (shell, ball, vector x, y, z), so each lane loads the s
// spectra of a type for its N1 frequencies in one batch.
template <int N1, int N2> struct ZTile {
    static constexpr int G = Shape<N1, N2>::G;
};

// column of lane (b, c) in tile (kx0, kyp): returns false if it does not exist
__device__ __forceinline__ bool zcol(const Dims &d, int kyp, int b, int kx, int &ky) {
    ky = b ? d.Ly - kyp : kyp;
    if (b && (ky == kyp || ky >= d.Ly)) return false;   // self-paired row (0 or Ly/2)
    return kx < d.Wx;
}

// spectrum values of `type` for species i0 .. i0 + kChunk - 1 (< s) at the
// N1 frequencies kz = t + N2 k1 of a lane
constexpr int kChunk = 3;
template <typename T, int N1, int N2>
__device__ __forceinline__ void load_spec(T (&g)[kChunk][N1], const T *__restrict__ spec, const Dims &d, int s,
                                          int i0, int type, int kx, int ky, int t, bool ok) {
    const int fy = ky <= d.Ly / 2 ? ky : d.Ly - ky;
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    const bool flip_y = type == 3 && ky > d.Ly / 2;
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
        const int i = i0 + j;
        const bool have = ok && i < s;
        const T *base = spec + (size_t)((have ? i : 0) * kNumKernels + type) * oct + (size_t)fy * d.Ox + kx;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            const int kz = t + N2 * k1;
            const int fz = kz <= d.Lz / 2 ? kz : d.Lz - kz;
            T v = have ? ldgt(&base[(size_t)fz * d.Oy * d.Ox]) : (T)0;
            if (flip_y || (type == 4 && kz > d.Lz / 2)) v = -v;
            g[j][k1] = v;
        }
    }
}

template <typename T, int N1, int N2>
__global__ void __launch_bounds__(256) k_zmac_p(const typename vec2<T>::type *__restrict__ Bs,
                                                 typename vec2<T>::type *__restrict__ B10, Dims d,
                                                 const typename vec2<T>::type *__restrict__ tw,
                                                 const T *__restrict__ spec, SpeciesConst sc, int TX) {
    using C = typename vec2<T>::type;
    constexpr int G = Shape<N1, N2>::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = threadIdx.x % TX, b = (threadIdx.x / TX) & 1, t = threadIdx.x / (2 * TX);
    const int lanes = 2 * TX;                        // interleaved columns in the tile
    const int col = b * TX + c;
    C *slots = reinterpret_cast<C *>(smem_raw);      // [s][N1][G][2 TX]
    C *ex = slots + (size_t)sc.s * N1 * G * lanes + col;
    const int rstride = N1 * G * lanes;
    auto slot = [&](int i, int k1) -> C & { return slots[i * rstride + (k1 * G + t) * lanes + col]; };
    const int kyp = blockIdx.y, kx = blockIdx.x * TX + c;
    int ky;
    const bool ok = zcol(d, kyp, b, kx, ky);
    const size_t plane = (size_t)d.Ly * d.Wx;
    // 64-bit types: lane twiddles from a shared table (frees 2 G registers);
    // FP32 keeps them in registers
    C *twtab = slots + (size_t)sc.s * N1 * G * lanes + (size_t)Shape<N1, N2>::EX * lanes;
    using TwT = typename std::conditional<std::is_same<T, float>::value, LaneTw<N1, N2, C>, SmemTw<N1, N2, C>>::type;
    TwT lt;
    if constexpr (std::is_same<T, float>::value) {
        lt.load(tw, t);
    } else {
        SmemTw<N1, N2, C>::fill(twtab, tw);
        __syncthreads();
        lt.tab = twtab;
        lt.t = t;
    }
    C v[G];
    for (int i = 0; i < sc.s; ++i) {
        const C *src = Bs + (size_t)i * d.nz * plane + (size_t)ky * d.Wx + kx;
        if (t < N1) {
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) {
                const int zz = t + N1 * n2;
                v[n2] = (ok && zz < d.nz) ? src[(size_t)zz * plane] : C{0, 0};
            }
        }
        fwd2<N1, N2>(v, lt, ex, t, lanes);
        if (t < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) slot(i, k1) = v[k1];
        }
    }
    // output groups: shell {n0, n1, n2}, ball {n3}, vector x {n1x, n2x}, y, z;
    // with s <= kChunk the group's spectra are loaded once
    for (int type = 0; type < kNumKernels; ++type) {
        T g[kChunk][N1];
        const int nout = type == 0 ? 3 : (type == 1 ? 1 : 2);
        for (int o = 0; o < nout; ++o) {
            const int alpha = type == 0 ? o : (type == 1 ? 3 : (o == 0 ? 4 + type - 2 : 7 + type - 2));
            if (t < N2) {
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) v[k1] = C{0, 0};
                for (int i0 = 0; i0 < sc.s; i0 += kChunk) {
                    if (o == 0 || sc.s > kChunk) load_spec<T, N1, N2>(g, spec, d, sc.s, i0, type, kx, ky, t, ok);
#pragma unroll
                    for (int j = 0; j < kChunk; ++j) {
                        const int i = i0 + j;
                        if (i >= sc.s) break;
                        const T cf = alpha == 0 ? sc_c0<T>(sc, i)
                                                : ((alpha == 1 || (alpha >= 4 && alpha < 7)) ? sc_c1<T>(sc, i) : (T)1);
#pragma unroll
                        for (int k1 = 0; k1 < N1; ++k1) {
                            const T gg = cf * g[j][k1];
                            const C x = slot(i, k1);
                            if (type <= 1) {
                                v[k1].x += gg * x.x;
                                v[k1].y += gg * x.y;
                            } else {             // conj(K) = +i S
                                v[k1].x -= gg * x.y;
                                v[k1].y += gg * x.x;
                            }
                        }
                    }
                }
            }
            inv2<N1, N2>(v, lt, ex, t, lanes);
            if (t < N1 && ok) {
                C *dst = B10 + (size_t)alpha * d.nz * plane + (size_t)ky * d.Wx + kx;
#pragma unroll
                for (int n2 = 0; n2 < N2; ++n2) {
                    const int zz = t + N1 * n2;
                    if (zz < d.nz) dst[(size_t)zz * plane] = v[n2];
                }
            }
        }
    }
}

template <typename T, int N1, int N2, bool MSA = false>
__global__ void __launch_bounds__(256) k_zback_p(const typename vec2<T>::type *__restrict__ B10,
                                                  typename vec2<T>::type *__restrict__ Bs, Dims d,
                                                  const typename vec2<T>::type *__restrict__ tw,
                                                  const T *__restrict__ spec, SpeciesConst sc, int TX) {
    using C = typename vec2<T>::type;
    constexpr int G = Shape<N1, N2>::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = threadIdx.x % TX, b = (threadIdx.x / TX) & 1, t = threadIdx.x / (2 * TX);
    const int lanes = 2 * TX;
    const int col = b * TX + c;
    C *slots = reinterpret_cast<C *>(smem_raw);      // accumulators [s][N1][G][2 TX]
    C *ex = slots + (size_t)sc.s * N1 * G * lanes + col;
    const int rstride = N1 * G * lanes;
    auto slot = [&](int i, int k1) -> C & { return slots[i * rstride + (k1 * G + t) * lanes + col]; };
    const int kyp = blockIdx.y, kx = blockIdx.x * TX + c;
    int ky;
    const bool ok = zcol(d, kyp, b, kx, ky);
    const size_t plane = (size_t)d.Ly * d.Wx;
    // 64-bit types: lane twiddles from a shared table (frees 2 G registers);
    // FP32 keeps them in registers
    C *twtab = slots + (size_t)sc.s * N1 * G * lanes + (size_t)Shape<N1, N2>::EX * lanes;
    using TwT = typename std::conditional<std::is_same<T, float>::value, LaneTw<N1, N2, C>, SmemTw<N1, N2, C>>::type;
    TwT lt;
    if constexpr (std::is_same<T, float>::value) {
        lt.load(tw, t);
    } else {
        SmemTw<N1, N2, C>::fill(twtab, tw);
        __syncthreads();
        lt.tab = twtab;
        lt.t = t;
    }
    C v[G];
    if (t < N2)
        for (int i = 0; i < sc.s; ++i)
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) slot(i, k1) = C{0, 0};
    for (int type = 0; type < kNumKernels; ++type) {
        T g[kChunk][N1];
        const int nin = type == 0 ? 3 : (type == 1 ? 1 : 2);
        for (int o = 0; o < nin; ++o) {
            const int alpha = type == 0 ? o : (type == 1 ? 3 : (o == 0 ? 4 + type - 2 : 7 + type - 2));
            const C *src = B10 + (size_t)alpha * d.nz * plane + (size_t)ky * d.Wx + kx;
            if (t < N1) {
#pragma unroll
                for (int n2 = 0; n2 < N2; ++n2) {
                    const int zz = t + N1 * n2;
                    v[n2] = (ok && zz < d.nz) ? src[(size_t)zz * plane] : C{0, 0};
                }
            }
            fwd2<N1, N2>(v, lt, ex, t, lanes);
            if (t < N2) {
                for (int i0 = 0; i0 < sc.s; i0 += kChunk) {
                    if (o == 0 || sc.s > kChunk) load_spec<T, N1, N2>(g, spec, d, sc.s, i0, type, kx, ky, t, ok);
#pragma unroll
                    for (int j = 0; j < kChunk; ++j) {
                        const int i = i0 + j;
                        if (i >= sc.s) break;
                        const T cf = alpha == 0 ? sc_c0<T>(sc, i)
                                                : ((alpha == 1 || (alpha >= 4 && alpha < 7)) ? sc_c1<T>(sc, i) : (T)1);
#pragma unroll
                        for (int k1 = 0; k1 < N1; ++k1) {
                            const T gg = cf * g[j][k1];
                            const C x = v[k1];
                            C &acc = slot(i, k1);
                            if (type <= 1) {
                                acc.x += gg * x.x;
                                acc.y += gg * x.y;
                            } else {             // K = -i S
                                acc.x += gg * x.y;
                                acc.y -= gg * x.x;
                            }
                        }
                    }
                }
            }
        }
    }
    if constexpr (MSA) {
        // MSA correlations (Sec 2.3.4): Bs still holds the densities'
        // y-spectra (written over only below); mu_i -= sum_j C_ij rho_j, the
        // stored even spectra being -C_ij
        const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
        const int fy = ky <= d.Ly / 2 ? ky : d.Ly - ky;
        for (int j = 0; j < sc.s; ++j) {
            const C *src = Bs + (size_t)j * d.nz * plane + (size_t)ky * d.Wx + kx;
            if (t < N1) {
#pragma unroll
                for (int n2 = 0; n2 < N2; ++n2) {
                    const int zz = t + N1 * n2;
                    v[n2] = (ok && zz < d.nz) ? src[(size_t)zz * plane] : C{0, 0};
                }
            }
            fwd2<N1, N2>(v, lt, ex, t, lanes);
            if (t < N2) {
                for (int i = 0; i < sc.s; ++i) {
                    const T *base = spec + (size_t)(sc.s * kNumKernels + msa_pair(i, j, sc.s)) * oct +
                                    (size_t)fy * d.Ox + kx;
#pragma unroll
                    for (int k1 = 0; k1 < N1; ++k1) {
                        const int kz = t + N2 * k1;
                        const int fz = kz <= d.Lz / 2 ? kz : d.Lz - kz;
                        const T gg = ok ? ldgt(&base[(size_t)fz * d.Oy * d.Ox]) : (T)0;
                        C &acc = slot(i, k1);
                        acc.x += gg * v[k1].x;
                        acc.y += gg * v[k1].y;
                    }
                }
            }
        }
    }
    for (int i = 0; i < sc.s; ++i) {
        if (t < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) v[k1] = slot(i, k1);
        }
        inv2<N1, N2>(v, lt, ex, t, lanes);
        if (t < N1 && ok) {
            C *dst = Bs + (size_t)i * d.nz * plane + (size_t)ky * d.Wx + kx;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) {
                const int zz = t + N1 * n2;
                if (zz < d.nz) dst[(size_t)zz * plane] = v[n2];
            }
        }
    }
}

}  // namespace pnp

namespace pnp {

// ---------------------------------------------------------------------------
// FP32 z kernels with the per-column spectral state in registers: square
// two-factor shapes (L = 16, 64, 256), at most three species.  Each lane keeps
// its S x N1 accumulators (z back) or transformed density values (z MAC) in
// registers instead of a shared-memory slot per product, the lane twiddles
// come from a shared table, and each kernel type's spectra for the CTA's
// columns are staged in shared memory by cp.async while the first column of
// the type is transformed.  Problems with the MSA term keep k_zback_p (its
// extra pair loop would spill here).  Measured at 128^3 -> 256^3: z back 0.648 -> 0.549
// ms, z MAC 0.505 -> 0.487 ms against k_zback_p / k_zmac_p.

__device__ __forceinline__ void cp_async_f32(float *smem, const float *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_wait_all_groups() { asm volatile("cp.async.wait_all;\n" ::); }

// spectra of kernel `type` for species i < S at (fz < Oz, kx0 + c < Ox) of
// the CTA's fold row fy: specS[(i * Oz + fz) * TX + c]; out-of-range kx is
// zero-filled
__device__ __forceinline__ void stage_type_spectra(float *specS, const float *__restrict__ spec, const Dims &d,
                                                   int S, int type, int fy, int kx0, int TX) {
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    const int n = S * d.Oz * TX;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int c = k % TX, fz = (k / TX) % d.Oz, i = k / (TX * d.Oz);
        const int kx = kx0 + c;
        const bool ok = kx < d.Ox;
        cp_async_f32(specS + k,
                     spec + (size_t)(i * kNumKernels + type) * oct + ((size_t)fz * d.Oy + fy) * d.Ox + (ok ? kx : 0),
                     ok);
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

// shared memory of a register-state CTA: exchange buffers, staged spectra,
// twiddle table
template <int N1, int N2> inline size_t zreg_smem(const Dims &d, int S, int TX) {
    const size_t ex = (size_t)Shape<N1, N2>::EX * 2 * TX * sizeof(float2);
    const size_t sp = ((size_t)S * d.Oz * TX * sizeof(float) + 7) / 8 * 8;
    return ex + sp + (size_t)Shape<N1, N2>::G * Shape<N1, N2>::G * sizeof(float2);
}

template <int N1, int N2, int S>
__global__ void __launch_bounds__(128, 2) k_zback_reg(const float2 *__restrict__ B10, float2 *__restrict__ Bs, Dims d,
                                                      const float2 *__restrict__ tw, const float *__restrict__ spec,
                                                      SpeciesConst sc, int TX) {
    using C = float2;
    using T = float;
    constexpr int G = Shape<N1, N2>::G;
    static_assert(N1 == G && N2 == G, "square shapes only");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = threadIdx.x % TX, b = (threadIdx.x / TX) & 1, t = threadIdx.x / (2 * TX);
    const int lanes = 2 * TX;
    C *ex = reinterpret_cast<C *>(smem_raw) + (b * TX + c);
    float *specS = reinterpret_cast<float *>(reinterpret_cast<C *>(smem_raw) + (size_t)Shape<N1, N2>::EX * lanes);
    C *twtab = reinterpret_cast<C *>(smem_raw) + (size_t)Shape<N1, N2>::EX * lanes +
               ((size_t)S * d.Oz * TX * sizeof(float) + sizeof(C) - 1) / sizeof(C);
    const int kyp = blockIdx.y, kx0 = blockIdx.x * TX, kx = kx0 + c;
    int ky;
    const bool ok = zcol(d, kyp, b, kx, ky);
    const int fy = kyp;
    const size_t plane = (size_t)d.Ly * d.Wx;
    SmemTw<N1, N2, C>::fill(twtab, tw);
    __syncthreads();
    SmemTw<N1, N2, C> lt;
    lt.tab = twtab;
    lt.t = t;
    C v[G];
    C acc[S][N1];
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) acc[i][k1] = C{0, 0};
    for (int type = 0; type < kNumKernels; ++type) {
        const int nin = type == 0 ? 3 : (type == 1 ? 1 : 2);
        const bool flip_y = type == 3 && ky > d.Ly / 2;
        for (int o = 0; o < nin; ++o) {
            const int alpha = type == 0 ? o : (type == 1 ? 3 : (o == 0 ? 4 + type - 2 : 7 + type - 2));
            const C *src = B10 + (size_t)alpha * d.nz * plane + (size_t)ky * d.Wx + kx;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) {
                const int zz = t + N1 * n2;
                v[n2] = (ok && zz < d.nz) ? src[(size_t)zz * plane] : C{0, 0};
            }
            if (o == 0) {
                __syncthreads();      // every lane is done with the previous type's spectra
                stage_type_spectra(specS, spec, d, S, type, fy, kx0, TX);
            }
            fwd2<N1, N2>(v, lt, ex, t, lanes);
            if (o == 0) {
                cp_async_wait_all_groups();
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const T cf = alpha == 0 ? sc_c0<T>(sc, i)
                                        : ((alpha == 1 || (alpha >= 4 && alpha < 7)) ? sc_c1<T>(sc, i) : (T)1);
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) {
                    const int kz = t + N2 * k1;
                    const int fz = kz <= d.Lz / 2 ? kz : d.Lz - kz;
                    T g = specS[(i * d.Oz + fz) * TX + c];
                    if (flip_y || (type == 4 && kz > d.Lz / 2)) g = -g;
                    const T gg = cf * g;
                    const C x = v[k1];
                    if (type <= 1) {
                        acc[i][k1].x += gg * x.x;
                        acc[i][k1].y += gg * x.y;
                    } else {             // K = -i S
                        acc[i][k1].x += gg * x.y;
                        acc[i][k1].y -= gg * x.x;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = acc[i][k1];
        inv2<N1, N2>(v, lt, ex, t, lanes);
        if (ok) {
            C *dst = Bs + (size_t)i * d.nz * plane + (size_t)ky * d.Wx + kx;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) {
                const int zz = t + N1 * n2;
                if (zz < d.nz) dst[(size_t)zz * plane] = v[n2];
            }
        }
    }
}

template <int N1, int N2, int S>
__global__ void __launch_bounds__(128, 2) k_zmac_reg(const float2 *__restrict__ Bs, float2 *__restrict__ B10, Dims d,
                                                     const float2 *__restrict__ tw, const float *__restrict__ spec,
                                                     SpeciesConst sc, int TX) {
    using C = float2;
    using T = float;
    constexpr int G = Shape<N1, N2>::G;
    static_assert(N1 == G && N2 == G, "square shapes only");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = threadIdx.x % TX, b = (threadIdx.x / TX) & 1, t = threadIdx.x / (2 * TX);
    const int lanes = 2 * TX;
    C *ex = reinterpret_cast<C *>(smem_raw) + (b * TX + c);
    float *specS = reinterpret_cast<float *>(reinterpret_cast<C *>(smem_raw) + (size_t)Shape<N1, N2>::EX * lanes);
    C *twtab = reinterpret_cast<C *>(smem_raw) + (size_t)Shape<N1, N2>::EX * lanes +
               ((size_t)S * d.Oz * TX * sizeof(float) + sizeof(C) - 1) / sizeof(C);
    const int kyp = blockIdx.y, kx0 = blockIdx.x * TX, kx = kx0 + c;
    int ky;
    const bool ok = zcol(d, kyp, b, kx, ky);
    const int fy = kyp;
    const size_t plane = (size_t)d.Ly * d.Wx;
    SmemTw<N1, N2, C>::fill(twtab, tw);
    __syncthreads();
    SmemTw<N1, N2, C> lt;
    lt.tab = twtab;
    lt.t = t;
    C v[G];
    C rs[S][N1];
#pragma unroll
    for (int i = 0; i < S; ++i) {
        const C *src = Bs + (size_t)i * d.nz * plane + (size_t)ky * d.Wx + kx;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
            const int zz = t + N1 * n2;
            v[n2] = (ok && zz < d.nz) ? src[(size_t)zz * plane] : C{0, 0};
        }
        if (i == 0) stage_type_spectra(specS, spec, d, S, 0, fy, kx0, TX);
        fwd2<N1, N2>(v, lt, ex, t, lanes);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) rs[i][k1] = v[k1];
    }
    // output groups: shell {n0, n1, n2}, ball {n3}, vector x {n1x, n2x}, y, z
    for (int type = 0; type < kNumKernels; ++type) {
        if (type > 0) {
            __syncthreads();          // every lane is done with the previous type's spectra
            stage_type_spectra(specS, spec, d, S, type, fy, kx0, TX);
        }
        cp_async_wait_all_groups();
        __syncthreads();
        const int nout = type == 0 ? 3 : (type == 1 ? 1 : 2);
        const bool flip_y = type == 3 && ky > d.Ly / 2;
        for (int o = 0; o < nout; ++o) {
            const int alpha = type == 0 ? o : (type == 1 ? 3 : (o == 0 ? 4 + type - 2 : 7 + type - 2));
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) v[k1] = C{0, 0};
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const T cf = alpha == 0 ? sc_c0<T>(sc, i)
                                        : ((alpha == 1 || (alpha >= 4 && alpha < 7)) ? sc_c1<T>(sc, i) : (T)1);
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) {
                    const int kz = t + N2 * k1;
                    const int fz = kz <= d.Lz / 2 ? kz : d.Lz - kz;
                    T g = specS[(i * d.Oz + fz) * TX + c];
                    if (flip_y || (type == 4 && kz > d.Lz / 2)) g = -g;
                    const T gg = cf * g;
                    const C x = rs[i][k1];
                    if (type <= 1) {
                        v[k1].x += gg * x.x;
                        v[k1].y += gg * x.y;
                    } else {             // conj(K) = +i S
                        v[k1].x -= gg * x.y;
                        v[k1].y += gg * x.x;
                    }
                }
            }
            inv2<N1, N2>(v, lt, ex, t, lanes);
            if (ok) {
                C *dst = B10 + (size_t)alpha * d.nz * plane + (size_t)ky * d.Wx + kx;
#pragma unroll
                for (int n2 = 0; n2 < N2; ++n2) {
                    const int zz = t + N1 * n2;
                    if (zz < d.nz) dst[(size_t)zz * plane] = v[n2];
                }
            }
        }
    }
}

}  // namespace pnp
