// Excess chemical potential mu_ex = mu_hs + mu_sh by zero-padded FFT
// convolution (Sec 3.4) of the quadrature stencils of Sec 3.5.
//
// Pipeline for s species on an nx x ny x nz grid padded to Lx x Ly x Lz
// (Wx = Lx/2 + 1 half-spectrum columns).  Passes only touch the lines that can
// be non-zero (input inside the domain) or that are needed (output inside the
// domain), so a zero-extended axis costs about half a full transform:
//   1 x-fwd   : rho_i real lines -> R2C (two lines per complex FFT)   [s][nz][ny][Wx]
//   2 y-fwd   : ny -> Ly                                              [s][nz][Ly][Wx]
//   3 z-mac   : per (ky,kx) column: FFT_z(rho_i), n_alpha = sum_i conj(K_alpha,i) rho_i,
//               inverse FFT_z, keep z < nz                            [10][nz][Ly][Wx]
//   4 y-inv   : Ly -> ny                                              [10][nz][ny][Wx]
//   5 x-fused : C2R of the ten n_alpha, Rosenfeld dPhi/dn_alpha in FP64 masked to
//               the domain (Sec 2.3.1), R2C of the ten Psi_alpha      [10][nz][ny][Wx]
//   6 y-fwd   : ny -> Ly                                              [10][nz][Ly][Wx]
//   7 z-back  : FFT_z(Psi_alpha), mu_i = sum_alpha K_alpha,i Psi_alpha, inverse, z < nz
//   8 y-inv   : Ly -> ny                                              [s][nz][ny][Wx]
//   9 x-inv   : C2R, + mu_sh,i, write rho-shaped output
// The kernel spectra are stored as one real octant per kernel (the stencils
// are even or odd in each axis) with 1/(Lx Ly Lz) folded in.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <type_traits>
#include <vector>

#include "fft_smem.cuh"
#include "pnp_internal.h"

namespace pnp {

struct Dims {
    int nx, ny, nz;
    int Lx, Ly, Lz;
    int Wx;            // Lx / 2 + 1
    int Ox, Oy, Oz;    // octant extents
    int npairs;        // (ny + 1) / 2
};

struct SpeciesConst {
    int s;
    double c0[8];      // 1 / (4 pi R^2)
    double c1[8];      // 1 / (4 pi R)
    double sh[8];      // mu_sh coefficient
    float c0f[8], c1f[8];   // the same, pre-rounded for FP32 kernels
};

template <typename T> __device__ __forceinline__ T sc_c0(const SpeciesConst &sc, int i);
template <> __device__ __forceinline__ double sc_c0<double>(const SpeciesConst &sc, int i) { return sc.c0[i]; }
template <> __device__ __forceinline__ float sc_c0<float>(const SpeciesConst &sc, int i) { return sc.c0f[i]; }
template <typename T> __device__ __forceinline__ T sc_c1(const SpeciesConst &sc, int i);
template <> __device__ __forceinline__ double sc_c1<double>(const SpeciesConst &sc, int i) { return sc.c1[i]; }
template <> __device__ __forceinline__ float sc_c1<float>(const SpeciesConst &sc, int i) { return sc.c1f[i]; }

struct DeviceBuffers {
    int prec = 0;
    void *tw[3] = {nullptr, nullptr, nullptr};
    void *spec = nullptr;      // [s][5][Oz][Oy][Ox]
    size_t bytes = 0;
};

static Dims make_dims(const Problem *p) {
    Dims d;
    d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
    d.Lx = p->L[0]; d.Ly = p->L[1]; d.Lz = p->L[2];
    d.Wx = d.Lx / 2 + 1;
    d.Ox = d.Lx / 2 + 1; d.Oy = d.Ly / 2 + 1; d.Oz = d.Lz / 2 + 1;
    d.npairs = (d.ny + 1) / 2;
    return d;
}

static SpeciesConst make_sc(const Problem *p) {
    SpeciesConst sc{};
    sc.s = p->s;
    for (int i = 0; i < p->s; ++i) {
        sc.c0[i] = 1.0 / (4.0 * M_PI * p->R[i] * p->R[i]);
        sc.c1[i] = 1.0 / (4.0 * M_PI * p->R[i]);
        sc.sh[i] = p->has_wells ? p->sh_coef[i] : 0.0;
        sc.c0f[i] = (float)sc.c0[i];
        sc.c1f[i] = (float)sc.c1[i];
    }
    return sc;
}

// ---------------------------------------------------------------------------
// spectrum lookup: kernel `type` (0 shell, 1 ball, 2..4 vector x,y,z) of
// species i at half-spectrum index (kx, ky, kz); vector kernels carry the
// sign of their odd axis.
template <typename T>
__device__ __forceinline__ T spec_at(const T *__restrict__ sp, const Dims &d, int i, int type, int kx, int ky,
                                     int kz) {
    const int fy = ky <= d.Ly / 2 ? ky : d.Ly - ky;
    const int fz = kz <= d.Lz / 2 ? kz : d.Lz - kz;
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    T v = __ldg(&sp[(size_t)(i * kNumKernels + type) * oct + ((size_t)fz * d.Oy + fy) * d.Ox + kx]);
    if (type == 3 && ky > d.Ly / 2) v = -v;
    if (type == 4 && kz > d.Lz / 2) v = -v;
    return v;
}

// Rosenfeld FMT derivatives of Sec 2.3.1, FP64.
__device__ __forceinline__ bool fmt_dphi(const double n[kNumWeighted], double psi[kNumWeighted]) {
    const double n0 = n[0], n1 = n[1], n2 = n[2], n3 = n[3];
    const double g = 1.0 / (1.0 - n3);
    const double g2 = g * g;
    const double v1v2 = n[4] * n[7] + n[5] * n[8] + n[6] * n[9];
    const double v2v2 = n[7] * n[7] + n[8] * n[8] + n[9] * n[9];
    psi[0] = -log1p(-n3);
    psi[1] = n2 * g;
    psi[2] = n1 * g + (n2 * n2 - v2v2) * g2 * (1.0 / (8.0 * M_PI));
    psi[3] = n0 * g + (n1 * n2 - v1v2) * g2 + (n2 * n2 * n2 - 3.0 * n2 * v2v2) * g2 * g * (1.0 / (12.0 * M_PI));
    for (int c = 0; c < 3; ++c) {
        psi[4 + c] = -n[7 + c] * g;
        psi[7 + c] = -n[4 + c] * g - n2 * n[7 + c] * g2 * (1.0 / (4.0 * M_PI));
    }
    bool ok = n3 < 1.0;
    for (int a = 0; a < kNumWeighted; ++a) ok = ok && isfinite(psi[a]);
    return ok;
}

}  // namespace pnp

#include "mu_ex_reg.cuh"

namespace pnp {

// ---------------------------------------------------------------------------
// 1: real lines (FP64 input) -> half spectra along x.  Two y-lines share one
// complex FFT.  grid (ceil(npairs/P), nz, F).
template <typename T>
__global__ void k_xfwd(const double *__restrict__ in, size_t in_fstride, typename vec2<T>::type *__restrict__ A,
                       Dims d, FftAxis ax, const typename vec2<T>::type *__restrict__ tw, int P) {
    using C = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + (size_t)P * d.Lx;
    const int z = blockIdx.y, f = blockIdx.z;
    const int pair0 = blockIdx.x * P;
    const double *src = in + f * in_fstride + (size_t)z * d.ny * d.nx;
    for (int idx = threadIdx.x; idx < P * d.Lx; idx += blockDim.x) {
        const int p = idx / d.Lx, x = idx % d.Lx;
        const int y0 = 2 * (pair0 + p);
        T re = 0, im = 0;
        if (x < d.nx && y0 < d.ny) {
            re = (T)src[(size_t)y0 * d.nx + x];
            if (y0 + 1 < d.ny) im = (T)src[(size_t)(y0 + 1) * d.nx + x];
        }
        a[x * P + p] = C{re, im};
    }
    __syncthreads();
    C *r = fft_lines<false>(a, b, P, ax, tw);
    C *dst = A + ((size_t)f * d.nz + z) * d.ny * d.Wx;
    for (int idx = threadIdx.x; idx < P * d.Wx; idx += blockDim.x) {
        const int p = idx / d.Wx, k = idx % d.Wx;
        const int y0 = 2 * (pair0 + p);
        if (y0 >= d.ny) continue;
        C zk = r[k * P + p];
        C zm = r[((d.Lx - k) % d.Lx) * P + p];
        // X = (Z_k + conj Z_{L-k}) / 2,  Y = (Z_k - conj Z_{L-k}) / (2i)
        C X = C{(T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)};
        C Y = C{(T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x)};
        dst[(size_t)y0 * d.Wx + k] = X;
        if (y0 + 1 < d.ny) dst[(size_t)(y0 + 1) * d.Wx + k] = Y;
    }
}

// ---------------------------------------------------------------------------
// 2/4/6/8: complex FFT along y of TX half-spectrum columns.  Input rows
// j < n_in of an array with rows_in rows per plane (others are zero); output
// rows j < n_out of an array with rows_out rows per plane.  grid (ceil(Wx/TX), nz, F).
template <typename T, bool INV>
__global__ void k_ypass(const typename vec2<T>::type *__restrict__ in, typename vec2<T>::type *__restrict__ out,
                        Dims d, int rows_in, int n_in, int rows_out, int n_out, FftAxis ax,
                        const typename vec2<T>::type *__restrict__ tw, int TX) {
    using C = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + (size_t)TX * d.Ly;
    const int z = blockIdx.y, f = blockIdx.z, kx0 = blockIdx.x * TX;
    const C *src = in + ((size_t)f * d.nz + z) * rows_in * d.Wx;
    for (int idx = threadIdx.x; idx < TX * d.Ly; idx += blockDim.x) {
        const int j = idx / TX, c = idx % TX, kx = kx0 + c;
        C v = C{0, 0};
        if (j < n_in && kx < d.Wx) v = src[(size_t)j * d.Wx + kx];
        a[j * TX + c] = v;
    }
    __syncthreads();
    C *r = fft_lines<INV>(a, b, TX, ax, tw);
    C *dst = out + ((size_t)f * d.nz + z) * rows_out * d.Wx;
    for (int idx = threadIdx.x; idx < TX * n_out; idx += blockDim.x) {
        const int j = idx / TX, c = idx % TX, kx = kx0 + c;
        if (kx < d.Wx) dst[(size_t)j * d.Wx + kx] = r[j * TX + c];
    }
}

// ---------------------------------------------------------------------------
// 3: per (ky, kx-tile) column: forward z-FFT of the s density columns, the
// weighted-density spectra n_alpha = sum_i conj(K_alpha,i) rho_i, inverse
// z-FFT, rows z < nz.  grid (ceil(Wx/TX), Ly).
template <typename T>
__global__ void k_zmac(const typename vec2<T>::type *__restrict__ Bs, typename vec2<T>::type *__restrict__ B10,
                       Dims d, FftAxis ax, const typename vec2<T>::type *__restrict__ tw, const T *__restrict__ spec,
                       SpeciesConst sc, int TX) {
    using C = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int col = TX * d.Lz;
    C *rho = reinterpret_cast<C *>(smem_raw);   // s columns
    C *work = rho + (size_t)sc.s * col;
    C *scr = work + col;
    const int ky = blockIdx.y, kx0 = blockIdx.x * TX;
    for (int i = 0; i < sc.s; ++i) {
        const C *src = Bs + (size_t)i * d.nz * d.Ly * d.Wx + (size_t)ky * d.Wx;
        C *dst = rho + (size_t)i * col;
        for (int idx = threadIdx.x; idx < col; idx += blockDim.x) {
            const int j = idx / TX, c = idx % TX, kx = kx0 + c;
            C v = C{0, 0};
            if (j < d.nz && kx < d.Wx) v = src[(size_t)j * d.Ly * d.Wx + kx];
            dst[idx] = v;
        }
        __syncthreads();
        fft_lines_inplace<false>(dst, scr, TX, ax, tw);
    }
    for (int alpha = 0; alpha < kNumWeighted; ++alpha) {
        for (int idx = threadIdx.x; idx < col; idx += blockDim.x) {
            const int kz = idx / TX, c = idx % TX, kx = kx0 + c;
            C acc = C{0, 0};
            if (kx < d.Wx) {
                for (int i = 0; i < sc.s; ++i) {
                    const C r = rho[(size_t)i * col + idx];
                    if (alpha < 4) {
                        T g = spec_at(spec, d, i, alpha == 3 ? 1 : 0, kx, ky, kz);
                        if (alpha == 0) g *= (T)sc.c0[i];
                        if (alpha == 1) g *= (T)sc.c1[i];
                        acc.x += g * r.x;
                        acc.y += g * r.y;
                    } else {
                        const int comp = (alpha - 4) % 3;
                        T sv = spec_at(spec, d, i, 2 + comp, kx, ky, kz);
                        if (alpha < 7) sv *= (T)sc.c1[i];
                        // conj(K) = +i S:  (i S)(a + ib) = (-S b, S a)
                        acc.x -= sv * r.y;
                        acc.y += sv * r.x;
                    }
                }
            }
            work[idx] = acc;
        }
        __syncthreads();
        C *r = fft_lines<true>(work, scr, TX, ax, tw);
        C *dst = B10 + (size_t)alpha * d.nz * d.Ly * d.Wx + (size_t)ky * d.Wx;
        for (int idx = threadIdx.x; idx < TX * d.nz; idx += blockDim.x) {
            const int j = idx / TX, c = idx % TX, kx = kx0 + c;
            if (kx < d.Wx) dst[(size_t)j * d.Ly * d.Wx + kx] = r[idx];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 5: for P pairs of y-lines in plane z: inverse x-FFT of the ten n_alpha,
// dPhi/dn_alpha (FP64) inside the domain (zero outside), forward x-FFT of the
// ten Psi_alpha, in place in A.  grid (ceil(npairs/P), nz).
template <typename T>
__global__ void k_xfused(typename vec2<T>::type *__restrict__ A, Dims d, FftAxis ax,
                         const typename vec2<T>::type *__restrict__ tw, int *__restrict__ flag, int P) {
    using C = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int line = P * d.Lx;
    C *fld = reinterpret_cast<C *>(smem_raw);   // 10 fields
    C *scr = fld + (size_t)kNumWeighted * line;
    const int z = blockIdx.y, pair0 = blockIdx.x * P;
    const size_t fstride = (size_t)d.nz * d.ny * d.Wx;
    C *base = A + (size_t)z * d.ny * d.Wx;
    for (int alpha = 0; alpha < kNumWeighted; ++alpha) {
        C *buf = fld + (size_t)alpha * line;
        const C *src = base + alpha * fstride;
        for (int idx = threadIdx.x; idx < line; idx += blockDim.x) {
            const int p = idx / d.Lx, k = idx % d.Lx;
            const int y0 = 2 * (pair0 + p);
            C Z = C{0, 0};
            if (y0 < d.ny) {
                const bool up = k > d.Lx / 2;
                const int kk = up ? d.Lx - k : k;
                C X = src[(size_t)y0 * d.Wx + kk];
                C Y = (y0 + 1 < d.ny) ? src[(size_t)(y0 + 1) * d.Wx + kk] : C{0, 0};
                if (up) { X.y = -X.y; Y.y = -Y.y; }
                Z = C{X.x - Y.y, X.y + Y.x};     // X + iY
            }
            buf[k * P + p] = Z;
        }
        __syncthreads();
        fft_lines_inplace<true>(buf, scr, P, ax, tw);
    }
    // pointwise derivatives; line y0 in .x, line y0+1 in .y
    int bad = 0;
    for (int idx = threadIdx.x; idx < line; idx += blockDim.x) {
        const int p = idx / d.Lx, x = idx % d.Lx;
        const int y0 = 2 * (pair0 + p);
        for (int h = 0; h < 2; ++h) {
            const int y = y0 + h;
            double n[kNumWeighted], psi[kNumWeighted];
            const bool inside = x < d.nx && y < d.ny;
            for (int a = 0; a < kNumWeighted; ++a) {
                C v = fld[(size_t)a * line + x * P + p];
                n[a] = (double)(h ? v.y : v.x);
            }
            if (inside) {
                if (!fmt_dphi(n, psi)) bad = 1;
            } else {
                for (int a = 0; a < kNumWeighted; ++a) psi[a] = 0.0;
            }
            for (int a = 0; a < kNumWeighted; ++a) {
                C &v = fld[(size_t)a * line + x * P + p];
                if (h) v.y = (T)psi[a]; else v.x = (T)psi[a];
            }
        }
    }
    if (bad) atomicOr(flag, kFlagPacking);
    __syncthreads();
    for (int alpha = 0; alpha < kNumWeighted; ++alpha) {
        C *buf = fld + (size_t)alpha * line;
        C *r = fft_lines<false>(buf, scr, P, ax, tw);
        C *dst = base + alpha * fstride;
        for (int idx = threadIdx.x; idx < P * d.Wx; idx += blockDim.x) {
            const int p = idx / d.Wx, k = idx % d.Wx;
            const int y0 = 2 * (pair0 + p);
            if (y0 >= d.ny) continue;
            C zk = r[k * P + p];
            C zm = r[((d.Lx - k) % d.Lx) * P + p];
            C X = C{(T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)};
            C Y = C{(T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x)};
            dst[(size_t)y0 * d.Wx + k] = X;
            if (y0 + 1 < d.ny) dst[(size_t)(y0 + 1) * d.Wx + k] = Y;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 7: per column: forward z-FFT of each Psi_alpha, accumulate
// mu_i = sum_alpha K_alpha,i Psi_alpha, inverse z-FFT, rows z < nz.
template <typename T>
__global__ void k_zback(const typename vec2<T>::type *__restrict__ B10, typename vec2<T>::type *__restrict__ Bs,
                        Dims d, FftAxis ax, const typename vec2<T>::type *__restrict__ tw, const T *__restrict__ spec,
                        SpeciesConst sc, int TX) {
    using C = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int col = TX * d.Lz;
    C *acc = reinterpret_cast<C *>(smem_raw);   // s accumulators
    C *work = acc + (size_t)sc.s * col;
    C *scr = work + col;
    const int ky = blockIdx.y, kx0 = blockIdx.x * TX;
    for (int idx = threadIdx.x; idx < sc.s * col; idx += blockDim.x) acc[idx] = C{0, 0};
    for (int alpha = 0; alpha < kNumWeighted; ++alpha) {
        const C *src = B10 + (size_t)alpha * d.nz * d.Ly * d.Wx + (size_t)ky * d.Wx;
        for (int idx = threadIdx.x; idx < col; idx += blockDim.x) {
            const int j = idx / TX, c = idx % TX, kx = kx0 + c;
            C v = C{0, 0};
            if (j < d.nz && kx < d.Wx) v = src[(size_t)j * d.Ly * d.Wx + kx];
            work[idx] = v;
        }
        __syncthreads();
        C *r = fft_lines<false>(work, scr, TX, ax, tw);
        for (int idx = threadIdx.x; idx < col; idx += blockDim.x) {
            const int kz = idx / TX, c = idx % TX, kx = kx0 + c;
            if (kx >= d.Wx) continue;
            const C v = r[idx];
            for (int i = 0; i < sc.s; ++i) {
                C &o = acc[(size_t)i * col + idx];
                if (alpha < 4) {
                    T g = spec_at(spec, d, i, alpha == 3 ? 1 : 0, kx, ky, kz);
                    if (alpha == 0) g *= (T)sc.c0[i];
                    if (alpha == 1) g *= (T)sc.c1[i];
                    o.x += g * v.x;
                    o.y += g * v.y;
                } else {
                    const int comp = (alpha - 4) % 3;
                    T sv = spec_at(spec, d, i, 2 + comp, kx, ky, kz);
                    if (alpha < 7) sv *= (T)sc.c1[i];
                    // K = -i S:  (-i S)(a + ib) = (S b, -S a)
                    o.x += sv * v.y;
                    o.y -= sv * v.x;
                }
            }
        }
        __syncthreads();
    }
    for (int i = 0; i < sc.s; ++i) {
        C *r = fft_lines<true>(acc + (size_t)i * col, work, TX, ax, tw);
        C *dst = Bs + (size_t)i * d.nz * d.Ly * d.Wx + (size_t)ky * d.Wx;
        for (int idx = threadIdx.x; idx < TX * d.nz; idx += blockDim.x) {
            const int j = idx / TX, c = idx % TX, kx = kx0 + c;
            if (kx < d.Wx) dst[(size_t)j * d.Ly * d.Wx + kx] = r[idx];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 9: inverse x-FFT of F half-spectrum fields, write real values x < nx as
// FP64, optionally adding coef_f * U.  grid (ceil(npairs/P), nz, F).
template <typename T>
__global__ void k_xinv(const typename vec2<T>::type *__restrict__ A, double *__restrict__ out, size_t out_fstride,
                       Dims d, FftAxis ax, const typename vec2<T>::type *__restrict__ tw,
                       const double *__restrict__ U, SpeciesConst sc, int P) {
    using C = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + (size_t)P * d.Lx;
    const int z = blockIdx.y, f = blockIdx.z, pair0 = blockIdx.x * P;
    const C *src = A + ((size_t)f * d.nz + z) * d.ny * d.Wx;
    for (int idx = threadIdx.x; idx < P * d.Lx; idx += blockDim.x) {
        const int p = idx / d.Lx, k = idx % d.Lx;
        const int y0 = 2 * (pair0 + p);
        C Z = C{0, 0};
        if (y0 < d.ny) {
            const bool up = k > d.Lx / 2;
            const int kk = up ? d.Lx - k : k;
            C X = src[(size_t)y0 * d.Wx + kk];
            C Y = (y0 + 1 < d.ny) ? src[(size_t)(y0 + 1) * d.Wx + kk] : C{0, 0};
            if (up) { X.y = -X.y; Y.y = -Y.y; }
            Z = C{X.x - Y.y, X.y + Y.x};
        }
        a[k * P + p] = Z;
    }
    __syncthreads();
    C *r = fft_lines<true>(a, b, P, ax, tw);
    double *dst = out + f * out_fstride + (size_t)z * d.ny * d.nx;
    const double coef = U ? sc.sh[f] : 0.0;
    for (int idx = threadIdx.x; idx < P * d.nx; idx += blockDim.x) {
        const int p = idx / d.nx, x = idx % d.nx;
        const int y0 = 2 * (pair0 + p);
        if (y0 >= d.ny) continue;
        C v = r[x * P + p];
        double u0 = 0, u1 = 0;
        if (U) {
            u0 = coef * U[((size_t)z * d.ny + y0) * d.nx + x];
            if (y0 + 1 < d.ny) u1 = coef * U[((size_t)z * d.ny + y0 + 1) * d.nx + x];
        }
        dst[(size_t)y0 * d.nx + x] = (double)v.x + u0;
        if (y0 + 1 < d.ny) dst[(size_t)(y0 + 1) * d.nx + x] = (double)v.y + u1;
    }
}

// ---------------------------------------------------------------------------
// square-well set-up: one field, forward z-FFT, multiply by the real even
// spectrum of the shell stencil, inverse, rows z < nz.  grid (ceil(Wx/TX), Ly).
__global__ void k_zconv(const double2 *__restrict__ Bin, double2 *__restrict__ Bout, Dims d, FftAxis ax,
                        const double2 *__restrict__ tw, const double *__restrict__ spec, int TX) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int col = TX * d.Lz;
    double2 *work = reinterpret_cast<double2 *>(smem_raw);
    double2 *scr = work + col;
    const int ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const double2 *src = Bin + (size_t)ky * d.Wx;
    for (int idx = threadIdx.x; idx < col; idx += blockDim.x) {
        const int j = idx / TX, c = idx % TX, kx = kx0 + c;
        double2 v = {0, 0};
        if (j < d.nz && kx < d.Wx) v = src[(size_t)j * d.Ly * d.Wx + kx];
        work[idx] = v;
    }
    __syncthreads();
    fft_lines_inplace<false>(work, scr, TX, ax, tw);
    for (int idx = threadIdx.x; idx < col; idx += blockDim.x) {
        const int kz = idx / TX, c = idx % TX, kx = kx0 + c;
        if (kx >= d.Wx) continue;
        const int fy = ky <= d.Ly / 2 ? ky : d.Ly - ky;
        const int fz = kz <= d.Lz / 2 ? kz : d.Lz - kz;
        const double g = spec[((size_t)fz * d.Oy + fy) * d.Ox + kx];
        work[idx].x *= g;
        work[idx].y *= g;
    }
    __syncthreads();
    double2 *r = fft_lines<true>(work, scr, TX, ax, tw);
    double2 *dst = Bout + (size_t)ky * d.Wx;
    for (int idx = threadIdx.x; idx < TX * d.nz; idx += blockDim.x) {
        const int j = idx / TX, c = idx % TX, kx = kx0 + c;
        if (kx < d.Wx) dst[(size_t)j * d.Ly * d.Wx + kx] = r[idx];
    }
}

// Normalised Gaussian site density of Sec 2.3.2 at the grid nodes.  Terms with
// alpha d^2 > 60 (below 1e-26 of the peak) are dropped; periodic axes add the
// images of each site.
__global__ void k_site_density(double *__restrict__ rho_s, Dims d, const double *__restrict__ sites, int nsites,
                               double alpha, int px, int py, int pz, int mx, int my, int mz) {
    const size_t N = (size_t)d.nx * d.ny * d.nz;
    const double cut = 60.0 / alpha;
    const double norm = pow(alpha / M_PI, 1.5);
    for (size_t pt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; pt < N; pt += (size_t)gridDim.x * blockDim.x) {
        const double x = (double)(pt % d.nx), y = (double)((pt / d.nx) % d.ny), z = (double)(pt / ((size_t)d.nx * d.ny));
        double acc = 0.0;
        for (int k = 0; k < nsites; ++k) {
            const double sx = sites[3 * k], sy = sites[3 * k + 1], sz = sites[3 * k + 2];
            for (int iz = -mz; iz <= mz; ++iz) {
                const double dz = z - sz - iz * (double)d.nz;
                if (dz * dz > cut) continue;
                for (int iy = -my; iy <= my; ++iy) {
                    const double dy = y - sy - iy * (double)d.ny;
                    if (dy * dy + dz * dz > cut) continue;
                    for (int ix = -mx; ix <= mx; ++ix) {
                        const double dx = x - sx - ix * (double)d.nx;
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 <= cut) acc += exp(-alpha * r2);
                    }
                }
            }
        }
        rho_s[pt] = norm * acc;
    }
    (void)px; (void)py; (void)pz;
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
// host side
static int pick_pow2(long limit, int cap) {
    int v = 1;
    while (v * 2 <= cap && v * 2 <= limit) v *= 2;
    return v;
}

struct Launch {
    int P_x, P_fused, TX_y, TX_z;
    size_t sm_x, sm_fused, sm_y, sm_zmac, sm_zback, sm_zconv;
};

static Launch launch_shape(const Problem *p, int prec) {
    const Dims d = make_dims(p);
    const size_t cs = prec == PNP_PREC_FP64 ? 16 : 8;
    const long budget = 96 * 1024;
    Launch l;
    l.P_x = pick_pow2(std::min<long>(48 * 1024 / (2 * cs * d.Lx), d.npairs), 16);
    l.P_fused = pick_pow2(std::min<long>(budget / ((kNumWeighted + 1) * cs * d.Lx), d.npairs), 8);
    l.TX_y = pick_pow2(std::min<long>(48 * 1024 / (2 * cs * d.Ly), d.Wx), 16);
    l.TX_z = pick_pow2(std::min<long>(budget / ((p->s + 2) * cs * d.Lz), d.Wx), 16);
    l.sm_x = 2 * cs * l.P_x * d.Lx;
    l.sm_fused = (kNumWeighted + 1) * cs * l.P_fused * d.Lx;
    l.sm_y = 2 * cs * l.TX_y * d.Ly;
    l.sm_zmac = (p->s + 2) * cs * l.TX_z * d.Lz;
    l.sm_zback = (p->s + 2) * cs * l.TX_z * d.Lz;
    l.sm_zconv = 2 * 16 * l.TX_z * d.Lz;
    return l;
}

template <typename T> static int set_smem_attrs() {
    static bool done = false;
    if (done) return PNP_OK;
    const int big = 200 * 1024;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaFuncSetAttribute(k_xfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_ypass<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_ypass<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_zmac<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_xfused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_zback<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_xinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_zconv, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e != cudaSuccess) return cuda_status(e);
    done = true;
    return PNP_OK;
}

static size_t workspace_bytes(const Problem *p) {
    const Dims d = make_dims(p);
    const size_t wx = d.Wx, cs = 16;
    size_t A = (size_t)kNumWeighted * d.nz * d.ny * wx;
    size_t B10 = (size_t)kNumWeighted * d.nz * d.Ly * wx;
    size_t Bs = (size_t)p->s * d.nz * d.Ly * wx;
    return cs * (A + B10 + Bs) + 3 * 256;
}

struct Work {
    void *A, *B10, *Bs;
};

static Work carve(const Problem *p, int prec) {
    const Dims d = make_dims(p);
    const size_t cs = prec == PNP_PREC_FP64 ? 16 : 8;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char *base = (char *)p->d_work;
    size_t A = cs * kNumWeighted * d.nz * d.ny * d.Wx;
    size_t B10 = cs * kNumWeighted * d.nz * d.Ly * d.Wx;
    Work w;
    w.A = base;
    w.B10 = base + up(A);
    w.Bs = base + up(A) + up(B10);
    return w;
}

// Padded lengths with a register-resident two-factor FFT (fft_reg.cuh);
// every other length uses the shared-memory Stockham kernels.
template <typename F> static bool with_shape(int L, F &&f) {
    using std::integral_constant;
    switch (L) {
        case 32: f(integral_constant<int, 8>{}, integral_constant<int, 4>{}); return true;
        case 40: f(integral_constant<int, 8>{}, integral_constant<int, 5>{}); return true;
        case 64: f(integral_constant<int, 8>{}, integral_constant<int, 8>{}); return true;
        case 128: f(integral_constant<int, 16>{}, integral_constant<int, 8>{}); return true;
        case 256: f(integral_constant<int, 16>{}, integral_constant<int, 16>{}); return true;
        default: return false;
    }
}

template <auto K> static void ensure_smem() {
    static const bool done = [] {
        cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return true;
    }();
    (void)done;
}

template <typename T>
static int run_pipeline(Problem *p, DeviceBuffers *db, const double *d_rho, double *d_mu, cudaStream_t st) {
    using C = typename vec2<T>::type;
    const int prec = sizeof(T) == 8 ? PNP_PREC_FP64 : PNP_PREC_FP32;
    int rc = set_smem_attrs<T>();
    if (rc) return rc;
    const Dims d = make_dims(p);
    const Launch l = launch_shape(p, prec);
    const SpeciesConst sc = make_sc(p);
    Work w = carve(p, prec);
    C *A = (C *)w.A, *B10 = (C *)w.B10, *Bs = (C *)w.Bs;
    const C *twx = (const C *)db->tw[0], *twy = (const C *)db->tw[1], *twz = (const C *)db->tw[2];
    const T *spec = (const T *)db->spec;
    const int s = p->s;
    const size_t N = p->npts();
    const int T256 = 256;
    StageTimer &tm = p->timer;
    const size_t cs = sizeof(C);
    const long kBudget = 96 * 1024;
    auto pow2_le = [](long v) { long r = 1; while (r * 2 <= v) r *= 2; return (int)r; };

    // 1: x forward
    tm.begin(0, st);
    if (!with_shape(d.Lx, [&](auto a, auto b) {
            constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
            const int P = std::max(1, std::min(256 / G, d.npairs));
            ensure_smem<k_xfwd_r<T, N1, N2>>();
            dim3 g((d.npairs + P - 1) / P, d.nz, s);
            k_xfwd_r<T, N1, N2><<<g, P * G, P * Shape<N1, N2>::EX * cs, st>>>(d_rho, N, A, d, twx, P);
        })) {
        dim3 gx((d.npairs + l.P_x - 1) / l.P_x, d.nz, s);
        k_xfwd<T><<<gx, T256, l.sm_x, st>>>(d_rho, N, A, d, p->ax[0], twx, l.P_x);
    }
    tm.end(st);

    // y passes: forward (rows ny -> Ly) or inverse (Ly -> ny) of F fields
    auto ypass = [&](int stage, bool inv, const C *in, C *out, int F) {
        tm.begin(stage, st);
        const int rows_in = inv ? d.Ly : d.ny, rows_out = inv ? d.ny : d.Ly;
        if (!with_shape(d.Ly, [&](auto a, auto b) {
                constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
                const int TX = pow2_le(std::min<long>(256 / G, 16));
                dim3 g((d.Wx + TX - 1) / TX, d.nz, F);
                const size_t sm = (size_t)TX * Shape<N1, N2>::EX * cs;
                if (inv) {
                    ensure_smem<k_ypass_r<T, true, N1, N2>>();
                    k_ypass_r<T, true, N1, N2><<<g, TX * G, sm, st>>>(in, out, d, rows_in, rows_in, rows_out,
                                                                     rows_out, twy, TX);
                } else {
                    ensure_smem<k_ypass_r<T, false, N1, N2>>();
                    k_ypass_r<T, false, N1, N2><<<g, TX * G, sm, st>>>(in, out, d, rows_in, rows_in, rows_out,
                                                                      rows_out, twy, TX);
                }
            })) {
            dim3 g((d.Wx + l.TX_y - 1) / l.TX_y, d.nz, F);
            if (inv)
                k_ypass<T, true><<<g, T256, l.sm_y, st>>>(in, out, d, rows_in, rows_in, rows_out, rows_out,
                                                         p->ax[1], twy, l.TX_y);
            else
                k_ypass<T, false><<<g, T256, l.sm_y, st>>>(in, out, d, rows_in, rows_in, rows_out, rows_out,
                                                          p->ax[1], twy, l.TX_y);
        }
        tm.end(st);
    };

    // z column kernels (MAC forward / back)
    auto zpass = [&](int stage, bool back) {
        tm.begin(stage, st);
        if (!with_shape(d.Lz, [&](auto a, auto b) {
                constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
                // paired columns (ky, Ly - ky): 2 TX columns per CTA
                const long per_col = ((long)s * N1 * G + Shape<N1, N2>::EX) * (long)cs;
                const int TX = pow2_le(std::max<long>(1, std::min<long>(std::min<long>(128 / G, 8), kBudget / (2 * per_col))));
                dim3 g((d.Wx + TX - 1) / TX, d.Ly / 2 + 1);
                if (back) {
                    ensure_smem<k_zback_p<T, N1, N2>>();
                    k_zback_p<T, N1, N2><<<g, 2 * TX * G, 2 * TX * per_col, st>>>(B10, Bs, d, twz, spec, sc, TX);
                } else {
                    ensure_smem<k_zmac_p<T, N1, N2>>();
                    k_zmac_p<T, N1, N2><<<g, 2 * TX * G, 2 * TX * per_col, st>>>(Bs, B10, d, twz, spec, sc, TX);
                }
            })) {
            dim3 gz((d.Wx + l.TX_z - 1) / l.TX_z, d.Ly);
            if (back)
                k_zback<T><<<gz, T256, l.sm_zback, st>>>(B10, Bs, d, p->ax[2], twz, spec, sc, l.TX_z);
            else
                k_zmac<T><<<gz, T256, l.sm_zmac, st>>>(Bs, B10, d, p->ax[2], twz, spec, sc, l.TX_z);
        }
        tm.end(st);
    };

    ypass(1, false, A, Bs, s);
    zpass(2, false);
    ypass(3, true, B10, A, kNumWeighted);

    // 5: x fused inverse -> dPhi/dn -> forward
    tm.begin(4, st);
    if (!with_shape(d.Lx, [&](auto a, auto b) {
            constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
            const int NQ = std::min(N2, (d.nx + N1 - 1) / N1);
            const long per_pair = ((long)kNumWeighted * NQ * N1 + Shape<N1, N2>::EX) * (long)cs;
            const int P = (int)std::max<long>(1, std::min<long>(std::min<long>(256 / G, d.npairs), kBudget / per_pair));
            ensure_smem<k_xfused_r<T, N1, N2>>();
            dim3 g((d.npairs + P - 1) / P, d.nz);
            k_xfused_r<T, N1, N2><<<g, P * G, P * per_pair, st>>>(A, d, twx, p->d_flag, P, NQ);
        })) {
        dim3 gf((d.npairs + l.P_fused - 1) / l.P_fused, d.nz);
        k_xfused<T><<<gf, T256, l.sm_fused, st>>>(A, d, p->ax[0], twx, p->d_flag, l.P_fused);
    }
    tm.end(st);

    ypass(5, false, A, B10, kNumWeighted);
    zpass(6, true);
    ypass(7, true, Bs, A, s);

    // 9: x inverse + mu_sh
    tm.begin(8, st);
    const double *U = p->has_wells ? p->d_U : nullptr;
    if (!with_shape(d.Lx, [&](auto a, auto b) {
            constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
            const int P = std::max(1, std::min(256 / G, d.npairs));
            ensure_smem<k_xinv_r<T, N1, N2>>();
            dim3 g((d.npairs + P - 1) / P, d.nz, s);
            k_xinv_r<T, N1, N2><<<g, P * G, P * Shape<N1, N2>::EX * cs, st>>>(A, d_mu, N, d, twx, U, sc, P);
        })) {
        dim3 gx((d.npairs + l.P_x - 1) / l.P_x, d.nz, s);
        k_xinv<T><<<gx, T256, l.sm_x, st>>>(A, d_mu, N, d, p->ax[0], twx, U, sc, l.P_x);
    }
    tm.end(st);
    return cuda_status(cudaGetLastError());
}

static int upload_twiddles(const Problem *p, DeviceBuffers *db, int prec) {
    for (int c = 0; c < 3; ++c) {
        const int L = p->L[c];
        std::vector<double> h(2 * (size_t)L);
        for (int m = 0; m < L; ++m) {
            double ang = -2.0 * M_PI * (double)m / L;
            h[2 * m] = std::cos(ang);
            h[2 * m + 1] = std::sin(ang);
        }
        // exact values at the quarter points
        for (int m = 0; m < L; ++m) {
            if ((4 * (long)m) % L == 0) {
                int q = (int)((4 * (long)m) / L);
                const double cs[4][2] = {{1, 0}, {0, -1}, {-1, 0}, {0, 1}};
                h[2 * m] = cs[q][0];
                h[2 * m + 1] = cs[q][1];
            }
        }
        size_t bytes = (prec == PNP_PREC_FP64 ? 16 : 8) * (size_t)L;
        cudaError_t e = dmalloc(&db->tw[c], bytes, p->stream);
        if (e != cudaSuccess) return PNP_ERR_NOMEM;
        db->bytes += bytes;
        if (prec == PNP_PREC_FP64) {
            e = cudaMemcpy(db->tw[c], h.data(), bytes, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> f(h.begin(), h.end());
            e = cudaMemcpy(db->tw[c], f.data(), bytes, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    return PNP_OK;
}

static void free_buffers(DeviceBuffers *db, cudaStream_t st) {
    if (!db) return;
    for (int c = 0; c < 3; ++c) dfree(db->tw[c], st);
    dfree(db->spec, st);
    delete db;
}

// FP64 spectra of every species' kernels, built on the host.
static int build_fp64(Problem *p) {
    DeviceBuffers *db = new DeviceBuffers();
    db->prec = PNP_PREC_FP64;
    p->buf[0] = db;
    int rc = upload_twiddles(p, db, PNP_PREC_FP64);
    if (rc) return rc;
    const Dims d = make_dims(p);
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    const size_t bytes = sizeof(double) * oct * kNumKernels * p->s;
    if (dmalloc(&db->spec, bytes, p->stream) != cudaSuccess) return PNP_ERR_NOMEM;
    db->bytes += bytes;
    const double scale = 1.0 / ((double)d.Lx * d.Ly * d.Lz);
    const bool odd[kNumKernels][3] = {{false, false, false}, {false, false, false}, {true, false, false},
                                      {false, true, false}, {false, false, true}};
    std::vector<double> h(oct);
    for (int i = 0; i < p->s; ++i) {
        Stencil st[kNumKernels];
        build_fmt_stencils(p->R[i], p->quad[0], p->quad[1], p->quad[2], p->S, st);
        for (int k = 0; k < kNumKernels; ++k) {
            octant_transform(st[k], p->L, odd[k], scale, h.data());
            cudaError_t e = cudaMemcpy((double *)db->spec + (size_t)(i * kNumKernels + k) * oct, h.data(),
                                       sizeof(double) * oct, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    p->device_bytes += db->bytes;
    return PNP_OK;
}

int mu_ex_prepare(Problem *p, int prec) {
    if (prec == PNP_PREC_FP64) return p->buf[0] ? PNP_OK : build_fp64(p);
    if (p->buf[1]) return PNP_OK;
    int rc = mu_ex_prepare(p, PNP_PREC_FP64);
    if (rc) return rc;
    DeviceBuffers *db = new DeviceBuffers();
    db->prec = PNP_PREC_FP32;
    p->buf[1] = db;
    rc = upload_twiddles(p, db, PNP_PREC_FP32);
    if (rc) return rc;
    const Dims d = make_dims(p);
    const size_t n = (size_t)d.Ox * d.Oy * d.Oz * kNumKernels * p->s;
    if (dmalloc(&db->spec, sizeof(float) * n, p->stream) != cudaSuccess) return PNP_ERR_NOMEM;
    db->bytes += sizeof(float) * n;
    k_to_float<<<1024, 256, 0, p->stream>>>((const double *)p->buf[0]->spec, (float *)db->spec, n);
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    p->device_bytes += db->bytes;
    return PNP_OK;
}

// Workspace, FP64 spectra and the square-well field U = K_sw (x) rho_s.
int mu_ex_setup(Problem *p) {
    p->work_bytes = workspace_bytes(p);
    if (dmalloc(&p->d_work, p->work_bytes, p->stream) != cudaSuccess) return PNP_ERR_NOMEM;
    p->device_bytes += p->work_bytes;
    int rc = build_fp64(p);
    if (rc) return rc;
    if (!p->has_wells) return PNP_OK;

    const Dims d = make_dims(p);
    const size_t N = p->npts();
    p->sh_coef.assign(p->s, 0.0);
    for (int i = 0; i < p->s; ++i) p->sh_coef[i] = (p->sw_half ? 0.5 : 1.0) * (-p->depth[i]);
    if (dmalloc((void **)&p->d_U, sizeof(double) * N, p->stream) != cudaSuccess) return PNP_ERR_NOMEM;
    p->device_bytes += sizeof(double) * N;
    // site density into the FP64 staging area of the workspace end
    double *d_sites = nullptr, *d_rs = nullptr, *d_spec = nullptr;
    cudaError_t e = dmalloc((void **)&d_sites, sizeof(double) * std::max<size_t>(3, p->sites.size()), p->stream);
    if (e == cudaSuccess) e = dmalloc((void **)&d_rs, sizeof(double) * N, p->stream);
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    if (e == cudaSuccess) e = dmalloc((void **)&d_spec, sizeof(double) * oct, p->stream);
    if (e != cudaSuccess) {
        dfree(d_sites, p->stream); dfree(d_rs, p->stream); dfree(d_spec, p->stream);
        return PNP_ERR_NOMEM;
    }
    e = cudaMemcpy(d_sites, p->sites.data(), sizeof(double) * p->sites.size(), cudaMemcpyHostToDevice);
    {
        const double reach = std::sqrt(60.0 / p->site_alpha);
        int m[3];
        const int n[3] = {p->nx, p->ny, p->nz};
        for (int c = 0; c < 3; ++c) m[c] = p->bc[c] == PNP_BC_PERIODIC ? (int)std::ceil(reach / n[c]) + 1 : 0;
        k_site_density<<<1024, 256, 0, p->stream>>>(d_rs, d, d_sites, (int)(p->sites.size() / 3), p->site_alpha,
                                                    0, 0, 0, m[0], m[1], m[2]);
    }
    Stencil sw;
    build_well_stencil(p->well_inner, p->well_outer, p->wquad[0], p->wquad[1], p->wquad[2], p->Ssw, sw);
    std::vector<double> h(oct);
    const bool even[3] = {false, false, false};
    octant_transform(sw, p->L, even, 1.0 / ((double)d.Lx * d.Ly * d.Lz), h.data());
    if (e == cudaSuccess) e = cudaMemcpy(d_spec, h.data(), sizeof(double) * oct, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        rc = set_smem_attrs<double>();
        const Launch l = launch_shape(p, PNP_PREC_FP64);
        Work w = carve(p, PNP_PREC_FP64);
        DeviceBuffers *db = p->buf[0];
        double2 *A = (double2 *)w.A, *B = (double2 *)w.B10, *B2 = (double2 *)w.Bs;
        SpeciesConst one{};
        one.s = 1;
        dim3 gx((d.npairs + l.P_x - 1) / l.P_x, d.nz, 1);
        k_xfwd<double><<<gx, 256, l.sm_x, p->stream>>>(d_rs, N, A, d, p->ax[0], (const double2 *)db->tw[0], l.P_x);
        dim3 gy((d.Wx + l.TX_y - 1) / l.TX_y, d.nz, 1);
        k_ypass<double, false><<<gy, 256, l.sm_y, p->stream>>>(A, B, d, d.ny, d.ny, d.Ly, d.Ly, p->ax[1],
                                                               (const double2 *)db->tw[1], l.TX_y);
        dim3 gz((d.Wx + l.TX_z - 1) / l.TX_z, d.Ly);
        k_zconv<<<gz, 256, l.sm_zconv, p->stream>>>(B, B2, d, p->ax[2], (const double2 *)db->tw[2], d_spec, l.TX_z);
        k_ypass<double, true><<<gy, 256, l.sm_y, p->stream>>>(B2, A, d, d.Ly, d.Ly, d.ny, d.ny, p->ax[1],
                                                              (const double2 *)db->tw[1], l.TX_y);
        k_xinv<double><<<gx, 256, l.sm_x, p->stream>>>(A, p->d_U, N, d, p->ax[0], (const double2 *)db->tw[0],
                                                       nullptr, one, l.P_x);
        e = cudaStreamSynchronize(p->stream);
    }
    dfree(d_sites, p->stream);
    dfree(d_rs, p->stream);
    dfree(d_spec, p->stream);
    if (rc) return rc;
    return cuda_status(e);
}

int mu_ex_enqueue(Problem *p, int prec, const double *d_rho, double *d_mu, cudaStream_t st) {
    int rc = mu_ex_prepare(p, prec);
    if (rc) return rc;
    if (prec == PNP_PREC_FP64) return run_pipeline<double>(p, p->buf[0], d_rho, d_mu, st);
    return run_pipeline<float>(p, p->buf[1], d_rho, d_mu, st);
}

// ---------------------------------------------------------------------------
// stage timing
cudaEvent_t StageTimer::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void StageTimer::begin(int s, cudaStream_t st) {
    if (!enabled) return;
    cudaEvent_t a = get();
    cudaEventRecord(a, st);
    stage.push_back(s);
    ev0.push_back(a);
}

void StageTimer::end(cudaStream_t st) {
    if (!enabled) return;
    cudaEvent_t b = get();
    cudaEventRecord(b, st);
    ev1.push_back(b);
}

int StageTimer::collect(double *ms, int *launches, int max) {
    const int n = std::min(max, kNumStages);
    for (int k = 0; k < n; ++k) {
        if (ms) ms[k] = 0.0;
        if (launches) launches[k] = 0;
    }
    for (size_t j = 0; j < ev1.size(); ++j) {
        cudaEventSynchronize(ev1[j]);
        float t = 0.f;
        cudaEventElapsedTime(&t, ev0[j], ev1[j]);
        const int s = stage[j];
        if (s < n) {
            if (ms) ms[s] += t;
            if (launches) launches[s] += 1;
        }
        pool.push_back(ev0[j]);
        pool.push_back(ev1[j]);
    }
    stage.clear();
    ev0.clear();
    ev1.clear();
    return kNumStages;
}

void StageTimer::release() {
    for (auto e : ev0) cudaEventDestroy(e);
    for (auto e : ev1) cudaEventDestroy(e);
    for (auto e : pool) cudaEventDestroy(e);
    ev0.clear();
    ev1.clear();
    pool.clear();
    stage.clear();
}

void mu_ex_free(Problem *p) {
    p->timer.release();
    for (int k = 0; k < 2; ++k) {
        free_buffers(p->buf[k], p->stream);
        p->buf[k] = nullptr;
    }
    dfree(p->d_work, p->stream);
    dfree(p->d_U, p->stream);
    p->d_work = nullptr;
    p->d_U = nullptr;
}

}  // namespace pnp

// ===========================================================================
// Fixed-scratch variant of the FP64 mu_ex pipeline.
//
// Some callers cannot allocate device memory once they are running: a host
// application whose GPU memory is owned by its own allocator (a framework
// whose caching allocator already holds nearly all of the device, or a
// simulation code that reserves its pool at start-up), or a latency-critical
// loop that must not call cudaMalloc/cudaFree because those calls can
// synchronise the whole device.  pnp_excess_mu_noalloc serves them: all of its
// device-side scratch -- status word, twiddle tables, kernel spectra and the
// FFT workspace -- lives in the file-scope array below, so the call performs
// no device allocation at all.  The caller passes the densities and the output
// buffer.
//
// The array is kNoAllocBytes (32 MiB) and every GPU that loads this library
// holds it until the process exits.  Its address is looked up once per device
// with cudaGetSymbolAddress on the first call made while that device is
// current; make that first call before any stream capture.  Every call shares
// the array and it keeps the previous call's contents: the status word is
// cleared by each call, everything else is fully overwritten before it is
// read.  Calls whose work overlaps on the GPU (other streams, other host
// threads) race on the array; serialise them.
namespace pnp {

constexpr size_t kNoAllocBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[64] = {nullptr};

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

// bytes of the fixed scratch a problem needs: status word, three FP64
// twiddle tables, the FP64 spectrum octants and the FP64 workspace
size_t noalloc_bytes(const Problem &p) {
    const Dims d = make_dims(&p);
    size_t b = 256;
    for (int c = 0; c < 3; ++c) b += round256(16 * (size_t)p.L[c]);
    b += round256(sizeof(double) * (size_t)d.Ox * d.Oy * d.Oz * kNumKernels * p.s);
    b += round256(workspace_bytes(&p));
    return b;
}

void twiddles_host(int L, std::vector<double> &h) {
    h.assign(2 * (size_t)L, 0.0);
    for (int m = 0; m < L; ++m) {
        if ((4 * (long)m) % L == 0) {
            const double cs[4][2] = {{1, 0}, {0, -1}, {-1, 0}, {0, 1}};
            const int q = (int)((4 * (long)m) / L);
            h[2 * m] = cs[q][0];
            h[2 * m + 1] = cs[q][1];
        } else {
            const double ang = -2.0 * M_PI * (double)m / L;
            h[2 * m] = std::cos(ang);
            h[2 * m + 1] = std::sin(ang);
        }
    }
}
}  // namespace

}  // namespace pnp

extern "C" int pnp_excess_mu_noalloc(const pnp_problem_desc *desc, const double *d_rho, double *d_mu_ex,
                                     void *stream) {
    using namespace pnp;
    if (!desc || !d_rho || !d_mu_ex) return PNP_ERR_INVALID;
    Problem p;
    std::string why;
    int rc = validate_and_copy(desc, &p, &why);
    if (rc) return rc;
    if (p.has_wells) return PNP_ERR_INVALID;        // hard-sphere part only
    if (noalloc_bytes(p) > kNoAllocBytes) return PNP_ERR_TOO_LARGE;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= 64) return PNP_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        g_noalloc_addr[dev] = ptr;
    }
    unsigned char *base = (unsigned char *)g_noalloc_addr[dev];
    cudaStream_t st = (cudaStream_t)stream;
    // carve: status word | twiddles x, y, z | spectra | workspace
    size_t off = 256;
    DeviceBuffers db;
    db.prec = PNP_PREC_FP64;
    std::vector<double> h;
    for (int c = 0; c < 3; ++c) {
        db.tw[c] = base + off;
        twiddles_host(p.L[c], h);
        e = cudaMemcpyAsync(db.tw[c], h.data(), 16 * (size_t)p.L[c], cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_status(e);
        off += round256(16 * (size_t)p.L[c]);
    }
    const Dims d = make_dims(&p);
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    db.spec = base + off;
    const double scale = 1.0 / ((double)d.Lx * d.Ly * d.Lz);
    const bool odd[kNumKernels][3] = {{false, false, false}, {false, false, false}, {true, false, false},
                                      {false, true, false}, {false, false, true}};
    h.assign(oct, 0.0);
    for (int i = 0; i < p.s; ++i) {
        Stencil stn[kNumKernels];
        build_fmt_stencils(p.R[i], p.quad[0], p.quad[1], p.quad[2], p.S, stn);
        for (int k = 0; k < kNumKernels; ++k) {
            octant_transform(stn[k], p.L, odd[k], scale, h.data());
            // synchronous copy: the host table is reused for the next kernel
            e = cudaMemcpy((double *)db.spec + (size_t)(i * kNumKernels + k) * oct, h.data(), sizeof(double) * oct,
                           cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    off += round256(sizeof(double) * oct * kNumKernels * p.s);
    p.d_work = base + off;
    p.d_flag = (int *)base;
    e = cudaMemsetAsync(p.d_flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e);
    rc = run_pipeline<double>(&p, &db, d_rho, d_mu_ex, st);
    if (rc) return rc;
    int flag = 0;
    e = cudaMemcpyAsync(&flag, p.d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    p.d_work = nullptr;
    p.d_flag = nullptr;
    return (flag & (kFlagPacking | kFlagNonFinite)) ? PNP_ERR_PACKING : PNP_OK;
}

namespace pnp {

// Device memory a problem will hold once its Gummel state exists: FFT
// workspace, spectra (FP64, plus FP32 when that is the problem's precision),
// square-well field, staging buffers and the multigrid hierarchy.
size_t estimate_device_bytes(const Problem &p) {
    const Dims d = make_dims(&p);
    const size_t N = p.npts();
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz * kNumKernels * p.s;
    size_t b = workspace_bytes(&p) + oct * sizeof(double);
    if (p.precision == PNP_PREC_FP32) b += oct * sizeof(float);
    if (p.has_wells) b += N * sizeof(double);
    b += sizeof(double) * (2 * N * p.s + N);                 // host-call staging
    b += sizeof(double) * N * 11 * 8 / 7;                    // multigrid levels
    b += sizeof(double) * N * (2 * (size_t)p.s + 7);         // solve state and CG vectors
    return b + b / 16 + (1 << 20);
}

}  // namespace pnp
