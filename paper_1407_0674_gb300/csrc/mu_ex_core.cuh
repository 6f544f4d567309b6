// Kernels and launch logic of the mu_ex pipeline, shared by the per-precision
// translation units (mu_ex_fp64.cu, mu_ex_fp32.cu, mu_ex_df64.cu) and mu_ex.cu.
//
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
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
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
    int fmt;           // hard-sphere functional: PNP_FMT_ROSENFELD or PNP_FMT_WHITE_BEAR
};

struct SpeciesConst {
    int s;
    int msa;           // 1: z-back also applies the MSA pair kernels (Sec 2.3.4)
    double c0[8];      // 1 / (4 pi R^2)
    double c1[8];      // 1 / (4 pi R)
    double sh[8];      // mu_sh coefficient
    float c0f[8], c1f[8];   // the same, pre-rounded for FP32 kernels
    float c0h[8], c0l[8], c1h[8], c1l[8];   // and split for double-float kernels
};

template <typename T> __device__ __forceinline__ T sc_c0(const SpeciesConst &sc, int i);
template <> __device__ __forceinline__ double sc_c0<double>(const SpeciesConst &sc, int i) { return sc.c0[i]; }
template <> __device__ __forceinline__ float sc_c0<float>(const SpeciesConst &sc, int i) { return sc.c0f[i]; }
template <> __device__ __forceinline__ dd sc_c0<dd>(const SpeciesConst &sc, int i) { return dd(sc.c0h[i], sc.c0l[i]); }
template <typename T> __device__ __forceinline__ T sc_c1(const SpeciesConst &sc, int i);
template <> __device__ __forceinline__ double sc_c1<double>(const SpeciesConst &sc, int i) { return sc.c1[i]; }
template <> __device__ __forceinline__ float sc_c1<float>(const SpeciesConst &sc, int i) { return sc.c1f[i]; }
template <> __device__ __forceinline__ dd sc_c1<dd>(const SpeciesConst &sc, int i) { return dd(sc.c1h[i], sc.c1l[i]); }

struct DeviceBuffers {
    int prec = 0;
    void *tw[3] = {nullptr, nullptr, nullptr};
    void *spec = nullptr;      // [s][5][Oz][Oy][Ox]
    float *tc_b = nullptr;     // split 16-point DFT matrices of the tensor-core y pass
    size_t bytes = 0;
};

static Dims make_dims(const Problem *p) {
    Dims d;
    d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
    d.Lx = p->L[0]; d.Ly = p->L[1]; d.Lz = p->L[2];
    d.Wx = d.Lx / 2 + 1;
    d.Ox = d.Lx / 2 + 1; d.Oy = d.Ly / 2 + 1; d.Oz = d.Lz / 2 + 1;
    d.npairs = (d.ny + 1) / 2;
    d.fmt = p->fmt;
    return d;
}

// kernels whose octant spectra a problem stores: five FMT weights per
// species, then the MSA pair kernels (packed upper triangle, negated)
static int spec_kernels(const Problem *p) {
    return kNumKernels * p->s + (p->msa ? p->s * (p->s + 1) / 2 : 0);
}

static SpeciesConst make_sc(const Problem *p) {
    SpeciesConst sc{};
    sc.s = p->s;
    sc.msa = p->msa ? 1 : 0;
    for (int i = 0; i < p->s; ++i) {
        sc.c0[i] = 1.0 / (4.0 * M_PI * p->R[i] * p->R[i]);
        sc.c1[i] = 1.0 / (4.0 * M_PI * p->R[i]);
        sc.sh[i] = p->has_wells ? p->sh_coef[i] : 0.0;
        sc.c0f[i] = (float)sc.c0[i];
        sc.c1f[i] = (float)sc.c1[i];
        const dd a(sc.c0[i]), b(sc.c1[i]);
        sc.c0h[i] = a.hi; sc.c0l[i] = a.lo;
        sc.c1h[i] = b.hi; sc.c1l[i] = b.lo;
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
    T v = ldgt(&sp[(size_t)(i * kNumKernels + type) * oct + ((size_t)fz * d.Oy + fy) * d.Ox + kx]);
    if (type == 3 && ky > d.Ly / 2) v = -v;
    if (type == 4 && kz > d.Lz / 2) v = -v;
    return v;
}

// Rosenfeld FMT derivatives of Sec 2.3.1, FP64.
// White Bear n3 function phi3(x) = [x + (1-x)^2 ln(1-x)] / [x^2 (1-x)^2] and
// its derivative.  Near x = 0 the closed form cancels (and x is exactly 0
// off the domain), so |x| < 0.05 sums the power series
// phi3 = sum_k (k+1)(k+3)/(k+2) x^k to x^24.
__device__ __forceinline__ void wb_phi3(double x, double &f, double &df) {
    if (fabs(x) < 0.05) {
        double v = 0.0, d = 0.0;
#pragma unroll
        for (int k = 24; k >= 1; --k) {
            const double c = (double)((k + 1) * (k + 3)) / (double)(k + 2);
            v = v * x + c;
            d = d * x + k * c;
        }
        f = v * x + 1.5;
        df = d;
        return;
    }
    const double o = 1.0 - x, L = log(o);
    f = (x + o * o * L) / (x * x * o * o);
    df = (x - 2.0 * o * L) / (x * x * o * o) - 2.0 * (1.0 - 2.0 * x) * f / (x * o);
}

// dPhi/dn_alpha of Rosenfeld's functional (Sec 2.3.1) or of the White Bear
// form (fmt 1: the n2^3 term carries phi3(n3) / 36 pi instead of
// 1 / (24 pi (1 - n3)^2)); false at a packing violation.
__device__ __forceinline__ bool fmt_dphi(const double n[kNumWeighted], double psi[kNumWeighted], int fmt = 0) {
    const double n0 = n[0], n1 = n[1], n2 = n[2], n3 = n[3];
    const double g = 1.0 / (1.0 - n3);
    const double g2 = g * g;
    const double v1v2 = n[4] * n[7] + n[5] * n[8] + n[6] * n[9];
    const double v2v2 = n[7] * n[7] + n[8] * n[8] + n[9] * n[9];
    psi[0] = -log1p(-n3);
    psi[1] = n2 * g;
    if (fmt == PNP_FMT_WHITE_BEAR) {
        double f = 0.0, df = 0.0;
        if (n3 < 1.0) wb_phi3(n3, f, df);
        psi[2] = n1 * g + (n2 * n2 - v2v2) * f * (1.0 / (12.0 * M_PI));
        psi[3] = n0 * g + (n1 * n2 - v1v2) * g2 + (n2 * n2 * n2 - 3.0 * n2 * v2v2) * df * (1.0 / (36.0 * M_PI));
        for (int c = 0; c < 3; ++c) {
            psi[4 + c] = -n[7 + c] * g;
            psi[7 + c] = -n[4 + c] * g - n2 * n[7 + c] * f * (1.0 / (6.0 * M_PI));
        }
    } else {
        psi[2] = n1 * g + (n2 * n2 - v2v2) * g2 * (1.0 / (8.0 * M_PI));
        psi[3] = n0 * g + (n1 * n2 - v1v2) * g2 + (n2 * n2 * n2 - 3.0 * n2 * v2v2) * g2 * g * (1.0 / (12.0 * M_PI));
        for (int c = 0; c < 3; ++c) {
            psi[4 + c] = -n[7 + c] * g;
            psi[7 + c] = -n[4 + c] * g - n2 * n[7 + c] * g2 * (1.0 / (4.0 * M_PI));
        }
    }
    bool ok = n3 < 1.0;
    for (int a = 0; a < kNumWeighted; ++a) ok = ok && isfinite(psi[a]);
    return ok;
}

// Rosenfeld dPhi/dn (FP64) in place on ten real fields [10][N] of type V:
// n_alpha in, Psi_alpha out.
template <typename V>
__global__ void k_dphi_fields(V *__restrict__ f, size_t N, int *__restrict__ flag, int fmt) {
    bool bad = false;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        double n[kNumWeighted], psi[kNumWeighted];
#pragma unroll
        for (int a = 0; a < kNumWeighted; ++a) n[a] = (double)f[a * N + p];
        if (!fmt_dphi(n, psi, fmt)) bad = true;
#pragma unroll
        for (int a = 0; a < kNumWeighted; ++a) f[a * N + p] = (V)psi[a];
    }
    if (bad) atomicOr(flag, kFlagPacking);
}

// The same derivatives for FP32 fields: the functions that are singular at
// packing, ln(1 - n3) and the powers of 1/(1 - n3), in FP64; their products
// with the other weighted densities in FP32 (the fields carry FP32 rounding
// already).  Internal linkage: one copy per translation unit.
static __global__ void k_dphi_fields_mixed(float *__restrict__ f, size_t N, int *__restrict__ flag, int fmt) {
    constexpr float k8pi = (float)(1.0 / (8.0 * M_PI)), k12pi = (float)(1.0 / (12.0 * M_PI)),
                    k4pi = (float)(1.0 / (4.0 * M_PI));
    bool bad = false;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        float n[kNumWeighted], psi[kNumWeighted];
#pragma unroll
        for (int a = 0; a < kNumWeighted; ++a) n[a] = f[a * N + p];
        const double n3 = (double)n[3];
        const double gd = 1.0 / (1.0 - n3);
        // coefficient functions of n2^2 (psi2, vector psi) and n2^3 (psi3)
        float c2, c3, cv;
        if (fmt == PNP_FMT_WHITE_BEAR) {
            double fw = 0.0, dfw = 0.0;
            if (n3 < 1.0) wb_phi3(n3, fw, dfw);
            c2 = (float)(fw * (1.0 / (12.0 * M_PI)));
            c3 = (float)(dfw * (1.0 / (36.0 * M_PI)));
            cv = (float)(fw * (1.0 / (6.0 * M_PI)));
        } else {
            c2 = (float)(gd * gd) * k8pi;
            c3 = (float)(gd * gd * gd) * k12pi;
            cv = (float)(gd * gd) * k4pi;
        }
        const float g = (float)gd, g2 = (float)(gd * gd);
        const float n0 = n[0], n1 = n[1], n2 = n[2];
        const float v1v2 = n[4] * n[7] + n[5] * n[8] + n[6] * n[9];
        const float v2v2 = n[7] * n[7] + n[8] * n[8] + n[9] * n[9];
        psi[0] = (float)(-log1p(-n3));
        psi[1] = n2 * g;
        psi[2] = n1 * g + (n2 * n2 - v2v2) * c2;
        psi[3] = n0 * g + (n1 * n2 - v1v2) * g2 + (n2 * n2 * n2 - 3.0f * n2 * v2v2) * c3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            psi[4 + c] = -n[7 + c] * g;
            psi[7 + c] = -n[4 + c] * g - n2 * n[7 + c] * cv;
        }
        bool ok = n3 < 1.0;
#pragma unroll
        for (int a = 0; a < kNumWeighted; ++a) ok = ok && isfinite(psi[a]);
        if (!ok) bad = true;
#pragma unroll
        for (int a = 0; a < kNumWeighted; ++a) f[a * N + p] = psi[a];
    }
    if (bad) atomicOr(flag, kFlagPacking);
}

// The same derivatives for double-float fields: the functions singular at
// packing, 1/(1 - n3) and ln(1 - n3) (and the White Bear phi3), in FP64;
// every product with the other weighted densities in double-float on the
// FP32 pipes, whose error (about 2^-47 of each term) stays far inside the
// FFT's.  Internal linkage: one copy per translation unit.
static __global__ void k_dphi_fields_dd(dd *__restrict__ f, size_t N, int *__restrict__ flag, int fmt) {
    const dd k8pi(1.0 / (8.0 * M_PI)), k12pi(1.0 / (12.0 * M_PI)), k4pi(1.0 / (4.0 * M_PI)), three(3);
    bool bad = false;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        dd n[kNumWeighted], psi[kNumWeighted];
#pragma unroll
        for (int a = 0; a < kNumWeighted; ++a) n[a] = f[a * N + p];
        const double n3 = (double)n[3];
        const double gd = 1.0 / (1.0 - n3);
        const dd g(gd), g2 = g * g;
        // coefficient functions of n2^2 (psi2, vector psi) and n2^3 (psi3)
        dd c2, c3, cv;
        if (fmt == PNP_FMT_WHITE_BEAR) {
            double fw = 0.0, dfw = 0.0;
            if (n3 < 1.0) wb_phi3(n3, fw, dfw);
            c2 = dd(fw * (1.0 / (12.0 * M_PI)));
            c3 = dd(dfw * (1.0 / (36.0 * M_PI)));
            cv = dd(fw * (1.0 / (6.0 * M_PI)));
        } else {
            c2 = g2 * k8pi;
            c3 = g2 * g * k12pi;
            cv = g2 * k4pi;
        }
        const dd n0 = n[0], n1 = n[1], n2 = n[2];
        const dd v1v2 = n[4] * n[7] + n[5] * n[8] + n[6] * n[9];
        const dd v2v2 = n[7] * n[7] + n[8] * n[8] + n[9] * n[9];
        psi[0] = dd(-log1p(-n3));
        psi[1] = n2 * g;
        psi[2] = n1 * g + (n2 * n2 - v2v2) * c2;
        psi[3] = n0 * g + (n1 * n2 - v1v2) * g2 + (n2 * n2 * n2 - three * n2 * v2v2) * c3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            psi[4 + c] = -(n[7 + c] * g);
            psi[7 + c] = -(n[4 + c] * g) - n2 * n[7 + c] * cv;
        }
        bool ok = n3 < 1.0;
#pragma unroll
        for (int a = 0; a < kNumWeighted; ++a) ok = ok && isfinite(psi[a].hi) && isfinite(psi[a].lo);
        if (!ok) bad = true;
#pragma unroll
        for (int a = 0; a < kNumWeighted; ++a) f[a * N + p] = psi[a];
    }
    if (bad) atomicOr(flag, kFlagPacking);
}

}  // namespace pnp

#include "mu_ex_reg.cuh"
#include "zcol256.cuh"

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
                        if (alpha == 0) g *= sc_c0<T>(sc, i);
                        if (alpha == 1) g *= sc_c1<T>(sc, i);
                        acc.x += g * r.x;
                        acc.y += g * r.y;
                    } else {
                        const int comp = (alpha - 4) % 3;
                        T sv = spec_at(spec, d, i, 2 + comp, kx, ky, kz);
                        if (alpha < 7) sv *= sc_c1<T>(sc, i);
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
                if (!fmt_dphi(n, psi, d.fmt)) bad = 1;
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
                    if (alpha == 0) g *= sc_c0<T>(sc, i);
                    if (alpha == 1) g *= sc_c1<T>(sc, i);
                    o.x += g * v.x;
                    o.y += g * v.y;
                } else {
                    const int comp = (alpha - 4) % 3;
                    T sv = spec_at(spec, d, i, 2 + comp, kx, ky, kz);
                    if (alpha < 7) sv *= sc_c1<T>(sc, i);
                    // K = -i S:  (-i S)(a + ib) = (S b, -S a)
                    o.x += sv * v.y;
                    o.y -= sv * v.x;
                }
            }
        }
        __syncthreads();
    }
    if (sc.msa) {
        // MSA correlations (Sec 2.3.4): Bs still holds the densities'
        // y-spectra; mu_i -= sum_j C_ij rho_j (the stored spectra are -C_ij)
        const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
        const int fy = ky <= d.Ly / 2 ? ky : d.Ly - ky;
        for (int j = 0; j < sc.s; ++j) {
            const C *src = Bs + (size_t)j * d.nz * d.Ly * d.Wx + (size_t)ky * d.Wx;
            for (int idx = threadIdx.x; idx < col; idx += blockDim.x) {
                const int z = idx / TX, c = idx % TX, kx = kx0 + c;
                C v = C{0, 0};
                if (z < d.nz && kx < d.Wx) v = src[(size_t)z * d.Ly * d.Wx + kx];
                work[idx] = v;
            }
            __syncthreads();
            C *r = fft_lines<false>(work, scr, TX, ax, tw);
            for (int idx = threadIdx.x; idx < col; idx += blockDim.x) {
                const int kz = idx / TX, c = idx % TX, kx = kx0 + c;
                if (kx >= d.Wx) continue;
                const int fz = kz <= d.Lz / 2 ? kz : d.Lz - kz;
                const C v = r[idx];
                for (int i = 0; i < sc.s; ++i) {
                    const T g = ldgt(&spec[(size_t)(sc.s * kNumKernels + msa_pair(i, j, sc.s)) * oct +
                                           ((size_t)fz * d.Oy + fy) * d.Ox + kx]);
                    C &o = acc[(size_t)i * col + idx];
                    o.x += g * v.x;
                    o.y += g * v.y;
                }
            }
            __syncthreads();
        }
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
                       const double *__restrict__ U, SpeciesConst sc, int P, const double *__restrict__ E) {
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
        double r0 = (double)v.x + u0, r1 = (double)v.y + u1;
        if (E) {
            const double *e = E + f * out_fstride;
            r0 += e[((size_t)z * d.ny + y0) * d.nx + x];
            if (y0 + 1 < d.ny) r1 += e[((size_t)z * d.ny + y0 + 1) * d.nx + x];
        }
        dst[(size_t)y0 * d.nx + x] = r0;
        if (y0 + 1 < d.ny) dst[(size_t)(y0 + 1) * d.nx + x] = r1;
    }
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
    const size_t cs = prec == PNP_PREC_FP32 ? 8 : 16;
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

// function attributes belong to a device's context: set them once per device
static inline int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev;
}

template <typename T> static int set_smem_attrs() {
    static std::atomic<unsigned long long> done_mask{0};
    const int dev = current_device();
    const unsigned long long bit = 1ull << (dev & 63);
    if (done_mask.load() & bit) return PNP_OK;
    const int big = 200 * 1024;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaFuncSetAttribute(k_xfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_ypass<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_ypass<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_zmac<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_xfused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_zback<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    e = e ? e : cudaFuncSetAttribute(k_xinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e != cudaSuccess) return cuda_status(e);
    done_mask.fetch_or(bit);
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
    const size_t cs = prec == PNP_PREC_FP32 ? 8 : 16;
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
// tensor-core (3xTF32) y pass of the FP32 pipeline, in its own unit
bool ypass_tc_supported(const Dims &d);
void ypass_tc_matrices(float *out);
int launch_ypass_tc(bool inv, const float2 *in, float2 *out, const Dims &d, int rows_in, int n_in, int rows_out,
                    int n_out, int F, const float2 *tw, const float *bmat, int *flag, cudaStream_t st);

template <typename F> static bool with_shape(int L, F &&f) {
    using std::integral_constant;
    switch (L) {
        case 16: f(integral_constant<int, 4>{}, integral_constant<int, 4>{}); return true;
        case 20: f(integral_constant<int, 5>{}, integral_constant<int, 4>{}); return true;
        case 24: f(integral_constant<int, 8>{}, integral_constant<int, 3>{}); return true;
        case 32: f(integral_constant<int, 8>{}, integral_constant<int, 4>{}); return true;
        case 40: f(integral_constant<int, 8>{}, integral_constant<int, 5>{}); return true;
        case 48: f(integral_constant<int, 16>{}, integral_constant<int, 3>{}); return true;
        case 64: f(integral_constant<int, 8>{}, integral_constant<int, 8>{}); return true;
        case 80: f(integral_constant<int, 16>{}, integral_constant<int, 5>{}); return true;
        case 96: f(integral_constant<int, 16>{}, integral_constant<int, 6>{}); return true;
        case 128: f(integral_constant<int, 16>{}, integral_constant<int, 8>{}); return true;
        case 256: f(integral_constant<int, 16>{}, integral_constant<int, 16>{}); return true;
        default: return false;
    }
}

template <auto K> static void ensure_smem() {
    static std::atomic<unsigned long long> done_mask{0};
    const unsigned long long bit = 1ull << (current_device() & 63);
    if (done_mask.load() & bit) return;
    cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    done_mask.fetch_or(bit);
}

// dynamic shared memory the register kernels may request (ensure_smem), and
// their threads per CTA (their __launch_bounds__)
constexpr long kSmemCap = 200 * 1024;
constexpr int kMaxThreads = 256;

// lines per CTA of the x kernels: the tuned tile if set, else 256 threads;
// at most 1024 threads, the shared-memory cap and the line pairs there are
static int x_lines(const Problem *p, int G, long ex_bytes, int npairs) {
    int P = p->tile[0] > 0 ? p->tile[0] : 256 / G;
    P = std::min<long>(P, std::min<long>(kMaxThreads / G, kSmemCap / ex_bytes));
    return std::max(1, std::min(P, npairs));
}

// split derivative stage (see stage 5 of run_pipeline)
constexpr bool kSplitDerivatives = true;

// z MAC / z back on the 64-lane radix-4 kernels (zcol256.cuh) when the z
// length is 256, there are at most three species and the values are
// double-float: measured 2.2x / 1.5x faster than the two-factor kernels at
// 128^3 -> 256^3, whose residency the shared-memory accumulators cap at 6
// warps per SM.  The FP32 (bound by latency) and FP64 (bound by the FP64
// pipe) two-factor kernels stay faster.  False otherwise.
template <typename T>
static bool launch_z4(bool back, int s, bool msa, typename vec2<T>::type *B10, typename vec2<T>::type *Bs,
                      const Dims &d, const typename vec2<T>::type *twz, const T *spec, const SpeciesConst &sc,
                      cudaStream_t st) {
    if constexpr (!std::is_same<T, dd>::value) {
        return false;
    } else {
        if (d.Lz != kZ4Len || s < 1 || s > kZ4MaxSpecies) return false;
        constexpr int TX = z4_tx<T>();
        const dim3 g((d.Wx + TX - 1) / TX, d.Ly / 2 + 1);
        const int threads = kZ4Lanes * 2 * TX;
        auto go = [&](auto sv) {
            constexpr int S = decltype(sv)::value;
            if (!back) {
                ensure_smem<k_zmac_q4<T, S>>();
                k_zmac_q4<T, S><<<g, threads, z4_smem_mac<T>(), st>>>(Bs, B10, d, twz, spec, sc);
            } else if (msa) {
                ensure_smem<k_zback_q4<T, S, true>>();
                k_zback_q4<T, S, true><<<g, threads, z4_smem_back<T>(), st>>>(B10, Bs, d, twz, spec, sc);
            } else {
                ensure_smem<k_zback_q4<T, S, false>>();
                k_zback_q4<T, S, false><<<g, threads, z4_smem_back<T>(), st>>>(B10, Bs, d, twz, spec, sc);
            }
        };
        if (s == 1) go(std::integral_constant<int, 1>{});
        else if (s == 2) go(std::integral_constant<int, 2>{});
        else go(std::integral_constant<int, 3>{});
        return true;
    }
}

// FP32 z MAC / z back with the per-column state in registers
// (k_zmac_reg / k_zback_reg) for Lz = 256, at most three species and no MSA
// term; false otherwise
template <typename T, int N1, int N2>
static bool launch_zreg(bool back, int s, bool msa, typename vec2<T>::type *B10, typename vec2<T>::type *Bs,
                        const Dims &d, const typename vec2<T>::type *twz, const T *spec, const SpeciesConst &sc,
                        cudaStream_t st) {
    if constexpr (!std::is_same<T, float>::value || N1 != 16 || N2 != 16) {
        return false;
    } else {
        if (s < 1 || s > 3 || msa) return false;
        constexpr int TX = 4;
        const dim3 g((d.Wx + TX - 1) / TX, d.Ly / 2 + 1);
        const int threads = Shape<N1, N2>::G * 2 * TX;
        const size_t sm = zreg_smem<N1, N2>(d, s, TX);
        auto go = [&](auto sv) {
            constexpr int S = decltype(sv)::value;
            if (!back)
                k_zmac_reg<N1, N2, S><<<g, threads, sm, st>>>(Bs, B10, d, twz, spec, sc, TX);
            else
                k_zback_reg<N1, N2, S><<<g, threads, sm, st>>>(B10, Bs, d, twz, spec, sc, TX);
        };
        if (s == 1) go(std::integral_constant<int, 1>{});
        else if (s == 2) go(std::integral_constant<int, 2>{});
        else go(std::integral_constant<int, 3>{});
        return true;
    }
}

template <typename T>
static int run_pipeline(Problem *p, DeviceBuffers *db, const double *d_rho, double *d_mu, cudaStream_t st,
                        bool tc = false) {
    using C = typename vec2<T>::type;
    const int prec = std::is_same<T, float>::value ? PNP_PREC_FP32
                     : (std::is_same<T, dd>::value ? PNP_PREC_DF64 : PNP_PREC_FP64);
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
            const int P = x_lines(p, G, Shape<N1, N2>::EX * (long)cs, d.npairs);
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
        if constexpr (std::is_same<T, float>::value) {
            if (tc && db->tc_b && ypass_tc_supported(d)) {
                launch_ypass_tc(inv, in, out, d, rows_in, rows_in, rows_out, rows_out, F, twy, db->tc_b, p->d_flag,
                                st);
                tm.end(st);
                return;
            }
        }
        if (!with_shape(d.Ly, [&](auto a, auto b) {
                constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
                int TX = pow2_le(std::min<long>(256 / G, 16));
                if (p->tile[1] > 0)
                    TX = std::max(1, std::min<int>(p->tile[1], (int)std::min<long>(kMaxThreads / G,
                                                                                    kSmemCap / (Shape<N1, N2>::EX * (long)cs))));
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
        if (launch_z4<T>(back, s, sc.msa != 0, B10, Bs, d, twz, spec, sc, st)) {
            tm.end(st);
            return;
        }
        if (!with_shape(d.Lz, [&](auto a, auto b) {
                constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
                if (launch_zreg<T, N1, N2>(back, s, sc.msa != 0, B10, Bs, d, twz, spec, sc, st)) return;
                // paired columns (ky, Ly - ky): 2 TX columns per CTA
                const long per_col = ((long)s * N1 * G + Shape<N1, N2>::EX) * (long)cs;
                int TX = pow2_le(std::max<long>(1, std::min<long>(std::min<long>(128 / G, 8), kBudget / (2 * per_col))));
                if (p->tile[2] > 0)
                    TX = std::max(1, std::min<int>(p->tile[2], (int)std::min<long>(kMaxThreads / (2 * G),
                                                                                    (kSmemCap - (long)G * G * cs) /
                                                                                        (2 * per_col))));
                dim3 g((d.Wx + TX - 1) / TX, d.Ly / 2 + 1);
                const size_t sm = 2 * TX * per_col + (size_t)G * G * cs;   // + twiddle table
                if (back && sc.msa) {
                    ensure_smem<k_zback_p<T, N1, N2, true>>();
                    k_zback_p<T, N1, N2, true><<<g, 2 * TX * G, sm, st>>>(B10, Bs, d, twz, spec, sc, TX);
                } else if (back) {
                    ensure_smem<k_zback_p<T, N1, N2>>();
                    k_zback_p<T, N1, N2><<<g, 2 * TX * G, sm, st>>>(B10, Bs, d, twz, spec, sc, TX);
                } else {
                    ensure_smem<k_zmac_p<T, N1, N2>>();
                    k_zmac_p<T, N1, N2><<<g, 2 * TX * G, sm, st>>>(Bs, B10, d, twz, spec, sc, TX);
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

    // 5: x inverse -> dPhi/dn -> forward.  Split form (real n fields through
    // the idle y-spectra buffer, a pointwise kernel at full occupancy) or one
    // fused kernel; both use the register FFT where the length allows.  The
    // real fields keep the FFT's number format (double-float as FP32 pairs:
    // no FP64 conversions in the x kernels).
    tm.begin(4, st);
    using V = typename std::conditional<std::is_same<T, double>::value, double, T>::type;
    V *nf = reinterpret_cast<V *>(B10);     // [10][nz][ny][nx], B10 is free here
    if (!with_shape(d.Lx, [&](auto a, auto b) {
            constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
            if (kSplitDerivatives) {
                const int P = x_lines(p, G, Shape<N1, N2>::EX * (long)cs, d.npairs);
                const size_t sm = P * Shape<N1, N2>::EX * cs;
                dim3 g((d.npairs + P - 1) / P, d.nz, kNumWeighted);
                ensure_smem<k_xinv_raw_r<T, N1, N2, V>>();
                k_xinv_raw_r<T, N1, N2, V><<<g, P * G, sm, st>>>(A, nf, d, twx, P);
                if constexpr (std::is_same<V, float>::value)
                    k_dphi_fields_mixed<<<std::min<size_t>((N + 255) / 256, 152 * 16), 256, 0, st>>>(
                        nf, N, p->d_flag, p->fmt);
                else if constexpr (std::is_same<V, dd>::value)
                    k_dphi_fields_dd<<<std::min<size_t>((N + 255) / 256, 152 * 16), 256, 0, st>>>(
                        nf, N, p->d_flag, p->fmt);
                else
                    k_dphi_fields<V><<<std::min<size_t>((N + 255) / 256, 152 * 16), 256, 0, st>>>(nf, N, p->d_flag,
                                                                                                p->fmt);
                ensure_smem<k_xfwd_r<T, N1, N2, V>>();
                k_xfwd_r<T, N1, N2, V><<<g, P * G, sm, st>>>(nf, N, A, d, twx, P);
            } else {
                const int NQ = std::min(N2, (d.nx + N1 - 1) / N1);
                const long per_pair = ((long)kNumWeighted * NQ * N1 + Shape<N1, N2>::EX) * (long)cs;
                const int P =
                    (int)std::max<long>(1, std::min<long>(std::min<long>(256 / G, d.npairs), kBudget / per_pair));
                ensure_smem<k_xfused_r<T, N1, N2>>();
                dim3 g((d.npairs + P - 1) / P, d.nz);
                k_xfused_r<T, N1, N2><<<g, P * G, P * per_pair, st>>>(A, d, twx, p->d_flag, P, NQ);
            }
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
    const double *E = p->msa ? p->d_E : nullptr;
    if (!with_shape(d.Lx, [&](auto a, auto b) {
            constexpr int N1 = decltype(a)::value, N2 = decltype(b)::value, G = Shape<N1, N2>::G;
            const int P = x_lines(p, G, Shape<N1, N2>::EX * (long)cs, d.npairs);
            ensure_smem<k_xinv_r<T, N1, N2>>();
            dim3 g((d.npairs + P - 1) / P, d.nz, s);
            k_xinv_r<T, N1, N2><<<g, P * G, P * Shape<N1, N2>::EX * cs, st>>>(A, d_mu, N, d, twx, U, sc, P, E);
        })) {
        dim3 gx((d.npairs + l.P_x - 1) / l.P_x, d.nz, s);
        k_xinv<T><<<gx, T256, l.sm_x, st>>>(A, d_mu, N, d, p->ax[0], twx, U, sc, l.P_x, E);
    }
    tm.end(st);
    return cuda_status(cudaGetLastError());
}

// one instantiation of run_pipeline per precision, each in its own file
int run_pipeline_fp64(Problem *p, DeviceBuffers *db, const double *d_rho, double *d_mu, cudaStream_t st);
int run_pipeline_fp32(Problem *p, DeviceBuffers *db, const double *d_rho, double *d_mu, cudaStream_t st,
                      bool tc = false);
int run_pipeline_df64(Problem *p, DeviceBuffers *db, const double *d_rho, double *d_mu, cudaStream_t st);

}  // namespace pnp
