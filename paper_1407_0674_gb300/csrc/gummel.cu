// Relaxed Gummel iteration on the device (Sec 3.2) with multigrid-
// preconditioned conjugate gradients for the Poisson equation (Sec 2.1) and
// the Slotboom-transformed Nernst-Planck equations (Sec 2.1, 7-point
// harmonic-mean stencil of Sec 3.1).
//
// Operators are matrix-free: per grid level, face coefficients cx[p] (face to
// the +x neighbour, wrapping; zero across a no-flux wall), cy[p], cz[p] (face
// to +z; on the top plane the face to the upper Dirichlet plane) and czlo[p]
// (face to the lower Dirichlet plane, plane 0 only);
//   (A u)_p = sum_faces c (u_p - u_nbr),  Dirichlet neighbours moved to b.
// Multigrid (replacing the paper's external algebraic multigrid, Sec 3.3):
// cells are aggregated 2x2x2 (per axis while even and >= 4); the coarse
// operator is the Galerkin product with piecewise-constant interpolation,
// i.e. coarse face coefficients are sums of the fine faces between two
// aggregates; restriction sums the 8 fine residuals, prolongation adds the
// coarse value.  One V(1,1) cycle with red-black sweeps (red-black before,
// black-red after, so the cycle is a symmetric operator) preconditions CG;
// the coarsest level gets 40 symmetric sweeps in one CTA.  All dot products
// use a fixed-shape two-stage reduction, so results are bitwise reproducible.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "pnp_internal.h"

namespace pnp {

struct Op {
    int nx, ny, nz;
    const double *cx, *cy, *cz, *czlo;
    const double *dg = nullptr;    // optional extra diagonal (Poisson-Boltzmann screening)
};

struct Level {
    int nx, ny, nz;
    size_t n;
    int fx, fy, fz;                // aggregation factors to the next level
    double *cx, *cy, *cz, *czlo;   // operator being solved (Poisson or NP)
    double *pcx, *pcy, *pcz, *pczlo;   // Poisson copy (built once)
    double *dg;                    // diagonal term of the screened Poisson operator
    double *x, *b, *r;
};

constexpr int kRedBlocks = 512;
constexpr int kCoarseSweeps = 40;
constexpr double kCoarseScale = 1.8;
constexpr double kMixStepLimit = 0.2;     // |step in ln rho| of PNP_MIX_GEOMETRIC_LIMITED

// device-side record of a solve (written by the loop-control kernels)
struct DevStats {
    int status;            // PNP_OK, PNP_ERR_NOT_CONVERGED, PNP_ERR_PACKING, PNP_ERR_OVERFLOW
    int iters;             // Gummel iterations done
    int pcg_it;            // iterations of the current linear solve
    int pad;
    double residual;       // last Gummel residual
    long long lin;         // linear iterations over the solve
    double lin_tol;        // current tolerance of the linear solves (adaptive mode)
    int eq_enable;         // run the equilibrium stage (set before each launch)
    int eq_iters;          // its iterations
    double eq_residual;    // its last residual
    int redos;             // Anderson: sweeps repeated after an unphysical one
};

// control block of the Anderson mixing (see the kernels further down)
constexpr int kAaMaxDepth = 6;
constexpr int kAaMaxK = kAaMaxDepth * (kAaMaxDepth + 1) / 2 + kAaMaxDepth;   // Gram entries + right-hand side
struct AaCtl {
    int m;             // depth
    int head, hlen;    // ring of m + 1 entries: logical a -> physical (head + a) % (m + 1)
    int slot;          // physical entry of this iteration
    int redo;          // 1: this sweep is repeated from the restored plain iterate
    int skip;          // 1: no extrapolation this iteration (converged or failed)
    int rslot;         // entry whose X + F is restored on a redo
    int kd;            // differences in the history this iteration
    int bt;            // backtracking level after a failed sweep (-1: none)
    double theta;      // step factor of the state being retried
    double gamma[kAaMaxDepth];
};
constexpr int kAaBacktrack = 8;    // step halvings after the restart from the plain iterate

struct GummelState {
    std::vector<Level> lv;
    double *mu = nullptr, *rho_new = nullptr;
    double *phi = nullptr, *rho = nullptr;    // solve state the graph works on
    DevStats *stats = nullptr;
    int *keep_q = nullptr;                    // valences and fixed charge used by the graph
    double *keep_rhof = nullptr;
    cudaStream_t cap[2] = {nullptr, nullptr}; // capture streams of the loop bodies
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double *rhs = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *pv = nullptr, *Ap = nullptr;
    double *partial = nullptr;     // kRedBlocks
    double *lam = nullptr, *prev = nullptr;   // PNP_MIX_ADAPTIVE: per-point factor and last step
    double *scal = nullptr;        // device scalars
    // Anderson mixing (depth m > 0): history of m + 1 iterates x = (phi, ln rho)
    // and residuals f = G(x) - x, [m+1][(1+s) N] each, a control block and the
    // Gram reduction's block partials
    double *aa_X = nullptr, *aa_F = nullptr, *aa_part = nullptr;
    double *aa_xb = nullptr, *aa_fb = nullptr;   // base pair (x, f) of a backtrack
    struct AaCtl *aa = nullptr;
    double *phase = nullptr;          // PNP_FLAG_PHASE_TIMING: ns per phase, then the last mark
    unsigned long long *dmax = nullptr;
    size_t bytes = 0;
    bool poisson_ready = false;
    bool shift = false;            // operators carry the levels' dg while capturing
};

enum { S_RZ = 0, S_PAP, S_RR, S_ALPHA, S_BETA, S_RZNEW, S_BB, S_TGT, S_COUNT };

__device__ __forceinline__ size_t pidx(int i, int j, int k, int nx, int ny) {
    return ((size_t)k * ny + j) * nx + i;
}

__device__ __forceinline__ double op_diag(const Op &A, int i, int j, int k, size_t p) {
    const int im = i == 0 ? A.nx - 1 : i - 1, jm = j == 0 ? A.ny - 1 : j - 1;
    double d = A.cx[p] + A.cy[p] + A.cz[p];
    d += A.cx[pidx(im, j, k, A.nx, A.ny)] + A.cy[pidx(i, jm, k, A.nx, A.ny)];
    d += k > 0 ? A.cz[p - (size_t)A.nx * A.ny] : A.czlo[p];
    if (A.dg) d += A.dg[p];
    return d;
}

__device__ __forceinline__ double op_nbr(const Op &A, const double *__restrict__ u, int i, int j, int k, size_t p) {
    const int ip = i + 1 == A.nx ? 0 : i + 1, im = i == 0 ? A.nx - 1 : i - 1;
    const int jp = j + 1 == A.ny ? 0 : j + 1, jm = j == 0 ? A.ny - 1 : j - 1;
    const size_t plane = (size_t)A.nx * A.ny;
    const size_t pxm = pidx(im, j, k, A.nx, A.ny), pym = pidx(i, jm, k, A.nx, A.ny);
    double s = A.cx[p] * u[pidx(ip, j, k, A.nx, A.ny)] + A.cx[pxm] * u[pxm];
    s += A.cy[p] * u[pidx(i, jp, k, A.nx, A.ny)] + A.cy[pym] * u[pym];
    if (k + 1 < A.nz) s += A.cz[p] * u[p + plane];
    if (k > 0) s += A.cz[p - plane] * u[p - plane];
    return s;
}

#define GRID_LOOP(p, n) for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < (n); p += (size_t)gridDim.x * blockDim.x)

__global__ void k_residual(Op A, const double *__restrict__ x, const double *__restrict__ b, double *__restrict__ r) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    GRID_LOOP(p, n) {
        const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / ((size_t)A.nx * A.ny);
        r[p] = b[p] - (op_diag(A, i, j, k, p) * x[p] - op_nbr(A, x, i, j, k, p));
    }
}

__global__ void k_apply(Op A, const double *__restrict__ x, double *__restrict__ y) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    GRID_LOOP(p, n) {
        const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / ((size_t)A.nx * A.ny);
        y[p] = op_diag(A, i, j, k, p) * x[p] - op_nbr(A, x, i, j, k, p);
    }
}

// one colour of a red-black sweep: x_p = (b_p + sum c x_nbr) / diag_p for
// points with (i + j + k) % 2 == color.  With zero_init the other colour is
// taken as zero (first sweep from x = 0).
__global__ void k_color_sweep(Op A, double *__restrict__ x, const double *__restrict__ b, int color) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    GRID_LOOP(p, n) {
        const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / ((size_t)A.nx * A.ny);
        if (((i + j + k) & 1) != color) continue;
        x[p] = (b[p] + op_nbr(A, x, i, j, k, p)) / op_diag(A, i, j, k, p);
    }
}

// coarsest level: x = 0, then kCoarseSweeps symmetric (red, black, black, red) sweeps in one CTA
__global__ void k_coarse_solve(Op A, double *__restrict__ x, const double *__restrict__ b) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    for (size_t p = threadIdx.x; p < n; p += blockDim.x) x[p] = 0.0;
    __syncthreads();
    for (int s = 0; s < kCoarseSweeps; ++s) {
        const int order[4] = {0, 1, 1, 0};
        for (int c = 0; c < 4; ++c) {
            for (size_t p = threadIdx.x; p < n; p += blockDim.x) {
                const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / ((size_t)A.nx * A.ny);
                if (((i + j + k) & 1) != order[c]) continue;
                x[p] = (b[p] + op_nbr(A, x, i, j, k, p)) / op_diag(A, i, j, k, p);
            }
            __syncthreads();
        }
    }
}

// coarse face coefficients: sums of the fine faces leaving each aggregate
__global__ void k_coarsen(Op F, int fx, int fy, int fz, int cnx, int cny, int cnz, double *__restrict__ cx,
                          double *__restrict__ cy, double *__restrict__ cz, double *__restrict__ czlo) {
    const size_t n = (size_t)cnx * cny * cnz;
    GRID_LOOP(q, n) {
        const int I = q % cnx, J = (q / cnx) % cny, K = q / ((size_t)cnx * cny);
        double sx = 0, sy = 0, sz = 0, sl = 0;
        for (int c = 0; c < fz; ++c)
            for (int b = 0; b < fy; ++b)
                for (int a = 0; a < fx; ++a) {
                    const int i = I * fx + a, j = J * fy + b, k = K * fz + c;
                    const size_t p = pidx(i, j, k, F.nx, F.ny);
                    if (a == fx - 1) sx += F.cx[p];
                    if (b == fy - 1) sy += F.cy[p];
                    if (c == fz - 1) sz += F.cz[p];
                    if (c == 0 && K == 0) sl += F.czlo[p];
                }
        cx[q] = sx;
        cy[q] = sy;
        cz[q] = sz;
        czlo[q] = sl;
    }
}

__global__ void k_restrict(const double *__restrict__ rf, int nx, int ny, int fx, int fy, int fz, int cnx, int cny,
                           int cnz, double *__restrict__ bc) {
    const size_t n = (size_t)cnx * cny * cnz;
    GRID_LOOP(q, n) {
        const int I = q % cnx, J = (q / cnx) % cny, K = q / ((size_t)cnx * cny);
        double s = 0;
        for (int c = 0; c < fz; ++c)
            for (int b = 0; b < fy; ++b)
                for (int a = 0; a < fx; ++a) s += rf[pidx(I * fx + a, J * fy + b, K * fz + c, nx, ny)];
        bc[q] = s;
    }
}

// x_fine += scale * x_coarse (piecewise constant); scale > 1 compensates the
// weak correction of piecewise-constant interpolation
__global__ void k_prolong_add(double *__restrict__ xf, int nx, int ny, int nz, int fx, int fy, int fz, int cnx,
                              int cny, const double *__restrict__ xc, double scale) {
    const size_t n = (size_t)nx * ny * nz;
    GRID_LOOP(p, n) {
        const int i = p % nx, j = (p / nx) % ny, k = p / ((size_t)nx * ny);
        xf[p] += scale * xc[pidx(i / fx, j / fy, k / fz, cnx, cny)];
    }
}

__global__ void k_fill(double *__restrict__ a, double v, size_t n) {
    GRID_LOOP(p, n) a[p] = v;
}

// deterministic dot product, stage 1: fixed grid of kRedBlocks blocks
__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, size_t n,
                              double *__restrict__ partial) {
    __shared__ double sh[256];
    double s = 0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        s += a[p] * b[p];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// stage 2: one block sums the partials into scal[slot]
__global__ void k_dot_final(const double *__restrict__ partial, double *__restrict__ scal, int slot) {
    __shared__ double sh[kRedBlocks];
    for (int t = threadIdx.x; t < kRedBlocks; t += blockDim.x) sh[t] = partial[t];
    __syncthreads();
    for (int w = kRedBlocks / 2; w > 0; w >>= 1) {
        for (int t = threadIdx.x; t < w; t += blockDim.x) sh[t] += sh[t + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[slot] = sh[0];
}

__global__ void k_scalars_alpha(double *scal) {
    scal[S_ALPHA] = scal[S_RZ] / scal[S_PAP];
}

__global__ void k_scalars_beta(double *scal) {
    scal[S_BETA] = scal[S_RZNEW] / scal[S_RZ];
    scal[S_RZ] = scal[S_RZNEW];
}

// x += alpha p ; r -= alpha Ap
__global__ void k_update_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const double *__restrict__ Ap, const double *__restrict__ scal, size_t n) {
    const double a = scal[S_ALPHA];
    GRID_LOOP(k, n) {
        x[k] += a * p[k];
        r[k] -= a * Ap[k];
    }
}

// p = z + beta p
__global__ void k_update_p(double *__restrict__ p, const double *__restrict__ z, const double *__restrict__ scal,
                           size_t n) {
    const double b = scal[S_BETA];
    GRID_LOOP(k, n) p[k] = z[k] + b * p[k];
}

__global__ void k_copy(double *__restrict__ d, const double *__restrict__ s, size_t n) {
    GRID_LOOP(k, n) d[k] = s[k];
}

// ---------------------------------------------------------------------------
// physics kernels
struct PhysConst {
    int nx, ny, nz, bcx, bcy;
    double lB;
    double phi_lo, phi_hi;
};

// Poisson face coefficients (h = 1): 1, zero across no-flux walls
__global__ void k_poisson_coefs(PhysConst c, double *cx, double *cy, double *cz, double *czlo) {
    const size_t n = (size_t)c.nx * c.ny * c.nz;
    GRID_LOOP(p, n) {
        const int i = p % c.nx, j = (p / c.nx) % c.ny, k = p / ((size_t)c.nx * c.ny);
        cx[p] = (c.bcx == PNP_BC_NOFLUX && i == c.nx - 1) ? 0.0 : 1.0;
        cy[p] = (c.bcy == PNP_BC_NOFLUX && j == c.ny - 1) ? 0.0 : 1.0;
        cz[p] = 1.0;
        czlo[p] = k == 0 ? 1.0 : 0.0;
    }
}

// b = 4 pi lB (rho_f + sum_i q_i rho_i) + Dirichlet contributions
__global__ void k_poisson_rhs(PhysConst c, const double *__restrict__ rho, int s, const int *__restrict__ q,
                              const double *__restrict__ rho_f, double *__restrict__ b) {
    const size_t n = (size_t)c.nx * c.ny * c.nz;
    const size_t plane = (size_t)c.nx * c.ny;
    GRID_LOOP(p, n) {
        double ch = rho_f ? rho_f[p] : 0.0;
        for (int i = 0; i < s; ++i) ch += q[i] * rho[i * n + p];
        double v = 4.0 * M_PI * c.lB * ch;
        if (p < plane) v += c.phi_lo;
        if (p >= n - plane) v += c.phi_hi;
        b[p] = v;
    }
}

// Screened Poisson step of the Gummel iteration: Newton right-hand side
// b(rho) - A phi at the current densities and the screening term
// dg = 4 pi lB sum q^2 rho (A: the Poisson operator)
__global__ void k_scr_rhs(Op A, PhysConst c, const double *__restrict__ rho, int s, const int *__restrict__ q,
                          const double *__restrict__ rho_f, const double *__restrict__ phi, double *__restrict__ rhs,
                          double *__restrict__ dg) {
    const size_t n = (size_t)c.nx * c.ny * c.nz;
    const size_t plane = (size_t)c.nx * c.ny;
    GRID_LOOP(p, n) {
        const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / plane;
        double ch = rho_f ? rho_f[p] : 0.0, sc = 0.0;
        for (int a = 0; a < s; ++a) {
            const double r = rho[a * n + p];
            ch += q[a] * r;
            sc += (double)(q[a] * q[a]) * r;
        }
        double b = 4.0 * M_PI * c.lB * ch;
        if (k == 0) b += c.phi_lo;
        if (k + 1 == c.nz) b += c.phi_hi;
        rhs[p] = b - (op_diag(A, i, j, k, p) * phi[p] - op_nbr(A, phi, i, j, k, p));
        dg[p] = 4.0 * M_PI * c.lB * sc;
    }
}

// phi* = phi + dphi, then phi_new = l1 phi* + (1 - l1) phi; track max |phi_new - phi|
__global__ void k_relax_phi_step(double *__restrict__ phi, const double *__restrict__ dphi, double l1, size_t n,
                                 unsigned long long *__restrict__ dmax) {
    double m = 0;
    GRID_LOOP(p, n) {
        const double ps = phi[p] + dphi[p];
        const double v = l1 * ps + (1.0 - l1) * phi[p];
        m = fmax(m, fabs(v - phi[p]));
        phi[p] = v;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(dmax, (unsigned long long)__double_as_longlong(m));
}

// phi_new = l1 phi* + (1 - l1) phi ; track max |phi_new - phi|
__global__ void k_relax_phi(double *__restrict__ phi, const double *__restrict__ phis, double l1, size_t n,
                            unsigned long long *__restrict__ dmax) {
    double m = 0;
    GRID_LOOP(p, n) {
        const double v = l1 * phis[p] + (1.0 - l1) * phi[p];
        m = fmax(m, fabs(v - phi[p]));
        phi[p] = v;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(dmax, (unsigned long long)__double_as_longlong(m));
}

struct NpConst {
    double D, q, Dlo, Dhi, rlo, rhi;
};

// Slotboom coefficients (Sec 2.1) and the harmonic-mean face coefficients
// (Sec 3.1): Dbar = D exp(-(q phi + mu)); faces to the Dirichlet planes use
// the reservoir value D exp(-(q phi_face + mu_b)).  Also writes the Dirichlet
// right-hand side and the initial guess rhobar = rho exp(q phi + mu).
__global__ void k_np_setup(PhysConst c, NpConst s, const double *__restrict__ phi, const double *__restrict__ mu,
                           const double *__restrict__ rho, double *__restrict__ cx, double *__restrict__ cy,
                           double *__restrict__ cz, double *__restrict__ czlo, double *__restrict__ b,
                           double *__restrict__ x0, int *__restrict__ flag) {
    const size_t n = (size_t)c.nx * c.ny * c.nz;
    const size_t plane = (size_t)c.nx * c.ny;
    bool bad = false;
    GRID_LOOP(p, n) {
        const int i = p % c.nx, j = (p / c.nx) % c.ny, k = p / plane;
        auto Db = [&](size_t t) { return s.D * exp(-(s.q * phi[t] + mu[t])); };
        const double d0 = Db(p);
        const size_t pxp = pidx(i + 1 == c.nx ? 0 : i + 1, j, k, c.nx, c.ny);
        const size_t pyp = pidx(i, j + 1 == c.ny ? 0 : j + 1, k, c.nx, c.ny);
        double vx = 0, vy = 0;
        if (!(c.bcx == PNP_BC_NOFLUX && i == c.nx - 1)) {
            const double d1 = Db(pxp);
            vx = 2.0 * d0 * d1 / (d0 + d1);
        }
        if (!(c.bcy == PNP_BC_NOFLUX && j == c.ny - 1)) {
            const double d1 = Db(pyp);
            vy = 2.0 * d0 * d1 / (d0 + d1);
        }
        double vz;
        if (k + 1 < c.nz) {
            const double d1 = Db(p + plane);
            vz = 2.0 * d0 * d1 / (d0 + d1);
        } else {
            vz = 2.0 * d0 * s.Dhi / (d0 + s.Dhi);
        }
        const double vl = k == 0 ? 2.0 * d0 * s.Dlo / (d0 + s.Dlo) : 0.0;
        cx[p] = vx;
        cy[p] = vy;
        cz[p] = vz;
        czlo[p] = vl;
        double bv = 0;
        if (k == 0) bv += vl * s.rlo;
        if (k + 1 == c.nz) bv += vz * s.rhi;
        b[p] = bv;
        const double x = rho[p] * exp(s.q * phi[p] + mu[p]);
        x0[p] = x;
        if (!isfinite(d0) || !isfinite(x) || !(d0 > 0)) bad = true;
    }
    if (bad) atomicOr(flag, kFlagOverflow);
}

// rho* = rhobar exp(-(q phi + mu)); relaxation (linear or geometric); track
// max |rho_new - rho| / rho_b
__global__ void k_np_finish(size_t n, double q, double l2, int mix, double inv_rb, const double *__restrict__ phi,
                            const double *__restrict__ mu, const double *__restrict__ rbar, double *__restrict__ rho,
                            double *__restrict__ lam, double *__restrict__ prev,
                            unsigned long long *__restrict__ dmax, int *__restrict__ flag) {
    double m = 0;
    bool bad = false;
    GRID_LOOP(p, n) {
        const double rs = rbar[p] * exp(-(q * phi[p] + mu[p]));
        const double old = rho[p];
        double v;
        if (mix == PNP_MIX_LINEAR) {
            v = l2 * rs + (1.0 - l2) * old;
        } else if (mix == PNP_MIX_ADAPTIVE) {
            // per-point factor: halved when the step in ln rho changes sign
            const double d = log(rs / old);
            double a = lam[p];
            a = d * prev[p] < 0.0 ? fmax(0.5 * a, l2 / 1024.0) : fmin(1.1 * a, l2);
            const double step = fmin(fmax(a * d, -kMixStepLimit), kMixStepLimit);
            lam[p] = a;
            prev[p] = step;
            v = old * exp(step);
        } else {
            double step = l2 * log(rs / old);
            if (mix == PNP_MIX_GEOMETRIC_LIMITED) step = fmin(fmax(step, -kMixStepLimit), kMixStepLimit);
            v = old * exp(step);
        }
        if (!isfinite(v) || !(v > 0)) bad = true;
        m = fmax(m, fabs(v - old) * inv_rb);
        rho[p] = v;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(dmax, (unsigned long long)__double_as_longlong(m));
    if (bad) atomicOr(flag, kFlagOverflow);
}

__global__ void k_init_phi(PhysConst c, double *__restrict__ phi) {
    const size_t n = (size_t)c.nx * c.ny * c.nz;
    GRID_LOOP(p, n) {
        const int k = p / ((size_t)c.nx * c.ny);
        phi[p] = c.phi_lo + (c.phi_hi - c.phi_lo) * (k + 1.0) / (c.nz + 1.0);
    }
}


// first red sweep from x = 0: red points b/diag, black points 0 (replaces a
// fill and a sweep)
__global__ void k_sweep_zero(Op A, double *__restrict__ x, const double *__restrict__ b) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    GRID_LOOP(p, n) {
        const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / ((size_t)A.nx * A.ny);
        x[p] = ((i + j + k) & 1) ? 0.0 : b[p] / op_diag(A, i, j, k, p);
    }
}

// coarse right-hand side = sum of the fine residuals b - A x over each aggregate
__global__ void k_residual_restrict(Op F, const double *__restrict__ x, const double *__restrict__ b, int fx, int fy,
                                    int fz, int cnx, int cny, int cnz, double *__restrict__ bc) {
    const size_t n = (size_t)cnx * cny * cnz;
    GRID_LOOP(q, n) {
        const int I = q % cnx, J = (q / cnx) % cny, K = q / ((size_t)cnx * cny);
        double s = 0;
        for (int c = 0; c < fz; ++c)
            for (int bb = 0; bb < fy; ++bb)
                for (int a = 0; a < fx; ++a) {
                    const int i = I * fx + a, j = J * fy + bb, k = K * fz + c;
                    const size_t p = pidx(i, j, k, F.nx, F.ny);
                    s += b[p] - (op_diag(F, i, j, k, p) * x[p] - op_nbr(F, x, i, j, k, p));
                }
        bc[q] = s;
    }
}

// coarsest level in shared memory: x = 0, then kCoarseSweeps symmetric
// red-black sweeps; n <= kCoarseMax
constexpr int kCoarseMax = 1024;
__global__ void k_coarse_smem(Op A, double *__restrict__ x_out, const double *__restrict__ b_in) {
    extern __shared__ double csm[];
    const int n = A.nx * A.ny * A.nz;
    double *x = csm, *b = csm + n, *dg = csm + 2 * n, *cx = csm + 3 * n, *cy = csm + 4 * n, *cz = csm + 5 * n,
           *cl = csm + 6 * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        x[p] = 0.0;
        b[p] = b_in[p];
        cx[p] = A.cx[p];
        cy[p] = A.cy[p];
        cz[p] = A.cz[p];
        cl[p] = A.czlo[p];
    }
    __syncthreads();
    const Op S{A.nx, A.ny, A.nz, cx, cy, cz, cl};
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / (A.nx * A.ny);
        dg[p] = op_diag(S, i, j, k, p) + (A.dg ? A.dg[p] : 0.0);
    }
    __syncthreads();
    const int order[4] = {0, 1, 1, 0};
    for (int s = 0; s < kCoarseSweeps; ++s)
        for (int c = 0; c < 4; ++c) {
            for (int p = threadIdx.x; p < n; p += blockDim.x) {
                const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / (A.nx * A.ny);
                if (((i + j + k) & 1) != order[c]) continue;
                x[p] = (b[p] + op_nbr(S, x, i, j, k, p)) / dg[p];
            }
            __syncthreads();
        }
    for (int p = threadIdx.x; p < n; p += blockDim.x) x_out[p] = x[p];
}

// y = A x and the block partial sums of x . y
__global__ void k_apply_dot(Op A, const double *__restrict__ x, double *__restrict__ y, double *__restrict__ partial) {
    __shared__ double sh[256];
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    double acc = 0;
    GRID_LOOP(p, n) {
        const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / ((size_t)A.nx * A.ny);
        const double v = op_diag(A, i, j, k, p) * x[p] - op_nbr(A, x, i, j, k, p);
        y[p] = v;
        acc += x[p] * v;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// x += alpha p; r -= alpha Ap; block partial sums of r . r
__global__ void k_update_xr_dot(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                                const double *__restrict__ Ap, const double *__restrict__ scal, size_t n,
                                double *__restrict__ partial) {
    __shared__ double sh[256];
    const double a = scal[S_ALPHA];
    double acc = 0;
    GRID_LOOP(k, n) {
        x[k] += a * p[k];
        const double v = r[k] - a * Ap[k];
        r[k] = v;
        acc += v * v;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// fixed-order sum of nb block partials into scal[slot], then an optional
// scalar step: 1 alpha = rz / pAp, 2 beta = rz_new / rz
__device__ __forceinline__ double block_sum_partials(const double *__restrict__ partial, int nb) {
    __shared__ double sh[kRedBlocks];
    for (int t = threadIdx.x; t < kRedBlocks; t += blockDim.x) sh[t] = t < nb ? partial[t] : 0.0;
    __syncthreads();
    for (int w = kRedBlocks / 2; w > 0; w >>= 1) {
        for (int t = threadIdx.x; t < w; t += blockDim.x) sh[t] += sh[t + w];
        __syncthreads();
    }
    return sh[0];
}

__global__ void k_final(const double *__restrict__ partial, int nb, double *__restrict__ scal, int slot, int step) {
    const double v = block_sum_partials(partial, nb);
    if (threadIdx.x == 0) {
        scal[slot] = v;
        if (step == 1) scal[S_ALPHA] = scal[S_RZ] / v;
        if (step == 2) {
            scal[S_BETA] = v / scal[S_RZ];
            scal[S_RZ] = v;
        }
    }
}

// sum of r . r, then the loop decision of the CG iteration
__global__ void k_final_check(const double *__restrict__ partial, int nb, double *__restrict__ scal, int maxit,
                              DevStats *st, int *flag, cudaGraphConditionalHandle h) {
    const double rr = block_sum_partials(partial, nb);
    if (threadIdx.x == 0) {
        scal[S_RR] = rr;
        const int it = ++st->pcg_it;
        st->lin += 1;
        const bool finite = isfinite(rr);
        if (!finite) atomicOr(flag, kFlagOverflow);
        cudaGraphSetConditional(h, (finite && rr > scal[S_TGT] && it < maxit) ? 1u : 0u);
    }
}

// Nernst-Planck current of one species through every z face (Sec 2.1, 3.1):
// J_k = sum over the plane of Dbar_face (rhobar_k - rhobar_k+1) between planes
// k and k+1 (k = -1 .. nz-1; the Dirichlet planes carry the reservoir values),
// Dbar = D exp(-(q phi + mu)), rhobar = rho exp(q phi + mu), harmonic-mean
// faces.  One CTA per face, fixed-order reduction.
__global__ void k_plane_flux(PhysConst c, NpConst s, const double *__restrict__ phi, const double *__restrict__ mu,
                             const double *__restrict__ rho, double *__restrict__ flux) {
    __shared__ double sh[256];
    const int kf = (int)blockIdx.x - 1;
    const size_t plane = (size_t)c.nx * c.ny;
    double acc = 0.0;
    for (size_t t = threadIdx.x; t < plane; t += blockDim.x) {
        double Da, ra, Db, rb;
        if (kf < 0) {
            Da = s.Dlo;
            ra = s.rlo;
        } else {
            const size_t a = (size_t)kf * plane + t;
            const double e = s.q * phi[a] + mu[a];
            Da = s.D * exp(-e);
            ra = rho[a] * exp(e);
        }
        if (kf + 1 >= c.nz) {
            Db = s.Dhi;
            rb = s.rhi;
        } else {
            const size_t b = (size_t)(kf + 1) * plane + t;
            const double e = s.q * phi[b] + mu[b];
            Db = s.D * exp(-e);
            rb = rho[b] * exp(e);
        }
        acc += 2.0 * Da * Db / (Da + Db) * (ra - rb);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) flux[blockIdx.x] = sh[0];
}

// ---------------------------------------------------------------------------
// equilibrium cDFT initial guess (Sec 3.2, choice of initial guess)
constexpr int kMaxSpecies = 8;
constexpr double kEqPhiStep = 1.0;        // |Newton step of phi| per point, kT/e
struct EqConst {
    int s;
    int q[kMaxSpecies];
    double cb[kMaxSpecies];       // rho_b,i exp(mu_b,i): rho_i = cb_i exp(-(mu_ex,i + q_i phi))
    double inv_rb[kMaxSpecies];
    double lam;
};

// Newton right-hand side of the Poisson-Boltzmann equation at the current
// phi with the Boltzmann densities of mu_ex: rhs = b(phi) - A phi, and the
// screening term dg = 4 pi lB sum q^2 rho (A: the Poisson operator)
__global__ void k_eq_rhs(Op A, PhysConst c, EqConst e, const double *__restrict__ phi, const double *__restrict__ mu,
                         const double *__restrict__ rho_f, double *__restrict__ rhs, double *__restrict__ dg,
                         int *__restrict__ flag) {
    const size_t n = (size_t)c.nx * c.ny * c.nz;
    const size_t plane = (size_t)c.nx * c.ny;
    bool bad = false;
    GRID_LOOP(p, n) {
        const int i = p % A.nx, j = (p / A.nx) % A.ny, k = p / plane;
        double ch = rho_f ? rho_f[p] : 0.0, sc = 0.0;
        for (int a = 0; a < e.s; ++a) {
            const double r = e.cb[a] * exp(-(mu[a * n + p] + e.q[a] * phi[p]));
            ch += e.q[a] * r;
            sc += (double)(e.q[a] * e.q[a]) * r;
        }
        double b = 4.0 * M_PI * c.lB * ch;
        if (k == 0) b += c.phi_lo;
        if (k + 1 == c.nz) b += c.phi_hi;
        const double v = b - (op_diag(A, i, j, k, p) * phi[p] - op_nbr(A, phi, i, j, k, p));
        const double d = 4.0 * M_PI * c.lB * sc;
        rhs[p] = v;
        dg[p] = d;
        if (!isfinite(v) || !isfinite(d)) bad = true;
    }
    if (bad) atomicOr(flag, kFlagOverflow);
}

// phi += clamp(dphi); rho moves toward the Boltzmann densities of the new phi
// by the step-limited geometric relaxation; track the residual
__global__ void k_eq_update(size_t n, EqConst e, double *__restrict__ phi, const double *__restrict__ dphi,
                            const double *__restrict__ mu, double *__restrict__ rho,
                            unsigned long long *__restrict__ dmax, int *__restrict__ flag) {
    double m = 0;
    bool bad = false;
    GRID_LOOP(p, n) {
        const double d = fmin(fmax(dphi[p], -kEqPhiStep), kEqPhiStep);
        const double ph = phi[p] + d;
        phi[p] = ph;
        m = fmax(m, fabs(d));
        for (int a = 0; a < e.s; ++a) {
            const size_t t = a * n + p;
            const double rs = e.cb[a] * exp(-(mu[t] + e.q[a] * ph));
            const double old = rho[t];
            const double step = fmin(fmax(e.lam * log(rs / old), -kMixStepLimit), kMixStepLimit);
            const double v = old * exp(step);
            if (!isfinite(v) || !(v > 0)) bad = true;
            m = fmax(m, fabs(v - old) * e.inv_rb[a]);
            rho[t] = v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(dmax, (unsigned long long)__double_as_longlong(m));
    if (bad) atomicOr(flag, kFlagOverflow);
}

// ---------------------------------------------------------------------------
// loop control on the device (conditional graph nodes)

// start of a linear solve: target = tol^2 ||b||^2; enter the loop unless the
// warm start already meets it
__global__ void k_pcg_init(double *scal, double tol, DevStats *st, int *flag, cudaGraphConditionalHandle h) {
    if (!(tol > 0)) tol = st->lin_tol;      // adaptive: set by the Gummel loop
    double bb = scal[S_BB];
    if (!(bb > 0)) bb = 1.0;
    const double tgt = tol * tol * bb;
    const double rr = scal[S_RR];
    scal[S_TGT] = tgt;
    st->pcg_it = 0;
    const bool finite = isfinite(rr);
    if (!finite) atomicOr(flag, kFlagOverflow);
    cudaGraphSetConditional(h, (finite && rr > tgt) ? 1u : 0u);
}

// end of a CG iteration: continue while ||r||^2 > target and below maxit
__global__ void k_pcg_check(const double *scal, int maxit, DevStats *st, int *flag, cudaGraphConditionalHandle h) {
    const double rr = scal[S_RR];
    const int it = ++st->pcg_it;
    st->lin += 1;
    const bool finite = isfinite(rr);
    if (!finite) atomicOr(flag, kFlagOverflow);
    cudaGraphSetConditional(h, (finite && rr > scal[S_TGT] && it < maxit) ? 1u : 0u);
}

// end of a Gummel iteration: residual, status, continue or stop
__global__ void k_gummel_check(const unsigned long long *dmax, const int *flag, double tol, int max_iter,
                               DevStats *st, cudaGraphConditionalHandle h, const AaCtl *aa) {
    const unsigned long long bits = *dmax;
    const double res = __longlong_as_double((long long)bits);
    if (aa && aa->redo) {
        // the sweep is repeated from the restored plain iterate: same iteration
        st->redos += 1;
        cudaGraphSetConditional(h, 1u);
        return;
    }
    const int it = ++st->iters;
    st->residual = res;
    const int f = *flag;
    // inexact inner solves: tolerance follows the outer residual (forcing term)
    st->lin_tol = fmin(1e-6, fmax(1e-12, 0.01 * res));
    unsigned cont = 0;
    if (f & kFlagPacking) st->status = PNP_ERR_PACKING;
    else if (f & (kFlagOverflow | kFlagNonFinite)) st->status = PNP_ERR_OVERFLOW;
    else if (res < tol) st->status = PNP_OK;
    else if (it >= max_iter) st->status = PNP_ERR_NOT_CONVERGED;
    else cont = 1;
    cudaGraphSetConditional(h, cont);
}

// end of an equilibrium iteration: residual, status, continue or hand over
// to the Gummel loop (which an error skips)
__global__ void k_eq_check(const unsigned long long *dmax, const int *flag, double tol, int max_iter, DevStats *st,
                           cudaGraphConditionalHandle h_eq, cudaGraphConditionalHandle h_g) {
    const unsigned long long bits = *dmax;
    const double res = __longlong_as_double((long long)bits);
    const int it = ++st->eq_iters;
    st->eq_residual = res;
    st->lin_tol = fmin(1e-6, fmax(1e-12, 0.01 * res));
    const int f = *flag;
    unsigned cont = 0;
    if (f & kFlagPacking) st->status = PNP_ERR_PACKING;
    else if (f & (kFlagOverflow | kFlagNonFinite)) st->status = PNP_ERR_OVERFLOW;
    else if (res < tol) st->status = PNP_OK;
    else if (it >= max_iter) st->status = PNP_ERR_NOT_CONVERGED;
    else cont = 1;
    cudaGraphSetConditional(h_eq, cont);
    if (!cont && (f & (kFlagPacking | kFlagOverflow | kFlagNonFinite))) cudaGraphSetConditional(h_g, 0u);
}

// first node of a graph with the equilibrium stage: enter it if requested,
// and the Gummel loop if it has iterations
__global__ void k_eq_gate(const DevStats *st, cudaGraphConditionalHandle h_eq, cudaGraphConditionalHandle h_g,
                          int gummel) {
    cudaGraphSetConditional(h_eq, st->eq_enable ? 1u : 0u);
    cudaGraphSetConditional(h_g, gummel ? 1u : 0u);
}

__global__ void k_stats_reset(DevStats *st, int eq_enable) {
    st->lin_tol = 1e-6;
    st->status = PNP_ERR_NOT_CONVERGED;
    st->iters = 0;
    st->pcg_it = 0;
    st->residual = 0;
    st->lin = 0;
    st->eq_enable = eq_enable;
    st->eq_iters = 0;
    st->eq_residual = 0;
    st->redos = 0;
}

// ---------------------------------------------------------------------------
// Anderson mixing of the relaxed Gummel iteration (an extension; the paper
// relaxes only).  G is one sweep of the loop body acting on x = (phi, ln rho);
// with the last k <= m differences dX_a, dF_a of iterates and residuals
// f = G(x) - x,
//   gamma = argmin || f - dF gamma ||_2   (normal equations, ridge 1e-12 tr),
//   x <- x + f - sum_a gamma_a (dX_a + dF_a).
// If the sweep from an extrapolated state is unphysical (packing, overflow,
// non-finite) the history is dropped and the sweep repeated from the last
// plain iterate G(x_prev) = X + F of the newest entry, in the same iteration;
// while that fails as well, the step from x_prev is halved (x_prev + F/2,
// x_prev + F/4, ..., kAaBacktrack times at most).
// The stopping test is on the plain sweep's residual, so the fixed point is
// the relaxed iteration's.
__global__ void k_aa_reset(AaCtl *a, int m) {
    a->m = m;
    a->head = a->hlen = a->slot = a->redo = a->skip = a->rslot = a->kd = 0;
    a->bt = -1;
    a->theta = 1.0;
}

// start of an iteration: make room for the entry of the current state
__global__ void k_aa_begin(AaCtl *a) {
    const int R = a->m + 1;
    if (a->hlen == R) {
        a->head = (a->head + 1) % R;
        a->hlen = a->m;
    }
    a->slot = (a->head + a->hlen) % R;
    a->redo = 0;
    a->skip = 0;
}

__device__ __forceinline__ double aa_state(const double *phi, const double *rho, size_t N, size_t e) {
    return e < N ? phi[e] : log(rho[e - N]);
}

// X[slot] = x = (phi, ln rho) before the sweep
__global__ void k_aa_save_x(const AaCtl *__restrict__ a, const double *__restrict__ phi,
                            const double *__restrict__ rho, double *__restrict__ X, size_t N, size_t M) {
    double *x = X + (size_t)a->slot * M;
    GRID_LOOP(e, M) x[e] = aa_state(phi, rho, N, e);
}

// after the sweep: a failed sweep from an extrapolated state (history and
// not the first iteration) is repeated from the last plain iterate x + f of
// the newest entry; while the repeat fails too, from x + theta f with theta
// halved each time (x swept cleanly), at most kAaBacktrack times; a converged
// or failed sweep is not extrapolated
__global__ void k_aa_post(AaCtl *a, const unsigned long long *dmax, int *flag, double tol, const DevStats *st) {
    const double rr = __longlong_as_double((long long)*dmax);
    const int bad = *flag & (kFlagPacking | kFlagOverflow | kFlagNonFinite);
    if (bad && st->iters > 0 && (a->hlen > 0 || a->bt >= 0)) {
        if (a->hlen > 0) {
            a->bt = 0;
            a->rslot = (a->head + a->hlen - 1) % (a->m + 1);
        } else {
            a->bt += 1;
        }
        a->skip = 1;
        if (a->bt > kAaBacktrack) {
            a->bt = -1;           // give up: the error ends the solve
            return;
        }
        a->redo = 1;
        a->theta = ldexp(1.0, -a->bt);
        a->hlen = 0;
        atomicAnd(flag, ~(kFlagPacking | kFlagOverflow | kFlagNonFinite));
        return;
    }
    if (!bad) a->bt = -1;
    if (bad || rr < tol) a->skip = 1;
}

// redo: (phi, rho) = x + theta f of the base pair, taken from the newest
// history entry at the first repeat (theta = 1: the plain iterate)
__global__ void k_aa_restore(const AaCtl *__restrict__ a, const double *__restrict__ X,
                             const double *__restrict__ F, double *__restrict__ xb, double *__restrict__ fb,
                             double *__restrict__ phi, double *__restrict__ rho, size_t N, size_t M) {
    if (!a->redo) return;
    const double *x = X + (size_t)a->rslot * M, *f = F + (size_t)a->rslot * M;
    const bool first = a->bt == 0;
    const double th = a->theta;
    GRID_LOOP(e, M) {
        double v;
        if (first) {
            const double xe = x[e], fe = f[e];
            xb[e] = xe;
            fb[e] = fe;
            v = xe + fe;
        } else {
            v = xb[e] + th * fb[e];
        }
        if (e < N) phi[e] = v;
        else rho[e - N] = exp(v);
    }
}

// F[slot] = G(x) - x, and block partials of the Gram entries
// dF_a . dF_b (b <= a < kd) and dF_a . f, dF_a = F[a+1] - F[a] in logical
// order, f = F[slot] (the newest entry)
template <int KD>
__device__ void aa_gram_body(const AaCtl &a, const double *__restrict__ phi, const double *__restrict__ rho,
                             const double *__restrict__ X, double *__restrict__ F, size_t N, size_t M,
                             double *__restrict__ part) {
    constexpr int K = KD * (KD + 1) / 2 + KD;
    double acc[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const int R = a.m + 1;
    const double *x = X + (size_t)a.slot * M;
    double *fs = F + (size_t)a.slot * M;
    GRID_LOOP(e, M) {
        const double f = aa_state(phi, rho, N, e) - x[e];
        fs[e] = f;
        if constexpr (KD > 0) {
            double Fv[KD + 1];
#pragma unroll
            for (int j = 0; j < KD; ++j) Fv[j] = F[(size_t)((a.head + j) % R) * M + e];
            Fv[KD] = f;
            double dF[KD];
#pragma unroll
            for (int j = 0; j < KD; ++j) dF[j] = Fv[j + 1] - Fv[j];
            int k = 0;
#pragma unroll
            for (int i = 0; i < KD; ++i) {
#pragma unroll
                for (int j = 0; j <= i; ++j) acc[k++] += dF[i] * dF[j];
                acc[k++] += dF[i] * f;
            }
        }
    }
    if constexpr (K > 0) {
        __shared__ double sh[K][8];
        const int w = threadIdx.x / 32, l = threadIdx.x % 32;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (l == 0) sh[k][w] = v;
        }
        __syncthreads();
        if (threadIdx.x < K) {
            double v = 0.0;
            for (int j = 0; j < 8; ++j) v += sh[threadIdx.x][j];
            part[(size_t)threadIdx.x * kRedBlocks + blockIdx.x] = v;
        }
    }
}

// block of 256 threads; entries are ordered (a, b <= a, then rhs a) for a < kd
__global__ void __launch_bounds__(256) k_aa_record(AaCtl *a, const double *__restrict__ phi,
                                                   const double *__restrict__ rho, const double *__restrict__ X,
                                                   double *__restrict__ F, size_t N, size_t M,
                                                   double *__restrict__ part) {
    if (a->skip) return;
    const int kd = a->hlen;       // differences once this entry is in: hlen + 1 entries
    switch (kd) {
        case 0: aa_gram_body<0>(*a, phi, rho, X, F, N, M, part); break;
        case 1: aa_gram_body<1>(*a, phi, rho, X, F, N, M, part); break;
        case 2: aa_gram_body<2>(*a, phi, rho, X, F, N, M, part); break;
        case 3: aa_gram_body<3>(*a, phi, rho, X, F, N, M, part); break;
        case 4: aa_gram_body<4>(*a, phi, rho, X, F, N, M, part); break;
        case 5: aa_gram_body<5>(*a, phi, rho, X, F, N, M, part); break;
        default: aa_gram_body<6>(*a, phi, rho, X, F, N, M, part); break;
    }
}

// sum the partials in a fixed order, enter the new entry into the history,
// and solve the kd x kd normal equations in one thread (Gaussian elimination
// with partial pivoting; gamma = 0, the plain iterate, if singular)
__global__ void k_aa_solve(AaCtl *a, const double *__restrict__ part, int nb) {
    __shared__ double tot[kAaMaxK];
    if (a->skip) return;
    const int kd = a->hlen;
    const int K = kd * (kd + 1) / 2 + kd;
    for (int k = 0; k < K; ++k) {
        const double v = block_sum_partials(part + (size_t)k * kRedBlocks, nb);
        if (threadIdx.x == 0) tot[k] = v;
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    a->hlen += 1;
    a->kd = kd;
    double A[kAaMaxDepth * kAaMaxDepth], b[kAaMaxDepth];
    int k = 0;
    for (int i = 0; i < kd; ++i) {
        for (int j = 0; j <= i; ++j) {
            A[i * kd + j] = A[j * kd + i] = tot[k];
            ++k;
        }
        b[i] = tot[k++];
    }
    double tr = 0.0;
    for (int i = 0; i < kd; ++i) tr += A[i * kd + i];
    for (int i = 0; i < kd; ++i) A[i * kd + i] += 1e-12 * tr + 1e-300;
    bool ok = true;
    for (int c = 0; c < kd && ok; ++c) {
        int piv = c;
        for (int r = c + 1; r < kd; ++r)
            if (fabs(A[r * kd + c]) > fabs(A[piv * kd + c])) piv = r;
        if (A[piv * kd + c] == 0.0) {
            ok = false;
            break;
        }
        if (piv != c) {
            for (int j = 0; j < kd; ++j) {
                const double t = A[c * kd + j];
                A[c * kd + j] = A[piv * kd + j];
                A[piv * kd + j] = t;
            }
            const double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < kd; ++r) {
            const double f = A[r * kd + c] / A[c * kd + c];
            for (int j = c; j < kd; ++j) A[r * kd + j] -= f * A[c * kd + j];
            b[r] -= f * b[c];
        }
    }
    if (ok)
        for (int c = kd - 1; c >= 0; --c) {
            double v = b[c];
            for (int j = c + 1; j < kd; ++j) v -= A[c * kd + j] * b[j];
            b[c] = v / A[c * kd + c];
        }
    for (int i = 0; i < kAaMaxDepth; ++i) a->gamma[i] = (ok && i < kd) ? b[i] : 0.0;
}

// x_new = x + f - sum_a gamma_a (dX_a + dF_a); (phi, rho) = (x_new, exp x_new).
// With no differences the state stays G(x), as computed by the sweep.
__global__ void k_aa_update(const AaCtl *__restrict__ a, const double *__restrict__ X,
                            const double *__restrict__ F, double *__restrict__ phi, double *__restrict__ rho,
                            size_t N, size_t M) {
    if (a->skip || a->kd == 0) return;
    const int R = a->m + 1, kd = a->kd;
    const double *x = X + (size_t)a->slot * M, *f = F + (size_t)a->slot * M;
    GRID_LOOP(e, M) {
        double v = x[e] + f[e];
        for (int j = 0; j < kd; ++j) {
            const size_t p0 = (size_t)((a->head + j) % R) * M + e, p1 = (size_t)((a->head + j + 1) % R) * M + e;
            v -= a->gamma[j] * ((X[p1] - X[p0]) + (F[p1] - F[p0]));
        }
        if (e < N) phi[e] = v;
        else rho[e - N] = exp(v);
    }
}

// ---------------------------------------------------------------------------
// phase boundaries of a Gummel iteration (PNP_FLAG_PHASE_TIMING): the global
// nanosecond timer at each mark; the time since the previous mark is added to
// phase `slot` (slot < 0: only the mark).  rec[kPhases] holds the last mark.
constexpr int kPhases = 4;
__global__ void k_phase_mark(double *rec, int slot) {
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    unsigned long long *last = reinterpret_cast<unsigned long long *>(rec + kPhases);
    if (slot >= 0) rec[slot] += (double)(now - *last);
    *last = now;
}

// ---------------------------------------------------------------------------
// host orchestration
static int grid_for(size_t n) { return (int)std::min<size_t>(std::max<size_t>((n + 255) / 256, 1), 152 * 16); }

static Op op_of(const Level &L, bool shift = false) {
    return Op{L.nx, L.ny, L.nz, L.cx, L.cy, L.cz, L.czlo, shift ? L.dg : nullptr};
}

// one V(1,1) cycle for level l: x = M b (x, b default to the level's vectors)
static void vcycle(GummelState *g, int l, cudaStream_t st, double *x = nullptr, const double *b = nullptr) {
    Level &L = g->lv[l];
    if (!x) x = L.x;
    if (!b) b = L.b;
    const Op A = op_of(L, g->shift);
    const int G = grid_for(L.n);
    if (l + 1 == (int)g->lv.size()) {
        if (L.n <= (size_t)kCoarseMax)
            k_coarse_smem<<<1, 256, 7 * L.n * sizeof(double), st>>>(A, x, b);
        else
            k_coarse_solve<<<1, 512, 0, st>>>(A, x, b);
        return;
    }
    Level &C = g->lv[l + 1];
    // V(2,2): red, black, red, black before; black, red, black, red after
    k_sweep_zero<<<G, 256, 0, st>>>(A, x, b);
    k_color_sweep<<<G, 256, 0, st>>>(A, x, b, 1);
    k_color_sweep<<<G, 256, 0, st>>>(A, x, b, 0);
    k_color_sweep<<<G, 256, 0, st>>>(A, x, b, 1);
    k_residual_restrict<<<grid_for(C.n), 256, 0, st>>>(A, x, b, L.fx, L.fy, L.fz, C.nx, C.ny, C.nz, C.b);
    vcycle(g, l + 1, st);
    k_prolong_add<<<G, 256, 0, st>>>(x, L.nx, L.ny, L.nz, L.fx, L.fy, L.fz, C.nx, C.ny, C.x, kCoarseScale);
    k_color_sweep<<<G, 256, 0, st>>>(A, x, b, 1);
    k_color_sweep<<<G, 256, 0, st>>>(A, x, b, 0);
    k_color_sweep<<<G, 256, 0, st>>>(A, x, b, 1);
    k_color_sweep<<<G, 256, 0, st>>>(A, x, b, 0);
}

static void coarsen_all(GummelState *g, cudaStream_t st) {
    for (size_t l = 0; l + 1 < g->lv.size(); ++l) {
        Level &F = g->lv[l], &C = g->lv[l + 1];
        k_coarsen<<<grid_for(C.n), 256, 0, st>>>(op_of(F), F.fx, F.fy, F.fz, C.nx, C.ny, C.nz, C.cx, C.cy, C.cz,
                                                 C.czlo);
    }
}

static void dot(GummelState *g, const double *a, const double *b, size_t n, int slot, cudaStream_t st) {
    k_dot_partial<<<kRedBlocks, 256, 0, st>>>(a, b, n, g->partial);
    k_dot_final<<<1, 256, 0, st>>>(g->partial, g->scal, slot);
}

// Append a conditional WHILE node to the capture on `st`; later captured work
// depends on it.  Returns its body graph and handle (default value `dflt`);
// with `have_handle` the caller's handle *h is used instead of a new one.
static cudaError_t add_while(cudaStream_t st, unsigned dflt, cudaGraphConditionalHandle *h, cudaGraph_t *body,
                             bool have_handle = false) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, &ed, &nd);
    if (e != cudaSuccess) return e;
    if (!have_handle) e = cudaGraphConditionalHandleCreate(h, cg, dflt, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = *h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, cg, deps, ed, nd, &prm);
    if (e != cudaSuccess) return e;
    *body = prm.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// MG-preconditioned CG on level 0's operator, recorded into the capture on
// `st` with the iteration loop as a conditional WHILE node whose body is
// captured on `sb`.  x holds the initial guess; stops at ||r||_2 <= tol ||b||_2
// or maxit iterations.  All reductions have a fixed shape.
static cudaError_t pcg_capture(GummelState *g, double *x, const double *b, double tol, int maxit, int *flag,
                               cudaStream_t st, cudaStream_t sb) {
    Level &L0 = g->lv[0];
    const Op A = op_of(L0, g->shift);
    const size_t n = L0.n;
    const int G = grid_for(n);
    const int NB = std::min(G, kRedBlocks);
    double *r = g->r, *z = g->z, *p = g->pv, *Ap = g->Ap;
    dot(g, b, b, n, S_BB, st);
    k_residual<<<G, 256, 0, st>>>(A, x, b, r);
    dot(g, r, r, n, S_RR, st);
    vcycle(g, 0, st, z, r);
    k_copy<<<G, 256, 0, st>>>(p, z, n);
    dot(g, r, z, n, S_RZ, st);
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    k_pcg_init<<<1, 1, 0, st>>>(g->scal, tol, g->stats, flag, h);
    cudaGraph_t body = nullptr;
    {
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *ed = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, &ed, &nd);
        if (e != cudaSuccess) return e;
        cudaGraphNodeParams prm = {};
        prm.type = cudaGraphNodeTypeConditional;
        prm.conditional.handle = h;
        prm.conditional.type = cudaGraphCondTypeWhile;
        prm.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, cg, deps, ed, nd, &prm);
        if (e != cudaSuccess) return e;
        body = prm.conditional.phGraph_out[0];
        e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e != cudaSuccess) return e;
    }
    e = cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    k_apply_dot<<<NB, 256, 0, sb>>>(A, p, Ap, g->partial);
    k_final<<<1, 256, 0, sb>>>(g->partial, NB, g->scal, S_PAP, 1);
    k_update_xr_dot<<<NB, 256, 0, sb>>>(x, r, p, Ap, g->scal, n, g->partial);
    k_final_check<<<1, 256, 0, sb>>>(g->partial, NB, g->scal, maxit, g->stats, flag, h);
    vcycle(g, 0, sb, z, r);
    k_dot_partial<<<NB, 256, 0, sb>>>(r, z, n, g->partial);
    k_final<<<1, 256, 0, sb>>>(g->partial, NB, g->scal, S_RZNEW, 2);
    k_update_p<<<G, 256, 0, sb>>>(p, z, g->scal, n);
    return cudaStreamEndCapture(sb, &body);
}

static void set_operator(GummelState *g, bool poisson) {
    for (auto &L : g->lv) {
        if (poisson) {
            std::swap(L.cx, L.pcx);
            std::swap(L.cy, L.pcy);
            std::swap(L.cz, L.pcz);
            std::swap(L.czlo, L.pczlo);
        }
    }
}

int gummel_setup(Problem *p) {
    if (p->gs) return PNP_OK;
    GummelState *g = new GummelState();
    p->gs = g;
    auto alloc = [&](double **ptr, size_t n) {
        if (dmalloc((void **)ptr, sizeof(double) * std::max<size_t>(n, 1), p->stream) != cudaSuccess) return false;
        g->bytes += sizeof(double) * std::max<size_t>(n, 1);
        return true;
    };
    // levels
    int nx = p->nx, ny = p->ny, nz = p->nz;
    while (true) {
        Level L{};
        L.nx = nx; L.ny = ny; L.nz = nz;
        L.n = (size_t)nx * ny * nz;
        // aggregate 2, 3 or 5 cells per axis, whichever divides: every
        // 2^a 3^b 5^c extent coarsens to a handful of unknowns
        auto fac = [](int n) { return (n >= 4 && n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : 1; };
        L.fx = fac(nx);
        L.fy = fac(ny);
        L.fz = fac(nz);
        bool last = L.n <= 8 || (L.fx == 1 && L.fy == 1 && L.fz == 1) || g->lv.size() >= 16;
        if (last) L.fx = L.fy = L.fz = 1;
        g->lv.push_back(L);
        if (last) break;
        nx /= L.fx; ny /= L.fy; nz /= L.fz;
    }
    // coarsest must fit the single-CTA solver comfortably
    const size_t N = p->npts();
    bool ok = true;
    for (size_t l = 0; l < g->lv.size() && ok; ++l) {
        Level &L = g->lv[l];
        ok = alloc(&L.cx, L.n) && alloc(&L.cy, L.n) && alloc(&L.cz, L.n) && alloc(&L.czlo, L.n) &&
             alloc(&L.pcx, L.n) && alloc(&L.pcy, L.n) && alloc(&L.pcz, L.n) && alloc(&L.pczlo, L.n) &&
             alloc(&L.x, L.n) && alloc(&L.b, L.n) && alloc(&L.r, L.n);
        L.dg = nullptr;
        if (ok && (p->eq_init || p->screened)) ok = alloc(&L.dg, L.n);
    }
    ok = ok && alloc(&g->mu, N * p->s) && alloc(&g->phi, N) && alloc(&g->rho, N * p->s) &&
         alloc(&g->rhs, N) && alloc(&g->x, N) && alloc(&g->r, N) &&
         alloc(&g->z, N) && alloc(&g->pv, N) && alloc(&g->Ap, N) && alloc(&g->partial, kRedBlocks) &&
         alloc(&g->scal, S_COUNT);
    if (ok && p->rho_mix == PNP_MIX_ADAPTIVE) ok = alloc(&g->lam, N * p->s) && alloc(&g->prev, N * p->s);
    if (ok && p->phase_timing) ok = alloc(&g->phase, kPhases + 1);
    if (ok && p->aa_depth > 0) {
        const size_t M = (1 + (size_t)p->s) * N;
        ok = alloc(&g->aa_X, (p->aa_depth + 1) * M) && alloc(&g->aa_F, (p->aa_depth + 1) * M) &&
             alloc(&g->aa_part, (size_t)kAaMaxK * kRedBlocks) && alloc(&g->aa_xb, M) && alloc(&g->aa_fb, M);
        if (ok && dmalloc((void **)&g->aa, sizeof(AaCtl), p->stream) != cudaSuccess) ok = false;
    }
    if (ok) {
        if (dmalloc((void **)&g->dmax, sizeof(unsigned long long), p->stream) != cudaSuccess) ok = false;
        if (ok && dmalloc((void **)&g->stats, sizeof(DevStats), p->stream) != cudaSuccess) ok = false;
        for (int k = 0; k < 2 && ok; ++k)
            if (cudaStreamCreateWithFlags(&g->cap[k], cudaStreamNonBlocking) != cudaSuccess) ok = false;
    }
    if (!ok) {
        // nothing half-built stays behind for a later solve to take as ready
        cudaStreamSynchronize(p->stream);
        gummel_free(p);
        return PNP_ERR_NOMEM;
    }
    p->device_bytes += g->bytes;
    p->mg_levels = (int)g->lv.size();
    cudaFuncSetAttribute(k_coarse_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, 7 * kCoarseMax * 8);
    // Poisson operator on every level (into the p* arrays)
    PhysConst c{p->nx, p->ny, p->nz, p->bc[0], p->bc[1], p->lB, p->phi_lo, p->phi_hi};
    set_operator(g, true);
    k_poisson_coefs<<<grid_for(N), 256, 0, p->stream>>>(c, g->lv[0].cx, g->lv[0].cy, g->lv[0].cz, g->lv[0].czlo);
    coarsen_all(g, p->stream);
    set_operator(g, true);
    const int rc = cuda_status(cudaStreamSynchronize(p->stream));
    if (rc) gummel_free(p);
    return rc;
}

void gummel_free(Problem *p) {
    GummelState *g = p->gs;
    if (!g) return;
    for (auto &L : g->lv) {
        for (double *a : {L.cx, L.cy, L.cz, L.czlo, L.pcx, L.pcy, L.pcz, L.pczlo, L.dg, L.x, L.b, L.r})
            dfree(a, p->stream);
    }
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (int k = 0; k < 2; ++k)
        if (g->cap[k]) cudaStreamDestroy(g->cap[k]);
    for (double *a : {g->mu, g->phi, g->rho, g->rhs, g->x, g->r, g->z, g->pv, g->Ap, g->partial, g->scal, g->lam,
                      g->prev, g->aa_X, g->aa_F, g->aa_part, g->aa_xb, g->aa_fb, g->phase})
        dfree(a, p->stream);
    dfree(g->aa, p->stream);
    dfree(g->dmax, p->stream);
    dfree(g->stats, p->stream);
    dfree(g->keep_q, p->stream);
    dfree(g->keep_rhof, p->stream);
    delete g;
    p->gs = nullptr;
}

// Record one whole Gummel solve into g->graph: an outer WHILE node over
// Gummel iterations whose body holds mu_ex, the Poisson solve, the phi
// relaxation, per species the Slotboom coefficients, the NP solve and the
// density update, and k_gummel_check, which ends the loop on convergence,
// a status error or max_iter.  Works on g->phi and g->rho.
static int build_graph(Problem *p, int *d_q, double *d_rhof) {
    NvtxRange range("build_solve_graph");
    GummelState *g = p->gs;
    const size_t N = p->npts();
    const int s = p->s;
    const int G = grid_for(N);
    PhysConst c{p->nx, p->ny, p->nz, p->bc[0], p->bc[1], p->lB, p->phi_lo, p->phi_hi};
    const int maxlin = 2000;
    cudaStream_t st = p->stream, sb = g->cap[0], sc = g->cap[1];
    const bool timer = p->timer.enabled;
    p->timer.enabled = false;
    cudaGraph_t top = nullptr;
    cudaError_t e = cudaGraphCreate(&top, 0);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(st, top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    cudaGraphConditionalHandle hg;
    cudaGraph_t body = nullptr;
    int rc = PNP_OK;
    if (e == cudaSuccess && p->eq_init) {
        // equilibrium stage: a gate node, then its own WHILE loop; the Gummel
        // loop's handle is set by the gate and cleared by a failed stage
        cudaGraphConditionalHandle he;
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&he, cg, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hg, cg, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) k_eq_gate<<<1, 1, 0, st>>>(g->stats, he, hg, p->max_iter > 0 ? 1 : 0);
        cudaGraph_t ebody = nullptr;
        if (e == cudaSuccess) e = add_while(st, 0, &he, &ebody, true);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(sb, ebody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            EqConst ec{};
            ec.s = s;
            for (int i = 0; i < s; ++i) {
                ec.q[i] = p->q[i];
                ec.cb[i] = p->rho_b[i] * std::exp(p->mu_bulk[i]);
                ec.inv_rb[i] = 1.0 / p->rho_b[i];
            }
            ec.lam = p->lambda_rho;
            rc = mu_ex_enqueue(p, p->precision, g->rho, g->mu, sb);
            cudaMemsetAsync(g->dmax, 0, sizeof(unsigned long long), sb);
            set_operator(g, true);
            Level &L0 = g->lv[0];
            k_eq_rhs<<<G, 256, 0, sb>>>(op_of(L0), c, ec, g->phi, g->mu, d_rhof, g->rhs, L0.dg, p->d_flag);
            for (size_t l = 0; l + 1 < g->lv.size(); ++l) {
                Level &F = g->lv[l], &C = g->lv[l + 1];
                k_restrict<<<grid_for(C.n), 256, 0, sb>>>(F.dg, F.nx, F.ny, F.fx, F.fy, F.fz, C.nx, C.ny, C.nz, C.dg);
            }
            k_fill<<<G, 256, 0, sb>>>(g->x, 0.0, N);
            g->shift = true;
            e = pcg_capture(g, g->x, g->rhs, p->lin_tol, maxlin, p->d_flag, sb, sc);
            g->shift = false;
            set_operator(g, true);
            k_eq_update<<<G, 256, 0, sb>>>(N, ec, g->phi, g->x, g->mu, g->rho, g->dmax, p->d_flag);
            k_eq_check<<<1, 1, 0, sb>>>(g->dmax, p->d_flag, p->eq_tol, p->eq_max_iter, g->stats, he, hg);
            cudaError_t e2 = cudaStreamEndCapture(sb, &ebody);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = add_while(st, 0, &hg, &body, true);
    } else if (e == cudaSuccess) {
        e = add_while(st, 1, &hg, &body);
    }
    if (e == cudaSuccess && rc == PNP_OK)
        e = cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    const size_t M = (1 + (size_t)s) * N;
    const int GM = grid_for(M), NBM = std::min(GM, kRedBlocks);
    if (e == cudaSuccess && rc == PNP_OK) {
        if (g->phase) k_phase_mark<<<1, 1, 0, sb>>>(g->phase, -1);
        if (g->aa) {
            // Anderson: the history entry of the state this sweep starts from
            k_aa_begin<<<1, 1, 0, sb>>>(g->aa);
            k_aa_save_x<<<GM, 256, 0, sb>>>(g->aa, g->phi, g->rho, g->aa_X, N, M);
        }
        // 1. mu_ex from rho^{n-1}
        rc = mu_ex_enqueue(p, p->precision, g->rho, g->mu, sb);
        if (g->phase) k_phase_mark<<<1, 1, 0, sb>>>(g->phase, 0);
        cudaMemsetAsync(g->dmax, 0, sizeof(unsigned long long), sb);
        // 2. Poisson for phi*, starting from phi; 3. relax phi
        set_operator(g, true);
        if (p->screened) {
            // one Newton step with the densities' Boltzmann response:
            // (A + dg) dphi = b(rho) - A phi, phi* = phi + dphi
            Level &L0 = g->lv[0];
            k_scr_rhs<<<G, 256, 0, sb>>>(op_of(L0), c, g->rho, s, d_q, d_rhof, g->phi, g->rhs, L0.dg);
            for (size_t l = 0; l + 1 < g->lv.size(); ++l) {
                Level &F = g->lv[l], &C = g->lv[l + 1];
                k_restrict<<<grid_for(C.n), 256, 0, sb>>>(F.dg, F.nx, F.ny, F.fx, F.fy, F.fz, C.nx, C.ny, C.nz, C.dg);
            }
            k_fill<<<G, 256, 0, sb>>>(g->x, 0.0, N);
            g->shift = true;
            e = pcg_capture(g, g->x, g->rhs, p->lin_tol, maxlin, p->d_flag, sb, sc);
            g->shift = false;
            set_operator(g, true);
            k_relax_phi_step<<<G, 256, 0, sb>>>(g->phi, g->x, p->lambda_phi, N, g->dmax);
        } else {
            k_poisson_rhs<<<G, 256, 0, sb>>>(c, g->rho, s, d_q, d_rhof, g->rhs);
            k_copy<<<G, 256, 0, sb>>>(g->x, g->phi, N);
            e = pcg_capture(g, g->x, g->rhs, p->lin_tol, maxlin, p->d_flag, sb, sc);
            set_operator(g, true);
            k_relax_phi<<<G, 256, 0, sb>>>(g->phi, g->x, p->lambda_phi, N, g->dmax);
        }
        if (g->phase) k_phase_mark<<<1, 1, 0, sb>>>(g->phase, 1);
        // 4. Nernst-Planck per species
        for (int i = 0; i < s && e == cudaSuccess; ++i) {
            NpConst nc;
            nc.D = p->D[i];
            nc.q = p->q[i];
            nc.Dlo = p->D[i] * std::exp(-(p->q[i] * p->phi_lo + p->mu_bulk[i]));
            nc.Dhi = p->D[i] * std::exp(-(p->q[i] * p->phi_hi + p->mu_bulk[i]));
            nc.rlo = p->rho_b[i] * std::exp(p->q[i] * p->phi_lo + p->mu_bulk[i]);
            nc.rhi = p->rho_b[i] * std::exp(p->q[i] * p->phi_hi + p->mu_bulk[i]);
            Level &L0 = g->lv[0];
            k_np_setup<<<G, 256, 0, sb>>>(c, nc, g->phi, g->mu + i * N, g->rho + i * N, L0.cx, L0.cy, L0.cz,
                                          L0.czlo, g->rhs, g->x, p->d_flag);
            coarsen_all(g, sb);
            e = pcg_capture(g, g->x, g->rhs, p->lin_tol, maxlin, p->d_flag, sb, sc);
            k_np_finish<<<G, 256, 0, sb>>>(N, (double)p->q[i], p->lambda_rho, p->rho_mix, 1.0 / p->rho_b[i], g->phi,
                                           g->mu + i * N, g->x, g->rho + i * N, g->lam ? g->lam + i * N : nullptr,
                                           g->prev ? g->prev + i * N : nullptr, g->dmax, p->d_flag);
        }
        if (g->phase) k_phase_mark<<<1, 1, 0, sb>>>(g->phase, 2);
        if (g->aa) {
            // Anderson extrapolation of the plain iterate (or a repeat of the
            // sweep from the last plain iterate after an unphysical one)
            k_aa_post<<<1, 1, 0, sb>>>(g->aa, g->dmax, p->d_flag, p->tol, g->stats);
            k_aa_restore<<<GM, 256, 0, sb>>>(g->aa, g->aa_X, g->aa_F, g->aa_xb, g->aa_fb, g->phi, g->rho, N, M);
            k_aa_record<<<NBM, 256, 0, sb>>>(g->aa, g->phi, g->rho, g->aa_X, g->aa_F, N, M, g->aa_part);
            k_aa_solve<<<1, 256, 0, sb>>>(g->aa, g->aa_part, NBM);
            k_aa_update<<<GM, 256, 0, sb>>>(g->aa, g->aa_X, g->aa_F, g->phi, g->rho, N, M);
        }
        // 5. residual, status, continue?
        k_gummel_check<<<1, 1, 0, sb>>>(g->dmax, p->d_flag, p->tol, p->max_iter, g->stats, hg, g->aa);
        if (g->phase) k_phase_mark<<<1, 1, 0, sb>>>(g->phase, 3);
        cudaError_t e2 = cudaStreamEndCapture(sb, &body);
        if (e == cudaSuccess) e = e2;
    }
    cudaError_t e3 = cudaStreamEndCapture(st, &top);
    if (e == cudaSuccess) e = e3;
    p->timer.enabled = timer;
    if (e == cudaSuccess && rc == PNP_OK) e = cudaGraphInstantiate(&g->exec, top, 0);
    if (e != cudaSuccess || rc != PNP_OK) {
        cudaGetLastError();
        if (top) cudaGraphDestroy(top);
        return rc != PNP_OK ? rc : cuda_status(e);
    }
    g->graph = top;
    return PNP_OK;
}

// Enqueue a whole solve on `st` (initial state, the solve graph, stats into
// g->stats) without waiting.  Builds the graph on first use.
int gummel_launch(Problem *p, const double *d_phi0, const double *d_rho0, cudaStream_t st) {
    NvtxRange range("gummel_launch");
    if (p->bc[2] != PNP_BC_DIRICHLET || p->bc[0] == PNP_BC_DIRICHLET || p->bc[1] == PNP_BC_DIRICHLET)
        return PNP_ERR_INVALID;
    int rc = gummel_setup(p);
    if (rc) return rc;
    rc = mu_ex_prepare(p, p->precision);
    if (rc) return rc;
    GummelState *g = p->gs;
    const size_t N = p->npts();
    const int s = p->s;
    const int G = grid_for(N);
    if (!g->exec) {
        // per-species integers and the fixed charge live as long as the graph
        int *d_q = nullptr;
        double *d_rhof = nullptr;
        cudaError_t e = dmalloc((void **)&d_q, sizeof(int) * s, p->stream);
        if (e == cudaSuccess) e = cudaMemcpy(d_q, p->q.data(), sizeof(int) * s, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !p->rho_f.empty()) {
            e = dmalloc((void **)&d_rhof, sizeof(double) * N, p->stream);
            if (e == cudaSuccess) e = cudaMemcpy(d_rhof, p->rho_f.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            dfree(d_q, p->stream);
            dfree(d_rhof, p->stream);
            return cuda_status(e);
        }
        g->keep_q = d_q;
        g->keep_rhof = d_rhof;
        rc = build_graph(p, d_q, d_rhof);
        if (rc) {
            dfree(g->keep_q, p->stream);
            dfree(g->keep_rhof, p->stream);
            g->keep_q = nullptr;
            g->keep_rhof = nullptr;
            return rc;
        }
    }
    PhysConst c{p->nx, p->ny, p->nz, p->bc[0], p->bc[1], p->lB, p->phi_lo, p->phi_hi};
    if (d_phi0) k_copy<<<G, 256, 0, st>>>(g->phi, d_phi0, N);
    else k_init_phi<<<G, 256, 0, st>>>(c, g->phi);
    if (d_rho0) {
        k_copy<<<G, 256, 0, st>>>(g->rho, d_rho0, N * s);
    } else {
        for (int i = 0; i < s; ++i) k_fill<<<G, 256, 0, st>>>(g->rho + i * N, p->rho_b[i], N);
    }
    if (g->lam) {
        k_fill<<<G, 256, 0, st>>>(g->lam, p->lambda_rho, N * s);
        k_fill<<<G, 256, 0, st>>>(g->prev, 0.0, N * s);
    }
    cudaMemsetAsync(p->d_flag, 0, sizeof(int), st);
    k_stats_reset<<<1, 1, 0, st>>>(g->stats, (p->eq_init && !d_phi0 && !d_rho0) ? 1 : 0);
    if (g->aa) k_aa_reset<<<1, 1, 0, st>>>(g->aa, p->aa_depth);
    if (g->phase) k_fill<<<1, 32, 0, st>>>(g->phase, 0.0, kPhases + 1);
    return cuda_status(cudaGraphLaunch(g->exec, st));
}

// Enqueue copies of the solve's state and record to caller buffers (device
// or pinned host, any direction the runtime infers).
int gummel_fetch(Problem *p, double *phi, double *rho, void *dev_stats_copy, cudaStream_t st) {
    GummelState *g = p->gs;
    const size_t N = p->npts();
    cudaError_t e = cudaSuccess;
    if (phi) e = cudaMemcpyAsync(phi, g->phi, sizeof(double) * N, cudaMemcpyDefault, st);
    if (rho && e == cudaSuccess) e = cudaMemcpyAsync(rho, g->rho, sizeof(double) * N * p->s, cudaMemcpyDefault, st);
    if (dev_stats_copy && e == cudaSuccess)
        e = cudaMemcpyAsync(dev_stats_copy, g->stats, sizeof(DevStats), cudaMemcpyDefault, st);
    return cuda_status(e);
}

int plane_flux(Problem *p, int i, const double *d_phi, const double *d_mu, const double *d_rho, double *d_flux,
               cudaStream_t st) {
    PhysConst c{p->nx, p->ny, p->nz, p->bc[0], p->bc[1], p->lB, p->phi_lo, p->phi_hi};
    NpConst nc;
    nc.D = p->D[i];
    nc.q = p->q[i];
    nc.Dlo = p->D[i] * std::exp(-(p->q[i] * p->phi_lo + p->mu_bulk[i]));
    nc.Dhi = p->D[i] * std::exp(-(p->q[i] * p->phi_hi + p->mu_bulk[i]));
    nc.rlo = p->rho_b[i] * std::exp(p->q[i] * p->phi_lo + p->mu_bulk[i]);
    nc.rhi = p->rho_b[i] * std::exp(p->q[i] * p->phi_hi + p->mu_bulk[i]);
    k_plane_flux<<<p->nz + 1, 256, 0, st>>>(c, nc, d_phi, d_mu, d_rho, d_flux);
    return cuda_status(cudaGetLastError());
}

size_t gummel_stats_bytes() { return sizeof(DevStats); }

int gummel_phase_times(Problem *p, double *ms, int max_phases) {
    GummelState *g = p->gs;
    if (!g || !g->phase || !ms || max_phases < 0) return PNP_ERR_INVALID;
    double h[kPhases];
    cudaError_t e = cudaMemcpyAsync(h, g->phase, sizeof(h), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int k = 0; k < kPhases && k < max_phases; ++k) ms[k] = h[k] * 1e-6;
    return kPhases;
}

void gummel_decode_stats(const void *raw, pnp_stats *out) {
    const DevStats *hs = (const DevStats *)raw;
    out->iterations = hs->iters;
    out->residual = hs->residual;
    out->linear_iterations = hs->lin;
    out->status = hs->status;
    out->init_iterations = hs->eq_iters;
    out->init_residual = hs->eq_residual;
    out->repeated_sweeps = hs->redos;
}

int gummel_run(Problem *p, const double *d_phi0, const double *d_rho0, double *d_phi, double *d_rho, pnp_stats *stats,
               cudaStream_t st) {
    int rc = gummel_launch(p, d_phi0, d_rho0, st);
    if (rc) return rc;
    DevStats hs;
    rc = gummel_fetch(p, d_phi, d_rho, &hs, st);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(p->d_flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    pnp_stats local{};
    gummel_decode_stats(&hs, &local);
    if (stats) {
        stats->iterations = local.iterations;
        stats->residual = local.residual;
        stats->linear_iterations = local.linear_iterations;
        stats->status = local.status;
        stats->init_iterations = local.init_iterations;
        stats->init_residual = local.init_residual;
        stats->repeated_sweeps = local.repeated_sweeps;
    }
    return local.status;
}

}  // namespace pnp
