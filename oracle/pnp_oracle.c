/*
 * pnp_oracle.c -- plain, slow, FP64 CPU oracle for the PNP-cDFT hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include, link
 * or call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * What it computes, in the paper's order (Meng, Zheng, Lin, Sushko,
 * "Numerical solution of 3D PNP equations coupled with cDFT", arXiv:1407.0674):
 *
 *   weighted densities  n_a(r) = sum_i int rho_i(r') w_i^a(r'-r) dr'      Sec 2.3.1
 *   Rosenfeld FMT derivatives dPhi/dn_a                                   Sec 2.3.1
 *   back-convolution  mu_hs,i(r) = sum_a int dPhi/dn_a(r') w_i^a(r-r') dr' Sec 2.3.1
 *   square-well mean field  mu_sh(r) = 1/2 int rho_s(r') Phi(|r-r'|) dr'  Sec 2.3.2
 *   delta-shell integrals by the (theta, phi) change of variables         Sec 3.5
 *   7-point harmonic-mean finite differences                              Sec 3.1
 *   relaxed Gummel iteration on the Slotboom form                         Sec 2.1, 3.2
 *   White Bear (MFMT) derivatives, series near n3 = 0                     Sec 2.3.1
 *   equilibrium cDFT initial guess (Poisson-Boltzmann Newton steps)       Sec 3.2.1
 *   screened Poisson step, per-point adaptive relaxation (options)        Sec 3.2
 *   Anderson-accelerated Gummel iteration with restart and step halving   Sec 3.2
 *     after an unphysical sweep (an extension)
 *   plane currents through the z faces                                    Sec 2.1, 3.1
 *   MSA electrostatic-correlation term (integral part)                    Sec 2.3.4
 *
 * Every function is pinned by a CPU test against closed forms, brute force,
 * independent library routines or invariants (see the tests named oracle_*).
 *
 * Every integral is evaluated as a DIRECT real-space sum over quadrature nodes
 * (no FFT).  The value at an off-grid node is trilinear in the 8 surrounding
 * grid values; grid values outside the domain are 0 on non-periodic axes
 * (zero extension, Sec 3.5) and wrap on periodic axes.
 *
 * Quadrature (Sec 3.5 leaves the rule open; this is the fixed reading):
 *   angular: theta_a = (a+1/2) 2 pi / n_theta (trapezoid), mu_b = cos(phi_b) at
 *            the n_mu Gauss-Legendre nodes on [-1,1]; weight (2 pi/n_theta) w_b
 *            (the R^2 sin(phi) dphi dtheta measure after mu = cos phi).
 *   shell of radius R: nodes R u, weights R^2 * angular weight.
 *   ball / thick shell [a,b]: radial Gauss-Legendre (n_r nodes) on [a,b] with
 *            the r^2 factor, times the angular rule.
 *   defaults: n_mu = max(8, ceil(2 pi R)), n_theta = 2 n_mu rounded up to a
 *            multiple of 4, n_r = max(4, ceil(2 (b - a))); for a thick shell
 *            the angular counts use its outer radius.
 * All lengths are in units of the grid spacing h; potentials in kT/e;
 * chemical potentials in kT.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1,1]: Newton iteration on P_n, evaluated by the
 * three-term recurrence (n+1)P_{n+1} = (2n+1) x P_n - n P_{n-1}.            */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            /* P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1) */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) {
                /* one more evaluation of the derivative at the final z */
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ------------------------------------------------------------------ */
/* Node sets (Sec 3.5).  kind 0: shell of radius r_out; kind 1: ball [0,r_out];
 * kind 2: thick shell [r_in, r_out].  Returns the node count.  With null
 * output pointers it only counts.                                        */
static int default_nmu(double r) { int n = (int)ceil(2.0 * M_PI * r); return n < 8 ? 8 : n; }
static int default_ntheta(int nmu) { int n = 2 * nmu; return (n + 3) / 4 * 4; }
static int default_nr(double len) { int n = (int)ceil(2.0 * len); return n < 4 ? 4 : n; }

int oracle_nodeset(int kind, double r_in, double r_out, int nmu, int ntheta, int nr,
                   double *px, double *py, double *pz, double *w,
                   double *ux, double *uy, double *uz)
{
    if (nmu <= 0) nmu = default_nmu(r_out);
    if (ntheta <= 0) ntheta = default_ntheta(nmu);
    double a = (kind == 1) ? 0.0 : r_in;
    if (kind == 0) nr = 1;
    else if (nr <= 0) nr = default_nr(r_out - a);
    int count = nmu * ntheta * nr;
    if (!px) return count;

    double *gx = malloc(sizeof(double) * nmu), *gw = malloc(sizeof(double) * nmu);
    double *rx = malloc(sizeof(double) * nr), *rw = malloc(sizeof(double) * nr);
    gauss_legendre(nmu, gx, gw);
    if (kind == 0) {
        rx[0] = r_out;
        rw[0] = r_out * r_out;           /* R^2 of the surface measure */
    } else {
        gauss_legendre(nr, rx, rw);
        for (int k = 0; k < nr; ++k) {   /* map [-1,1] -> [a, r_out], weight r^2 dr */
            double r = 0.5 * (r_out - a) * rx[k] + 0.5 * (r_out + a);
            rw[k] = 0.5 * (r_out - a) * rw[k] * r * r;
            rx[k] = r;
        }
    }
    int idx = 0;
    for (int k = 0; k < nr; ++k)
        for (int b = 0; b < nmu; ++b) {
            double mu = gx[b], sphi = sqrt(1.0 - mu * mu);
            for (int t = 0; t < ntheta; ++t) {
                double th = (t + 0.5) * 2.0 * M_PI / ntheta;
                double u0 = cos(th) * sphi, u1 = sin(th) * sphi, u2 = mu;
                px[idx] = rx[k] * u0;
                py[idx] = rx[k] * u1;
                pz[idx] = rx[k] * u2;
                w[idx] = rw[k] * (2.0 * M_PI / ntheta) * gw[b];
                if (ux) { ux[idx] = u0; uy[idx] = u1; uz[idx] = u2; }
                ++idx;
            }
        }
    free(gx); free(gw); free(rx); free(rw);
    return count;
}

/* ------------------------------------------------------------------ */
/* Grid with per-axis periodicity; fields are C order [z][y][x].         */
typedef struct {
    int n[3];          /* nx, ny, nz */
    int periodic[3];
} grid_t;

static inline double grid_value(const grid_t *g, const double *f, long ix, long iy, long iz)
{
    long idx[3] = {ix, iy, iz};
    for (int d = 0; d < 3; ++d) {
        long n = g->n[d];
        if (g->periodic[d]) {
            idx[d] %= n;
            if (idx[d] < 0) idx[d] += n;
        } else if (idx[d] < 0 || idx[d] >= n) {
            return 0.0;                   /* zero extension outside Omega */
        }
    }
    return f[(idx[2] * g->n[1] + idx[1]) * g->n[0] + idx[0]];
}

/* trilinear interpolation at the point (X, Y, Z) in grid-index units */
static double interp(const grid_t *g, const double *f, double X, double Y, double Z)
{
    double fx = floor(X), fy = floor(Y), fz = floor(Z);
    long i0 = (long)fx, j0 = (long)fy, k0 = (long)fz;
    double tx = X - fx, ty = Y - fy, tz = Z - fz;
    double v = 0.0;
    for (int c = 0; c < 8; ++c) {
        int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
        double wgt = (a ? tx : 1.0 - tx) * (b ? ty : 1.0 - ty) * (e ? tz : 1.0 - tz);
        if (wgt != 0.0) v += wgt * grid_value(g, f, i0 + a, j0 + b, k0 + e);
    }
    return v;
}

/* Test hook: instead of a grid field, evaluate rho_i(r) = amp_i cos(k.r + ph)
 * exactly at each node ("analytic" mode for the plane-wave pins).        */
typedef struct {
    int enabled;
    double k[3], phase;
    const double *amp;   /* per species */
} wave_t;

static double field_at(const grid_t *g, const double *f, const wave_t *wv, int sp,
                       double X, double Y, double Z)
{
    if (wv && wv->enabled)
        return wv->amp[sp] * cos(wv->k[0] * X + wv->k[1] * Y + wv->k[2] * Z + wv->phase);
    return interp(g, f, X, Y, Z);
}

/* ------------------------------------------------------------------ */
/* Problem description (oracle-private).                                 */
typedef struct {
    int nx, ny, nz;
    int bc[3];                 /* 0 periodic, 1 Dirichlet, 2 no-flux */
    int s;                     /* number of mobile species */
    const double *R;           /* hard-sphere radius per species (h) */
    const int *q;              /* valence */
    const double *rho_b;       /* bulk density (h^-3) */
    const double *D;           /* diffusion coefficient */
    const double *depth;       /* square-well depth eps_i (kT) */
    double well_inner, well_outer;   /* square-well shell radii (h) */
    int nsites;
    const double *sites;       /* 3*nsites, grid-index coordinates */
    double site_alpha;         /* Gaussian exponent (h^-2) */
    const double *rho_f;       /* fixed charge per cell (e h^-3) or NULL */
    double lB;                 /* Bjerrum length (h) */
    double phi_lo, phi_hi;     /* Dirichlet potentials on the z faces (kT/e) */
    double lambda_phi, lambda_rho, tol;
    int max_iter;
    int nmu, ntheta, nr;       /* FMT quadrature counts (0 = default rule) */
    int w_nmu, w_ntheta, w_nr; /* square-well quadrature counts */
    int sw_half;               /* 1: the 1/2 of Sec 2.3.2 kept; 0: dropped */
    double lin_tol;            /* PCG relative residual target */
    int lin_max_iter;
    int rho_mix;               /* 0: linear relaxation (Sec 3.2), 1: geometric,
                                  2: geometric with |step in ln rho| <= 0.2,
                                  3: 2 with a per-point factor: halved when the
                                     step changes sign, else grown 10% up to l2 */
    int screened;              /* Gummel Poisson step: 0 linear solve, 1 one Newton step
                                  with the densities' Boltzmann dependence on phi */
    int fmt;                   /* 0 Rosenfeld (Sec 2.3.1), 1 White Bear (MFMT) */
    int msa;                   /* 1: mu_ex also carries the MSA term of Sec 2.3.4 */
} oracle_problem;

static grid_t cdft_grid(const oracle_problem *p)
{
    grid_t g;
    g.n[0] = p->nx; g.n[1] = p->ny; g.n[2] = p->nz;
    for (int d = 0; d < 3; ++d) g.periodic[d] = (p->bc[d] == 0);
    return g;
}

typedef struct {
    int n;
    double *px, *py, *pz, *w, *ux, *uy, *uz;
} nodes_t;

static nodes_t make_nodes(int kind, double r_in, double r_out, int nmu, int ntheta, int nr)
{
    nodes_t t;
    t.n = oracle_nodeset(kind, r_in, r_out, nmu, ntheta, nr, 0, 0, 0, 0, 0, 0, 0);
    t.px = malloc(sizeof(double) * t.n * 7);
    t.py = t.px + t.n; t.pz = t.py + t.n; t.w = t.pz + t.n;
    t.ux = t.w + t.n; t.uy = t.ux + t.n; t.uz = t.uy + t.n;
    oracle_nodeset(kind, r_in, r_out, nmu, ntheta, nr, t.px, t.py, t.pz, t.w, t.ux, t.uy, t.uz);
    return t;
}
static void free_nodes(nodes_t *t) { free(t->px); }

/* ------------------------------------------------------------------ */
/* Weighted densities, Sec 2.3.1:
 *   n_a(r) = sum_i int_Omega rho_i(r') w_i^a(r' - r) dr'
 * with w3 the ball indicator, w2 = delta(|r|-R), vec w2 = (r/|r|) delta,
 * w0 = w2/(4 pi R^2), w1 = w2/(4 pi R), vec w1 = vec w2/(4 pi R).
 * Output layout: n[a*N + p], a = n0,n1,n2,n3,n1x,n1y,n1z,n2x,n2y,n2z.   */
void oracle_weighted_densities(const oracle_problem *p, const double *rho, double *n,
                               const double *wave_k, double wave_phase, const double *wave_amp)
{
    grid_t g = cdft_grid(p);
    long N = (long)p->nx * p->ny * p->nz;
    wave_t wv = {0};
    if (wave_k) {
        wv.enabled = 1;
        wv.k[0] = wave_k[0]; wv.k[1] = wave_k[1]; wv.k[2] = wave_k[2];
        wv.phase = wave_phase;
        wv.amp = wave_amp;
    }
    memset(n, 0, sizeof(double) * 10 * N);
    for (int i = 0; i < p->s; ++i) {
        double R = p->R[i];
        nodes_t sh = make_nodes(0, 0.0, R, p->nmu, p->ntheta, p->nr);
        nodes_t ba = make_nodes(1, 0.0, R, p->nmu, p->ntheta, p->nr);
        const double *rho_i = rho ? rho + i * N : 0;
        double c0 = 1.0 / (4.0 * M_PI * R * R), c1 = 1.0 / (4.0 * M_PI * R);
#pragma omp parallel for schedule(static)
        for (long pt = 0; pt < N; ++pt) {
            double X = (double)(pt % p->nx);
            double Y = (double)((pt / p->nx) % p->ny);
            double Z = (double)(pt / ((long)p->nx * p->ny));
            double n2 = 0, v2x = 0, v2y = 0, v2z = 0, n3 = 0;
            for (int q = 0; q < sh.n; ++q) {
                double v = field_at(&g, rho_i, &wv, i, X + sh.px[q], Y + sh.py[q], Z + sh.pz[q]);
                n2 += sh.w[q] * v;
                v2x += sh.w[q] * sh.ux[q] * v;
                v2y += sh.w[q] * sh.uy[q] * v;
                v2z += sh.w[q] * sh.uz[q] * v;
            }
            for (int q = 0; q < ba.n; ++q)
                n3 += ba.w[q] * field_at(&g, rho_i, &wv, i, X + ba.px[q], Y + ba.py[q], Z + ba.pz[q]);
            n[0 * N + pt] += c0 * n2;
            n[1 * N + pt] += c1 * n2;
            n[2 * N + pt] += n2;
            n[3 * N + pt] += n3;
            n[4 * N + pt] += c1 * v2x;
            n[5 * N + pt] += c1 * v2y;
            n[6 * N + pt] += c1 * v2z;
            n[7 * N + pt] += v2x;
            n[8 * N + pt] += v2y;
            n[9 * N + pt] += v2z;
        }
        free_nodes(&sh);
        free_nodes(&ba);
    }
}

/* Rosenfeld FMT free-energy density Phi (Sec 2.3.1) at one point.        */
static double phi_rosenfeld(const double *a)
{
    double n0 = a[0], n1 = a[1], n2 = a[2], n3 = a[3];
    double v1v2 = a[4] * a[7] + a[5] * a[8] + a[6] * a[9];
    double v2v2 = a[7] * a[7] + a[8] * a[8] + a[9] * a[9];
    double o = 1.0 - n3;
    return -n0 * log(o) + n1 * n2 / o + n2 * n2 * n2 / (24.0 * M_PI * o * o)
           - v1v2 / o - n2 * v2v2 / (8.0 * M_PI * o * o);
}

/* The ten partial derivatives printed in Sec 2.3.1.  Returns the number of
 * points where n3 >= 1 or a value is not finite (packing error).         */
long oracle_dphi(long N, const double *n, double *psi)
{
    long bad = 0;
    for (long pt = 0; pt < N; ++pt) {
        double n0 = n[0 * N + pt], n1 = n[1 * N + pt], n2 = n[2 * N + pt], n3 = n[3 * N + pt];
        double v1[3] = {n[4 * N + pt], n[5 * N + pt], n[6 * N + pt]};
        double v2[3] = {n[7 * N + pt], n[8 * N + pt], n[9 * N + pt]};
        int flagged = !(n3 < 1.0);
        double o = 1.0 - n3;
        double v1v2 = v1[0] * v2[0] + v1[1] * v2[1] + v1[2] * v2[2];
        double v2v2 = v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2];
        psi[0 * N + pt] = -log(1.0 - n3);
        psi[1 * N + pt] = n2 / (1.0 - n3);
        psi[2 * N + pt] = n1 / (1.0 - n3) + (n2 * n2 - v2v2) / (8.0 * M_PI * o * o);
        psi[3 * N + pt] = n0 / (1.0 - n3) + (n1 * n2 - v1v2) / (o * o)
                          + (n2 * n2 * n2 - 3.0 * n2 * v2v2) / (12.0 * M_PI * o * o * o);
        for (int c = 0; c < 3; ++c) {
            psi[(4 + c) * N + pt] = v2[c] / (n3 - 1.0);
            psi[(7 + c) * N + pt] = v1[c] / (n3 - 1.0) - n2 * v2[c] / (4.0 * M_PI * o * o);
        }
        for (int a = 0; a < 10; ++a)
            if (!isfinite(psi[a * N + pt])) flagged = 1;
        bad += flagged;
    }
    return bad;
}

/* White Bear (modified FMT) version of Phi, the variant Sec 2.3.1 names
 * beside Rosenfeld's: the n2^3 term carries
 *   phi3(x) = [x + (1-x)^2 ln(1-x)] / [x^2 (1-x)^2] / (36 pi)
 * instead of 1/(24 pi (1-x)^2).  phi3 and its derivative are taken from the
 * closed form for |x| >= 0.05 and from their power series
 * phi3(x) = sum_k (k+1)(k+3)/(k+2) x^k below (the closed form cancels as
 * x -> 0, and x = 0 off the domain); 25 terms leave < 1e-29.              */
static void wb_phi3(double x, double *f, double *df)
{
    if (fabs(x) < 0.05) {
        double v = 0.0, d = 0.0;
        for (int k = 24; k >= 0; --k) v = v * x + (double)(k + 1) * (k + 3) / (k + 2);
        for (int k = 24; k >= 1; --k) d = d * x + (double)k * (k + 1) * (k + 3) / (k + 2);
        *f = v;
        *df = d;
        return;
    }
    double o = 1.0 - x, L = log(o);
    double num = x + o * o * L, den = x * x * o * o;
    double dnum = x - 2.0 * o * L, dden = 2.0 * x * o * (1.0 - 2.0 * x);
    *f = num / den;
    *df = (dnum * den - num * dden) / (den * den);
}

static double phi_white_bear(const double *a)
{
    double n0 = a[0], n1 = a[1], n2 = a[2], n3 = a[3];
    double v1v2 = a[4] * a[7] + a[5] * a[8] + a[6] * a[9];
    double v2v2 = a[7] * a[7] + a[8] * a[8] + a[9] * a[9];
    double o = 1.0 - n3, f, df;
    wb_phi3(n3, &f, &df);
    return -n0 * log(o) + (n1 * n2 - v1v2) / o + (n2 * n2 * n2 - 3.0 * n2 * v2v2) * f / (36.0 * M_PI);
}

/* The ten partial derivatives of the White Bear Phi (same order as
 * oracle_dphi).  Returns the number of points with a packing error.      */
long oracle_dphi_wb(long N, const double *n, double *psi)
{
    long bad = 0;
    for (long pt = 0; pt < N; ++pt) {
        double n0 = n[0 * N + pt], n1 = n[1 * N + pt], n2 = n[2 * N + pt], n3 = n[3 * N + pt];
        double v1[3] = {n[4 * N + pt], n[5 * N + pt], n[6 * N + pt]};
        double v2[3] = {n[7 * N + pt], n[8 * N + pt], n[9 * N + pt]};
        int flagged = !(n3 < 1.0);
        double o = 1.0 - n3, f = 0.0, df = 0.0;
        if (!flagged) wb_phi3(n3, &f, &df);
        double v1v2 = v1[0] * v2[0] + v1[1] * v2[1] + v1[2] * v2[2];
        double v2v2 = v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2];
        psi[0 * N + pt] = -log(o);
        psi[1 * N + pt] = n2 / o;
        psi[2 * N + pt] = n1 / o + (n2 * n2 - v2v2) * f / (12.0 * M_PI);
        psi[3 * N + pt] = n0 / o + (n1 * n2 - v1v2) / (o * o)
                          + (n2 * n2 * n2 - 3.0 * n2 * v2v2) * df / (36.0 * M_PI);
        for (int c = 0; c < 3; ++c) {
            psi[(4 + c) * N + pt] = -v2[c] / o;
            psi[(7 + c) * N + pt] = -v1[c] / o - n2 * v2[c] * f / (6.0 * M_PI);
        }
        for (int a = 0; a < 10; ++a)
            if (!isfinite(psi[a * N + pt])) flagged = 1;
        bad += flagged;
    }
    return bad;
}

long oracle_dphi_fmt(int fmt, long N, const double *n, double *psi)
{
    return fmt == 1 ? oracle_dphi_wb(N, n, psi) : oracle_dphi(N, n, psi);
}

double oracle_fhs_fmt(int fmt, long N, const double *n)
{
    double F = 0.0;
    double a[10];
    for (long pt = 0; pt < N; ++pt) {
        for (int k = 0; k < 10; ++k) a[k] = n[k * N + pt];
        F += fmt == 1 ? phi_white_bear(a) : phi_rosenfeld(a);
    }
    return F;
}

/* Free energy h^3 sum_Omega Phi(n) (h = 1); used by the adjoint checks.   */
double oracle_fhs(long N, const double *n)
{
    double F = 0.0;
    double a[10];
    for (long pt = 0; pt < N; ++pt) {
        for (int k = 0; k < 10; ++k) a[k] = n[k * N + pt];
        F += phi_rosenfeld(a);
    }
    return F;
}

/* Back-convolution, Sec 2.3.1:
 *   mu_hs,i(r) = sum_a int_Omega dPhi/dn_a(r') w_i^a(r - r') dr'
 * psi is zero off Omega (zero extension).  Output mu[i*N + p].           */
void oracle_mu_hs(const oracle_problem *p, const double *psi, double *mu)
{
    grid_t g = cdft_grid(p);
    long N = (long)p->nx * p->ny * p->nz;
    for (int i = 0; i < p->s; ++i) {
        double R = p->R[i];
        nodes_t sh = make_nodes(0, 0.0, R, p->nmu, p->ntheta, p->nr);
        nodes_t ba = make_nodes(1, 0.0, R, p->nmu, p->ntheta, p->nr);
        double c0 = 1.0 / (4.0 * M_PI * R * R), c1 = 1.0 / (4.0 * M_PI * R);
#pragma omp parallel for schedule(static)
        for (long pt = 0; pt < N; ++pt) {
            double X = (double)(pt % p->nx);
            double Y = (double)((pt / p->nx) % p->ny);
            double Z = (double)(pt / ((long)p->nx * p->ny));
            double acc = 0.0;
            for (int q = 0; q < sh.n; ++q) {
                double x = X - sh.px[q], y = Y - sh.py[q], z = Z - sh.pz[q];
                double s0 = interp(&g, psi + 0 * N, x, y, z);
                double s1 = interp(&g, psi + 1 * N, x, y, z);
                double s2 = interp(&g, psi + 2 * N, x, y, z);
                double v1x = interp(&g, psi + 4 * N, x, y, z);
                double v1y = interp(&g, psi + 5 * N, x, y, z);
                double v1z = interp(&g, psi + 6 * N, x, y, z);
                double v2x = interp(&g, psi + 7 * N, x, y, z);
                double v2y = interp(&g, psi + 8 * N, x, y, z);
                double v2z = interp(&g, psi + 9 * N, x, y, z);
                double scal = c0 * s0 + c1 * s1 + s2;
                double vec = sh.ux[q] * (c1 * v1x + v2x) + sh.uy[q] * (c1 * v1y + v2y)
                             + sh.uz[q] * (c1 * v1z + v2z);
                acc += sh.w[q] * (scal + vec);
            }
            for (int q = 0; q < ba.n; ++q)
                acc += ba.w[q] * interp(&g, psi + 3 * N, X - ba.px[q], Y - ba.py[q], Z - ba.pz[q]);
            mu[i * N + pt] = acc;
        }
        free_nodes(&sh);
        free_nodes(&ba);
    }
}

/* Stationary-site density, Sec 2.3.2: normalised Gaussians at the sites,
 * evaluated exactly at grid nodes.  On periodic axes the sites repeat with the
 * box, so every image whose Gaussian does not underflow (alpha d^2 < 800) is
 * summed.                                                                  */
void oracle_site_density(const oracle_problem *p, double *rho_s)
{
    long N = (long)p->nx * p->ny * p->nz;
    int n[3] = {p->nx, p->ny, p->nz};
    double a = p->site_alpha;
    double norm = pow(a / M_PI, 1.5);
    double reach = sqrt(800.0 / a);
    int m[3];
    for (int d = 0; d < 3; ++d) m[d] = (p->bc[d] == 0) ? (int)ceil(reach / n[d]) + 1 : 0;
#pragma omp parallel for schedule(static)
    for (long pt = 0; pt < N; ++pt) {
        double r[3] = {(double)(pt % p->nx), (double)((pt / p->nx) % p->ny),
                       (double)(pt / ((long)p->nx * p->ny))};
        double acc = 0.0;
        for (int k = 0; k < p->nsites; ++k)
            for (int iz = -m[2]; iz <= m[2]; ++iz)
                for (int iy = -m[1]; iy <= m[1]; ++iy)
                    for (int ix = -m[0]; ix <= m[0]; ++ix) {
                        double dx = r[0] - p->sites[3 * k + 0] - (double)ix * n[0];
                        double dy = r[1] - p->sites[3 * k + 1] - (double)iy * n[1];
                        double dz = r[2] - p->sites[3 * k + 2] - (double)iz * n[2];
                        acc += exp(-a * (dx * dx + dy * dy + dz * dz));
                    }
        rho_s[pt] = norm * acc;
    }
}

/* Square-well chemical potential, Sec 2.3.2:
 *   mu_sh,i(r) = 1/2 int rho_s(r') Phi_is(|r - r'|) dr',
 * Phi_is = -eps_i on the shell well_inner <= |r-r'| <= well_outer and 0
 * beyond; the hard core is FMT's.  Output mu_sh[i*N + p].                */
void oracle_mu_sh(const oracle_problem *p, const double *rho_s, double *mu_sh)
{
    grid_t g = cdft_grid(p);
    long N = (long)p->nx * p->ny * p->nz;
    double half = p->sw_half ? 0.5 : 1.0;
    nodes_t ws = make_nodes(2, p->well_inner, p->well_outer, p->w_nmu, p->w_ntheta, p->w_nr);
    for (int i = 0; i < p->s; ++i) {
        double eps = p->depth ? p->depth[i] : 0.0;
        if (eps == 0.0 || p->nsites == 0) {
            memset(mu_sh + i * N, 0, sizeof(double) * N);
            continue;
        }
#pragma omp parallel for schedule(static)
        for (long pt = 0; pt < N; ++pt) {
            double X = (double)(pt % p->nx);
            double Y = (double)((pt / p->nx) % p->ny);
            double Z = (double)(pt / ((long)p->nx * p->ny));
            double acc = 0.0;
            for (int q = 0; q < ws.n; ++q)
                acc += ws.w[q] * interp(&g, rho_s, X + ws.px[q], Y + ws.py[q], Z + ws.pz[q]);
            mu_sh[i * N + pt] = half * (-eps) * acc;
        }
    }
    free_nodes(&ws);
}

/* Electrostatic correlations in the mean spherical approximation, Sec 2.3.4
 * (the second-order direct correlation function of the MSA):
 *   mu_el,i(r) = mu_el,i^bulk - sum_j int_Omega C_ij(|r - r'|) (rho_j(r') - rho_b,j) dr',
 *   C_ij(r) = -q_i q_j l_B [2B/s - (B/s)^2 r - 1/r] for r <= s, 0 beyond,
 *   s = (sigma_i + sigma_j)/2 = R_i + R_j,  B = [xi + 1 - sqrt(1 + 2 xi)] / xi,
 *   xi = kappa s,  kappa^2 = 4 pi l_B sum_k rho_b,k q_k^2.
 * The printed prefactor e^2/(k_B T eps) is read as l_B: its -1/r term is then
 * exactly minus the Coulomb kernel inside the core, which the MSA correction
 * replaces.  The bulk constant mu_el^bulk is not printed and is left out: a
 * constant shift of mu_i and of the reservoir value alike cancels in the
 * Slotboom form.  The integral is the ball quadrature of radius s (the FMT
 * counts nmu, ntheta, nr), with rho_j - rho_b,j interpolated trilinearly from
 * the grid and zero off Omega.  With wave_k set the difference field is
 * instead amp_j cos(k.r + phase) evaluated at the nodes (plane-wave pins).
 * For xi below 1e-3 B is taken as 2 xi / (1 + sqrt(1 + 2 xi))^2, the same
 * number without the cancellation.  Output mu_el[i*N + p].                  */
void oracle_mu_el(const oracle_problem *p, const double *rho, double *mu_el,
                  const double *wave_k, double wave_phase, const double *wave_amp)
{
    grid_t g = cdft_grid(p);
    long N = (long)p->nx * p->ny * p->nz;
    wave_t wv = {0};
    if (wave_k) {
        wv.enabled = 1;
        wv.k[0] = wave_k[0]; wv.k[1] = wave_k[1]; wv.k[2] = wave_k[2];
        wv.phase = wave_phase;
        wv.amp = wave_amp;
    }
    double kappa2 = 0.0;
    for (int k = 0; k < p->s; ++k) kappa2 += 4.0 * M_PI * p->lB * p->rho_b[k] * p->q[k] * p->q[k];
    double kappa = sqrt(kappa2);
    double *drho = malloc(sizeof(double) * (wave_k ? 1 : N));
    memset(mu_el, 0, sizeof(double) * p->s * N);
    for (int j = 0; j < p->s; ++j) {
        if (!wave_k)
            for (long k = 0; k < N; ++k) drho[k] = rho[j * N + k] - p->rho_b[j];
        for (int i = 0; i < p->s; ++i) {
            double qq = (double)p->q[i] * p->q[j];
            if (qq == 0.0) continue;
            double sg = p->R[i] + p->R[j];
            double xi = kappa * sg, B;
            if (xi < 1e-3) B = 2.0 * xi / ((1.0 + sqrt(1.0 + 2.0 * xi)) * (1.0 + sqrt(1.0 + 2.0 * xi)));
            else B = (xi + 1.0 - sqrt(1.0 + 2.0 * xi)) / xi;
            nodes_t ba = make_nodes(1, 0.0, sg, p->nmu, p->ntheta, p->nr);
            double *cw = malloc(sizeof(double) * ba.n);
            for (int q = 0; q < ba.n; ++q) {
                double r = sqrt(ba.px[q] * ba.px[q] + ba.py[q] * ba.py[q] + ba.pz[q] * ba.pz[q]);
                double C = -qq * p->lB * (2.0 * B / sg - (B / sg) * (B / sg) * r - 1.0 / r);
                cw[q] = ba.w[q] * C;
            }
#pragma omp parallel for schedule(static)
            for (long pt = 0; pt < N; ++pt) {
                double X = (double)(pt % p->nx);
                double Y = (double)((pt / p->nx) % p->ny);
                double Z = (double)(pt / ((long)p->nx * p->ny));
                double acc = 0.0;
                for (int q = 0; q < ba.n; ++q)
                    acc += cw[q] * field_at(&g, drho, &wv, j, X + ba.px[q], Y + ba.py[q], Z + ba.pz[q]);
                mu_el[i * N + pt] -= acc;
            }
            free(cw);
            free_nodes(&ba);
        }
    }
    free(drho);
}

/* mu_ex,i = mu_hs,i + mu_sh,i (Sec 2.3), plus mu_el,i (Sec 2.3.4) when the
 * problem asks for it.  Returns the packing-error count. */
long oracle_excess_mu(const oracle_problem *p, const double *rho, double *mu)
{
    long N = (long)p->nx * p->ny * p->nz;
    double *n = malloc(sizeof(double) * 10 * N);
    double *psi = malloc(sizeof(double) * 10 * N);
    double *rs = malloc(sizeof(double) * N);
    double *msh = malloc(sizeof(double) * p->s * N);
    oracle_weighted_densities(p, rho, n, 0, 0.0, 0);
    long bad = oracle_dphi_fmt(p->fmt, N, n, psi);
    oracle_mu_hs(p, psi, mu);
    oracle_site_density(p, rs);
    oracle_mu_sh(p, rs, msh);
    for (long k = 0; k < p->s * N; ++k) mu[k] += msh[k];
    if (p->msa) {
        oracle_mu_el(p, rho, msh, 0, 0.0, 0);
        for (long k = 0; k < p->s * N; ++k) mu[k] += msh[k];
    }
    free(n); free(psi); free(rs); free(msh);
    return bad;
}

/* mu_ex at selected grid points only (for checks of large grids): the
 * weighted densities and derivatives are evaluated on the union of the boxes
 * of half-width S around each sample (every point the back-convolution at the
 * sample reads), then the same sums as oracle_excess_mu at the samples.
 * out[i*nsamp + k] for species i and sample k.                              */
void oracle_excess_mu_sampled(const oracle_problem *p, const double *rho, int nsamp, const long *idx,
                              double *out)
{
    grid_t g = cdft_grid(p);
    long N = (long)p->nx * p->ny * p->nz;
    int n3d[3] = {p->nx, p->ny, p->nz};
    double Rmax = 0.0;
    for (int i = 0; i < p->s; ++i) if (p->R[i] > Rmax) Rmax = p->R[i];
    int S = (int)ceil(Rmax) + 1;
    double Rw = p->well_outer;
    int Sw = (int)ceil(Rw) + 1;
    char *mask = calloc(N, 1);
    for (int k = 0; k < nsamp; ++k) {
        long c[3] = {idx[k] % p->nx, (idx[k] / p->nx) % p->ny, idx[k] / ((long)p->nx * p->ny)};
        for (int dz = -S; dz <= S; ++dz)
            for (int dy = -S; dy <= S; ++dy)
                for (int dx = -S; dx <= S; ++dx) {
                    long q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                    int ok = 1;
                    for (int d = 0; d < 3; ++d) {
                        if (g.periodic[d]) q[d] = ((q[d] % n3d[d]) + n3d[d]) % n3d[d];
                        else if (q[d] < 0 || q[d] >= n3d[d]) ok = 0;
                    }
                    if (ok) mask[(q[2] * p->ny + q[1]) * p->nx + q[0]] = 1;
                }
    }
    double *n = calloc(10 * N, sizeof(double));
    double *psi = calloc(10 * N, sizeof(double));
    for (int i = 0; i < p->s; ++i) {
        double R = p->R[i];
        nodes_t sh = make_nodes(0, 0.0, R, p->nmu, p->ntheta, p->nr);
        nodes_t ba = make_nodes(1, 0.0, R, p->nmu, p->ntheta, p->nr);
        const double *rho_i = rho + i * N;
        double c0 = 1.0 / (4.0 * M_PI * R * R), c1 = 1.0 / (4.0 * M_PI * R);
#pragma omp parallel for schedule(dynamic, 64)
        for (long pt = 0; pt < N; ++pt) {
            if (!mask[pt]) continue;
            double X = (double)(pt % p->nx), Y = (double)((pt / p->nx) % p->ny);
            double Z = (double)(pt / ((long)p->nx * p->ny));
            double n2 = 0, v2x = 0, v2y = 0, v2z = 0, n3 = 0;
            for (int q = 0; q < sh.n; ++q) {
                double v = interp(&g, rho_i, X + sh.px[q], Y + sh.py[q], Z + sh.pz[q]);
                n2 += sh.w[q] * v;
                v2x += sh.w[q] * sh.ux[q] * v;
                v2y += sh.w[q] * sh.uy[q] * v;
                v2z += sh.w[q] * sh.uz[q] * v;
            }
            for (int q = 0; q < ba.n; ++q)
                n3 += ba.w[q] * interp(&g, rho_i, X + ba.px[q], Y + ba.py[q], Z + ba.pz[q]);
            n[0 * N + pt] += c0 * n2; n[1 * N + pt] += c1 * n2; n[2 * N + pt] += n2; n[3 * N + pt] += n3;
            n[4 * N + pt] += c1 * v2x; n[5 * N + pt] += c1 * v2y; n[6 * N + pt] += c1 * v2z;
            n[7 * N + pt] += v2x; n[8 * N + pt] += v2y; n[9 * N + pt] += v2z;
        }
        free_nodes(&sh);
        free_nodes(&ba);
    }
    /* derivatives at the masked points (zero elsewhere, as off Omega) */
    double a[10], b[10];
    for (long pt = 0; pt < N; ++pt) {
        if (!mask[pt]) continue;
        for (int k = 0; k < 10; ++k) a[k] = n[k * N + pt];
        oracle_dphi_fmt(p->fmt, 1, a, b);
        for (int k = 0; k < 10; ++k) psi[k * N + pt] = b[k];
    }
    double *rs = 0;
    nodes_t ws = {0};
    if (p->nsites > 0 && p->depth) {
        /* site density on the union of boxes of half-width Sw around samples */
        char *mw = calloc(N, 1);
        for (int k = 0; k < nsamp; ++k) {
            long c[3] = {idx[k] % p->nx, (idx[k] / p->nx) % p->ny, idx[k] / ((long)p->nx * p->ny)};
            for (int dz = -Sw; dz <= Sw; ++dz)
                for (int dy = -Sw; dy <= Sw; ++dy)
                    for (int dx = -Sw; dx <= Sw; ++dx) {
                        long q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                        int ok = 1;
                        for (int d = 0; d < 3; ++d) {
                            if (g.periodic[d]) q[d] = ((q[d] % n3d[d]) + n3d[d]) % n3d[d];
                            else if (q[d] < 0 || q[d] >= n3d[d]) ok = 0;
                        }
                        if (ok) mw[(q[2] * p->ny + q[1]) * p->nx + q[0]] = 1;
                    }
        }
        double *full = malloc(sizeof(double) * N);
        oracle_site_density(p, full);   /* exact at every node */
        rs = calloc(N, sizeof(double));
        for (long pt = 0; pt < N; ++pt) if (mw[pt]) rs[pt] = full[pt];
        free(full);
        free(mw);
        ws = make_nodes(2, p->well_inner, p->well_outer, p->w_nmu, p->w_ntheta, p->w_nr);
    }
    double half = p->sw_half ? 0.5 : 1.0;
    for (int i = 0; i < p->s; ++i) {
        double R = p->R[i];
        nodes_t sh = make_nodes(0, 0.0, R, p->nmu, p->ntheta, p->nr);
        nodes_t ba = make_nodes(1, 0.0, R, p->nmu, p->ntheta, p->nr);
        double c0 = 1.0 / (4.0 * M_PI * R * R), c1 = 1.0 / (4.0 * M_PI * R);
        double eps = p->depth ? p->depth[i] : 0.0;
        for (int k = 0; k < nsamp; ++k) {
            long pt = idx[k];
            double X = (double)(pt % p->nx), Y = (double)((pt / p->nx) % p->ny);
            double Z = (double)(pt / ((long)p->nx * p->ny));
            double acc = 0.0;
            for (int q = 0; q < sh.n; ++q) {
                double x = X - sh.px[q], y = Y - sh.py[q], z = Z - sh.pz[q];
                double scal = c0 * interp(&g, psi + 0 * N, x, y, z) + c1 * interp(&g, psi + 1 * N, x, y, z)
                              + interp(&g, psi + 2 * N, x, y, z);
                double vec = sh.ux[q] * (c1 * interp(&g, psi + 4 * N, x, y, z) + interp(&g, psi + 7 * N, x, y, z))
                             + sh.uy[q] * (c1 * interp(&g, psi + 5 * N, x, y, z) + interp(&g, psi + 8 * N, x, y, z))
                             + sh.uz[q] * (c1 * interp(&g, psi + 6 * N, x, y, z) + interp(&g, psi + 9 * N, x, y, z));
                acc += sh.w[q] * (scal + vec);
            }
            for (int q = 0; q < ba.n; ++q)
                acc += ba.w[q] * interp(&g, psi + 3 * N, X - ba.px[q], Y - ba.py[q], Z - ba.pz[q]);
            if (rs && eps != 0.0) {
                double a2 = 0.0;
                for (int q = 0; q < ws.n; ++q)
                    a2 += ws.w[q] * interp(&g, rs, X + ws.px[q], Y + ws.py[q], Z + ws.pz[q]);
                acc += half * (-eps) * a2;
            }
            out[i * nsamp + k] = acc;
        }
        free_nodes(&sh);
        free_nodes(&ba);
    }
    if (rs) { free(rs); free_nodes(&ws); }
    free(mask); free(n); free(psi);
}

/* Bulk mu_ex of the uniform reservoir: dPhi/dn_a at the bulk weighted
 * densities times the weight integrals (1, R, 4 pi R^2, 4 pi R^3 / 3).    */
void oracle_bulk_mu_fmt(int fmt, int s, const double *R, const double *rho_b, double *mu_b)
{
    double a[10] = {0}, psi[10];
    for (int i = 0; i < s; ++i) {
        a[0] += rho_b[i];
        a[1] += rho_b[i] * R[i];
        a[2] += rho_b[i] * 4.0 * M_PI * R[i] * R[i];
        a[3] += rho_b[i] * 4.0 * M_PI * R[i] * R[i] * R[i] / 3.0;
    }
    oracle_dphi_fmt(fmt, 1, a, psi);
    for (int i = 0; i < s; ++i)
        mu_b[i] = psi[0] + R[i] * psi[1] + 4.0 * M_PI * R[i] * R[i] * psi[2]
                  + 4.0 * M_PI * R[i] * R[i] * R[i] / 3.0 * psi[3];
}

void oracle_bulk_mu(int s, const double *R, const double *rho_b, double *mu_b)
{
    oracle_bulk_mu_fmt(0, s, R, rho_b, mu_b);
}

/* ------------------------------------------------------------------ */
/* 7-point finite-difference operators (Sec 3.1).  Unknowns sit on planes
 * k = 0..nz-1; the Dirichlet planes k = -1 and k = nz carry the boundary
 * values.  x and y are periodic (bc 0) or no-flux (bc 2).
 * The operator is  (A u)_p = sum_faces c_f (u_p - u_nbr)  with the Dirichlet
 * neighbour values moved to the right-hand side.  Face coefficients:
 *   cx[p] = face between p and its +x neighbour (0 across a no-flux wall),
 *   cy[p], cz[p] likewise; cz_lo[p] for plane 0 and the lower Dirichlet
 *   plane, cz[p] for the top plane is the face to the upper Dirichlet plane. */
typedef struct {
    int nx, ny, nz, bcx, bcy;
    double *cx, *cy, *cz, *czlo;
} fdop_t;

static long nbr(const fdop_t *A, long p, int axis, int dir, int *ok)
{
    int i = (int)(p % A->nx), j = (int)((p / A->nx) % A->ny), k = (int)(p / ((long)A->nx * A->ny));
    int n = axis == 0 ? A->nx : (axis == 1 ? A->ny : A->nz);
    int c = axis == 0 ? i : (axis == 1 ? j : k);
    int bc = axis == 0 ? A->bcx : (axis == 1 ? A->bcy : 1);
    c += dir;
    *ok = 1;
    if (c < 0 || c >= n) {
        if (bc == 0) c = (c + n) % n;
        else { *ok = 0; return -1; }
    }
    if (axis == 0) i = c; else if (axis == 1) j = c; else k = c;
    return ((long)k * A->ny + j) * A->nx + i;
}

/* coefficient of the face between p and its neighbour in (axis, dir) */
static double face(const fdop_t *A, long p, int axis, int dir)
{
    int ok;
    if (axis == 2) {
        int k = (int)(p / ((long)A->nx * A->ny));
        if (dir < 0) return k == 0 ? A->czlo[p] : A->cz[nbr(A, p, 2, -1, &ok)];
        return A->cz[p];
    }
    double *c = axis == 0 ? A->cx : A->cy;
    if (dir > 0) return c[p];
    long q = nbr(A, p, axis, -1, &ok);
    return ok ? c[q] : 0.0;
}

static void fd_apply(const fdop_t *A, const double *u, double *out)
{
    long N = (long)A->nx * A->ny * A->nz;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        double acc = 0.0;
        for (int axis = 0; axis < 3; ++axis)
            for (int dir = -1; dir <= 1; dir += 2) {
                double c = face(A, p, axis, dir);
                if (c == 0.0) continue;
                int ok;
                long q = nbr(A, p, axis, dir, &ok);
                acc += c * (u[p] - (ok ? u[q] : 0.0));
            }
        out[p] = acc;
    }
}

static void fd_diag(const fdop_t *A, double *dg)
{
    long N = (long)A->nx * A->ny * A->nz;
    for (long p = 0; p < N; ++p) {
        double acc = 0.0;
        for (int axis = 0; axis < 3; ++axis)
            for (int dir = -1; dir <= 1; dir += 2) acc += face(A, p, axis, dir);
        dg[p] = acc;
    }
}

static double dot(long N, const double *a, const double *b)
{
    double s = 0.0;
    for (long k = 0; k < N; ++k) s += a[k] * b[k];
    return s;
}

/* Jacobi-preconditioned conjugate gradients; x holds the initial guess on
 * entry.  Stops at ||r||_2 <= tol ||b||_2.  Returns the iteration count.  */
static int pcg(const fdop_t *A, const double *b, double *x, double tol, int maxit, double *relres)
{
    long N = (long)A->nx * A->ny * A->nz;
    double *r = malloc(sizeof(double) * N), *z = malloc(sizeof(double) * N);
    double *pd = malloc(sizeof(double) * N), *Ap = malloc(sizeof(double) * N);
    double *dg = malloc(sizeof(double) * N);
    fd_diag(A, dg);
    fd_apply(A, x, Ap);
    for (long k = 0; k < N; ++k) r[k] = b[k] - Ap[k];
    double bn = sqrt(dot(N, b, b));
    if (bn == 0.0) bn = 1.0;
    for (long k = 0; k < N; ++k) { z[k] = r[k] / dg[k]; pd[k] = z[k]; }
    double rz = dot(N, r, z);
    int it = 0;
    double rn = sqrt(dot(N, r, r));
    while (rn > tol * bn && it < maxit) {
        fd_apply(A, pd, Ap);
        double alpha = rz / dot(N, pd, Ap);
        for (long k = 0; k < N; ++k) { x[k] += alpha * pd[k]; r[k] -= alpha * Ap[k]; }
        for (long k = 0; k < N; ++k) z[k] = r[k] / dg[k];
        double rz2 = dot(N, r, z);
        double beta = rz2 / rz;
        rz = rz2;
        for (long k = 0; k < N; ++k) pd[k] = z[k] + beta * pd[k];
        rn = sqrt(dot(N, r, r));
        ++it;
    }
    if (relres) *relres = rn / bn;
    free(r); free(z); free(pd); free(Ap); free(dg);
    return it;
}

/* Jacobi-PCG for (A + diag(shift)) x = b, x = initial guess on entry. */
static int pcg_shifted(const fdop_t *A, const double *shift, const double *b, double *x, double tol, int maxit)
{
    long N = (long)A->nx * A->ny * A->nz;
    double *r = malloc(sizeof(double) * N), *z = malloc(sizeof(double) * N);
    double *pd = malloc(sizeof(double) * N), *Ap = malloc(sizeof(double) * N);
    double *dg = malloc(sizeof(double) * N);
    fd_diag(A, dg);
    for (long k = 0; k < N; ++k) dg[k] += shift[k];
    fd_apply(A, x, Ap);
    for (long k = 0; k < N; ++k) r[k] = b[k] - Ap[k] - shift[k] * x[k];
    double bn = sqrt(dot(N, b, b));
    if (bn == 0.0) bn = 1.0;
    for (long k = 0; k < N; ++k) { z[k] = r[k] / dg[k]; pd[k] = z[k]; }
    double rz = dot(N, r, z);
    int it = 0;
    double rn = sqrt(dot(N, r, r));
    while (rn > tol * bn && it < maxit) {
        fd_apply(A, pd, Ap);
        for (long k = 0; k < N; ++k) Ap[k] += shift[k] * pd[k];
        double alpha = rz / dot(N, pd, Ap);
        for (long k = 0; k < N; ++k) { x[k] += alpha * pd[k]; r[k] -= alpha * Ap[k]; }
        for (long k = 0; k < N; ++k) z[k] = r[k] / dg[k];
        double rz2 = dot(N, r, z);
        double beta = rz2 / rz;
        rz = rz2;
        for (long k = 0; k < N; ++k) pd[k] = z[k] + beta * pd[k];
        rn = sqrt(dot(N, r, r));
        ++it;
    }
    free(r); free(z); free(pd); free(Ap); free(dg);
    return it;
}

static fdop_t fd_alloc(const oracle_problem *p)
{
    fdop_t A;
    long N = (long)p->nx * p->ny * p->nz;
    A.nx = p->nx; A.ny = p->ny; A.nz = p->nz; A.bcx = p->bc[0]; A.bcy = p->bc[1];
    A.cx = calloc(4 * N, sizeof(double));
    A.cy = A.cx + N; A.cz = A.cy + N; A.czlo = A.cz + N;
    return A;
}

/* Poisson (Sec 2.1) in reduced units:  -lap phi = 4 pi lB (rho_f + sum q rho),
 * unit face coefficients (h = 1), no-flux walls carry a zero coefficient.  */
static void poisson_operator(const oracle_problem *p, fdop_t *A)
{
    long N = (long)p->nx * p->ny * p->nz;
    for (long k = 0; k < N; ++k) {
        int i = (int)(k % p->nx), j = (int)((k / p->nx) % p->ny);
        A->cx[k] = (p->bc[0] == 2 && i == p->nx - 1) ? 0.0 : 1.0;
        A->cy[k] = (p->bc[1] == 2 && j == p->ny - 1) ? 0.0 : 1.0;
        A->cz[k] = 1.0;
        A->czlo[k] = 1.0;
    }
}

/* Solve the Poisson equation for the given densities; phi holds the initial
 * guess on entry.  Exposed for the linear-solve pins.                      */
int oracle_poisson(const oracle_problem *p, const double *rho, double *phi, double *relres)
{
    long N = (long)p->nx * p->ny * p->nz, plane = (long)p->nx * p->ny;
    fdop_t A = fd_alloc(p);
    poisson_operator(p, &A);
    double *b = malloc(sizeof(double) * N);
    for (long k = 0; k < N; ++k) {
        double c = p->rho_f ? p->rho_f[k] : 0.0;
        for (int i = 0; i < p->s; ++i) c += p->q[i] * rho[i * N + k];
        b[k] = 4.0 * M_PI * p->lB * c;
    }
    for (long k = 0; k < plane; ++k) {
        b[k] += A.czlo[k] * p->phi_lo;
        b[N - plane + k] += A.cz[N - plane + k] * p->phi_hi;
    }
    int it = pcg(&A, b, phi, p->lin_tol, p->lin_max_iter, relres);
    free(b); free(A.cx);
    return it;
}

/* The Poisson step of the Gummel iteration with the densities' dependence
 * on phi kept to first order: with the Slotboom variables and mu_ex frozen,
 * rho_i(phi) = rho_i exp(-q_i (phi - phi_old)), and one Newton step of the
 * Poisson equation from phi_old is
 *   (A + diag 4 pi lB sum_i q_i^2 rho_i) dphi = b(rho) - A phi_old,
 *   phi* = phi_old + dphi.
 * Its fixed point is the Poisson solution (dphi = 0 there); unlike the plain
 * solve it carries the screening response, so the relaxed iteration stays
 * stable when the domain is many Debye lengths long.  phis gets phi*.     */
static int poisson_newton_step(const oracle_problem *p, const double *rho, const double *phi, double *phis)
{
    long N = (long)p->nx * p->ny * p->nz, plane = (long)p->nx * p->ny;
    fdop_t A = fd_alloc(p);
    poisson_operator(p, &A);
    double *b = malloc(sizeof(double) * N), *Aphi = malloc(sizeof(double) * N);
    double *shift = malloc(sizeof(double) * N), *dphi = calloc(N, sizeof(double));
    for (long k = 0; k < N; ++k) {
        double ch = p->rho_f ? p->rho_f[k] : 0.0, sc = 0.0;
        for (int i = 0; i < p->s; ++i) {
            ch += p->q[i] * rho[i * N + k];
            sc += (double)p->q[i] * p->q[i] * rho[i * N + k];
        }
        b[k] = 4.0 * M_PI * p->lB * ch;
        shift[k] = 4.0 * M_PI * p->lB * sc;
    }
    for (long k = 0; k < plane; ++k) {
        b[k] += A.czlo[k] * p->phi_lo;
        b[N - plane + k] += A.cz[N - plane + k] * p->phi_hi;
    }
    fd_apply(&A, phi, Aphi);
    for (long k = 0; k < N; ++k) b[k] -= Aphi[k];
    int it = pcg_shifted(&A, shift, b, dphi, p->lin_tol, p->lin_max_iter);
    for (long k = 0; k < N; ++k) phis[k] = phi[k] + dphi[k];
    free(b); free(Aphi); free(shift); free(dphi); free(A.cx);
    return it;
}

/* Slotboom Nernst-Planck solve (Sec 2.1 and 3.1) for species i:
 *   Dbar = D exp(-(q phi + mu)),  face coefficient = harmonic mean of the two
 *   node values, Dirichlet rhobar on the z faces from the reservoir
 *   rhobar_face = rho_b exp(q phi_face + mu_b), Dbar_face from phi_face, mu_b.
 * rhobar holds the initial guess on entry.                                  */
int oracle_np(const oracle_problem *p, int i, const double *phi, const double *mu, double mu_b,
              double *rhobar, double *relres)
{
    long N = (long)p->nx * p->ny * p->nz, plane = (long)p->nx * p->ny;
    double Di = p->D ? p->D[i] : 1.0;
    int qi = p->q[i];
    fdop_t A = fd_alloc(p);
    double *Db = malloc(sizeof(double) * N), *b = calloc(N, sizeof(double));
    for (long k = 0; k < N; ++k) Db[k] = Di * exp(-(qi * phi[k] + mu[k]));
    double Dlo = Di * exp(-(qi * p->phi_lo + mu_b)), Dhi = Di * exp(-(qi * p->phi_hi + mu_b));
    double rlo = p->rho_b[i] * exp(qi * p->phi_lo + mu_b), rhi = p->rho_b[i] * exp(qi * p->phi_hi + mu_b);
    for (long k = 0; k < N; ++k) {
        int ok;
        int x = (int)(k % p->nx), y = (int)((k / p->nx) % p->ny), z = (int)(k / plane);
        long qx = nbr(&A, k, 0, +1, &ok);
        A.cx[k] = (p->bc[0] == 2 && x == p->nx - 1) ? 0.0 : 2.0 * Db[k] * Db[qx] / (Db[k] + Db[qx]);
        long qy = nbr(&A, k, 1, +1, &ok);
        A.cy[k] = (p->bc[1] == 2 && y == p->ny - 1) ? 0.0 : 2.0 * Db[k] * Db[qy] / (Db[k] + Db[qy]);
        if (z == p->nz - 1) A.cz[k] = 2.0 * Db[k] * Dhi / (Db[k] + Dhi);
        else A.cz[k] = 2.0 * Db[k] * Db[k + plane] / (Db[k] + Db[k + plane]);
        A.czlo[k] = (z == 0) ? 2.0 * Db[k] * Dlo / (Db[k] + Dlo) : 0.0;
    }
    for (long k = 0; k < plane; ++k) {
        b[k] += A.czlo[k] * rlo;
        b[N - plane + k] += A.cz[N - plane + k] * rhi;
    }
    int it = pcg(&A, b, rhobar, p->lin_tol, p->lin_max_iter, relres);
    free(Db); free(b); free(A.cx);
    return it;
}

/* Discrete z-flux of species i through the face between planes k and k+1
 * (k = -1 .. nz-1), summed over the plane: J = sum c_f (rhobar_k - rhobar_k+1). */
void oracle_np_flux(const oracle_problem *p, int i, const double *phi, const double *mu, double mu_b,
                    const double *rhobar, double *flux /* nz+1 */)
{
    long plane = (long)p->nx * p->ny;
    double Di = p->D ? p->D[i] : 1.0;
    int qi = p->q[i];
    double Dlo = Di * exp(-(qi * p->phi_lo + mu_b)), Dhi = Di * exp(-(qi * p->phi_hi + mu_b));
    double rlo = p->rho_b[i] * exp(qi * p->phi_lo + mu_b), rhi = p->rho_b[i] * exp(qi * p->phi_hi + mu_b);
    for (int kf = -1; kf < p->nz; ++kf) {
        double J = 0.0;
        for (long c = 0; c < plane; ++c) {
            double Da, Dbv, ra, rb;
            if (kf < 0) { Da = Dlo; ra = rlo; }
            else { long a = kf * plane + c; Da = Di * exp(-(qi * phi[a] + mu[a])); ra = rhobar[a]; }
            if (kf + 1 >= p->nz) { Dbv = Dhi; rb = rhi; }
            else { long b = (kf + 1) * plane + c; Dbv = Di * exp(-(qi * phi[b] + mu[b])); rb = rhobar[b]; }
            J += 2.0 * Da * Dbv / (Da + Dbv) * (ra - rb);
        }
        flux[kf + 1] = J;
    }
}

/* ------------------------------------------------------------------ */
/* Relaxed Gummel iteration (Sec 3.2):
 *   mu_ex from rho^{n-1}; Poisson -> phi* (the linear solve with rho^{n-1}, or
 *   with p->screened one Newton step that keeps the densities' Boltzmann
 *   dependence on phi, see poisson_newton_step); phi^n = l1 phi* + (1-l1) phi^{n-1};
 *   per species Slotboom NP solve with Dbar from phi^n and mu_ex -> rhobar;
 *   rho* = rhobar exp(-(q phi^n + mu_ex)); rho^n = l2 rho* + (1-l2) rho^{n-1}
 *   (rho_mix 0, as printed) or rho^n = rho^{n-1} (rho* / rho^{n-1})^l2
 *   (rho_mix 1: the same update to first order, kept positive and bounded for
 *   the large first steps of a dense fluid next to a hard wall), or that step
 *   in ln rho limited to +-0.2 per iteration (rho_mix 2: deep square wells
 *   cannot push the packing fraction past 1 in one step; same fixed point),
 *   or that with a factor per point (rho_mix 3): halved (down to l2/1024)
 *   when the point's step changes sign from the last iteration, else grown
 *   by 10% up to l2 -- the stiff, densely packed points of deep wells then
 *   stop alternating at the step limit; same fixed point;
 *   stop when max(|dphi|_inf, max_i |drho_i|_inf / rho_b,i) < tol.
 * Initial state (when phi0/rho0 are NULL): phi linear in z between the
 * Dirichlet values, rho = rho_b.  Returns 0 converged, 1 not converged,
 * 2 packing error.  hist (max_iter entries, nullable) gets the residuals. */
int oracle_gummel(const oracle_problem *p, const double *phi0, const double *rho0,
                  double *phi, double *rho, int *iters, double *hist, long *lin_iters)
{
    long N = (long)p->nx * p->ny * p->nz, plane = (long)p->nx * p->ny;
    int s = p->s;
    double *mu = malloc(sizeof(double) * s * N);
    double *phis = malloc(sizeof(double) * N);
    double *rb = malloc(sizeof(double) * N);
    double *mub = malloc(sizeof(double) * s);
    double *rho_new = malloc(sizeof(double) * s * N);
    /* rho_mix 3: per-point relaxation factor and last step in ln rho */
    double *lam = malloc(sizeof(double) * s * N), *prev = calloc((size_t)s * N, sizeof(double));
    for (long k = 0; k < s * N; ++k) lam[k] = p->lambda_rho;
    oracle_bulk_mu_fmt(p->fmt, s, p->R, p->rho_b, mub);
    if (phi0) memcpy(phi, phi0, sizeof(double) * N);
    else
        for (long k = 0; k < N; ++k) {
            int z = (int)(k / plane);
            phi[k] = p->phi_lo + (p->phi_hi - p->phi_lo) * (z + 1.0) / (p->nz + 1.0);
        }
    if (rho0) memcpy(rho, rho0, sizeof(double) * s * N);
    else
        for (int i = 0; i < s; ++i)
            for (long k = 0; k < N; ++k) rho[i * N + k] = p->rho_b[i];
    long lin = 0;
    int status = 1, n;
    double rr = 0.0;
    for (n = 1; n <= p->max_iter; ++n) {
        if (oracle_excess_mu(p, rho, mu) > 0) { status = 2; break; }
        memcpy(phis, phi, sizeof(double) * N);
        if (p->screened) lin += poisson_newton_step(p, rho, phi, phis);
        else lin += oracle_poisson(p, rho, phis, 0);
        double dphi = 0.0;
        for (long k = 0; k < N; ++k) {
            double v = p->lambda_phi * phis[k] + (1.0 - p->lambda_phi) * phi[k];
            double d = fabs(v - phi[k]);
            if (d > dphi) dphi = d;
            phi[k] = v;
        }
        rr = dphi;
        for (int i = 0; i < s; ++i) {
            const double *mui = mu + i * N;
            /* initial guess: Slotboom variable of the current density */
            for (long k = 0; k < N; ++k) rb[k] = rho[i * N + k] * exp(p->q[i] * phi[k] + mui[k]);
            lin += oracle_np(p, i, phi, mui, mub[i], rb, 0);
            double drho = 0.0;
            for (long k = 0; k < N; ++k) {
                double rs = rb[k] * exp(-(p->q[i] * phi[k] + mui[k]));
                double v;
                if (p->rho_mix == 0) {
                    v = p->lambda_rho * rs + (1.0 - p->lambda_rho) * rho[i * N + k];
                } else if (p->rho_mix == 3) {
                    long t = i * N + k;
                    double d = log(rs / rho[t]);
                    if (d * prev[t] < 0.0) lam[t] = fmax(0.5 * lam[t], p->lambda_rho / 1024.0);
                    else lam[t] = fmin(1.1 * lam[t], p->lambda_rho);
                    double step = lam[t] * d;
                    step = step > 0.2 ? 0.2 : (step < -0.2 ? -0.2 : step);
                    prev[t] = step;
                    v = rho[t] * exp(step);
                } else {
                    double step = p->lambda_rho * log(rs / rho[i * N + k]);
                    if (p->rho_mix == 2) step = step > 0.2 ? 0.2 : (step < -0.2 ? -0.2 : step);
                    v = rho[i * N + k] * exp(step);
                }
                double d = fabs(v - rho[i * N + k]) / p->rho_b[i];
                if (d > drho) drho = d;
                rho_new[i * N + k] = v;
            }
            if (drho > rr) rr = drho;
        }
        memcpy(rho, rho_new, sizeof(double) * s * N);
        if (hist) hist[n - 1] = rr;
        if (rr < p->tol) { status = 0; break; }
    }
    if (iters) *iters = n > p->max_iter ? p->max_iter : n;
    if (lin_iters) *lin_iters = lin;
    free(mu); free(phis); free(rb); free(mub); free(rho_new); free(lam); free(prev);
    return status;
}

/* ------------------------------------------------------------------ */
/* Anderson acceleration of the relaxed Gummel iteration (an extension: the
 * paper relaxes only).  The base map G is one sweep of oracle_gummel's loop
 * body (mu_ex, Poisson step, phi relaxation, the NP solves and the density
 * relaxation) acting on x = (phi, ln rho).  With f = G(x) - x and the last
 * k <= m differences dX, dF of iterates and residuals,
 *   gamma = argmin || f - dF gamma ||_2   (normal equations, tiny ridge),
 *   x <- x + f - (dX + dF) gamma.
 * If the extrapolated state is unphysical (packing or a non-finite value in
 * the next sweep) the history is dropped and the plain iterate G(x) taken;
 * if the sweep from that fails as well, the step from the last recorded
 * iterate x is halved, x + f/2, x + f/4, ..., at most AA_BACKTRACK times (x
 * swept cleanly, so a short enough step does too).
 * Stops on the residual of the base map, max(|dphi|, max_i |drho_i| / rho_b,i)
 * < tol, like the plain iteration; so the fixed point is the same.
 * Returns 0 converged, 1 not converged, 2 packing of a plain iterate.     */
static int gummel_sweep(const oracle_problem *p, const double *mub, const double *phi, const double *rho,
                        double *phi_out, double *rho_out, double *mu, double *rb, double *rr)
{
    long N = (long)p->nx * p->ny * p->nz;
    int s = p->s;
    if (oracle_excess_mu(p, rho, mu) > 0) return 2;
    memcpy(phi_out, phi, sizeof(double) * N);
    if (p->screened) poisson_newton_step(p, rho, phi, phi_out);
    else oracle_poisson(p, rho, phi_out, 0);
    double r = 0.0;
    for (long k = 0; k < N; ++k) {
        double v = p->lambda_phi * phi_out[k] + (1.0 - p->lambda_phi) * phi[k];
        if (fabs(v - phi[k]) > r) r = fabs(v - phi[k]);
        phi_out[k] = v;
    }
    for (int i = 0; i < s; ++i) {
        const double *mui = mu + i * N;
        for (long k = 0; k < N; ++k) rb[k] = rho[i * N + k] * exp(p->q[i] * phi_out[k] + mui[k]);
        oracle_np(p, i, phi_out, mui, mub[i], rb, 0);
        for (long k = 0; k < N; ++k) {
            double rs = rb[k] * exp(-(p->q[i] * phi_out[k] + mui[k]));
            double old = rho[i * N + k], v;
            if (p->rho_mix == 0) {
                v = p->lambda_rho * rs + (1.0 - p->lambda_rho) * old;
            } else {
                double step = p->lambda_rho * log(rs / old);
                if (p->rho_mix >= 2) step = step > 0.2 ? 0.2 : (step < -0.2 ? -0.2 : step);
                v = old * exp(step);
            }
            if (!isfinite(v) || !(v > 0.0)) return 2;
            double d = fabs(v - old) / p->rho_b[i];
            if (d > r) r = d;
            rho_out[i * N + k] = v;
        }
    }
    *rr = r;
    return 0;
}

/* solve the k x k system A y = b in place (Gaussian elimination, partial
 * pivoting); returns 0 on success */
static int small_solve(int k, double *A, double *b)
{
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int r = c + 1; r < k; ++r) if (fabs(A[r * k + c]) > fabs(A[piv * k + c])) piv = r;
        if (A[piv * k + c] == 0.0) return 1;
        if (piv != c) {
            for (int j = 0; j < k; ++j) { double t = A[c * k + j]; A[c * k + j] = A[piv * k + j]; A[piv * k + j] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < k; ++r) {
            double f = A[r * k + c] / A[c * k + c];
            for (int j = c; j < k; ++j) A[r * k + j] -= f * A[c * k + j];
            b[r] -= f * b[c];
        }
    }
    for (int c = k - 1; c >= 0; --c) {
        double v = b[c];
        for (int j = c + 1; j < k; ++j) v -= A[c * k + j] * b[j];
        b[c] = v / A[c * k + c];
    }
    return 0;
}

#define AA_BACKTRACK 8
int oracle_gummel_anderson(const oracle_problem *p, int m, double *phi, double *rho, int *iters, double *hist)
{
    long N = (long)p->nx * p->ny * p->nz, plane = (long)p->nx * p->ny;
    int s = p->s;
    long M = (long)(1 + s) * N;
    if (m < 1) m = 1;
    if (m > 16) m = 16;
    double *mub = malloc(sizeof(double) * s), *mu = malloc(sizeof(double) * s * N), *rb = malloc(sizeof(double) * N);
    double *x = malloc(sizeof(double) * M), *g = malloc(sizeof(double) * M), *f = malloc(sizeof(double) * M);
    double *X = malloc(sizeof(double) * M * (m + 1)), *F = malloc(sizeof(double) * M * (m + 1));
    double *phi_g = malloc(sizeof(double) * N), *rho_g = malloc(sizeof(double) * s * N);
    double A[16 * 16], bvec[16];
    oracle_bulk_mu_fmt(p->fmt, s, p->R, p->rho_b, mub);
    for (long k = 0; k < N; ++k) {
        int z = (int)(k / plane);
        phi[k] = p->phi_lo + (p->phi_hi - p->phi_lo) * (z + 1.0) / (p->nz + 1.0);
    }
    for (int i = 0; i < s; ++i)
        for (long k = 0; k < N; ++k) rho[i * N + k] = p->rho_b[i];
    int hlen = 0, status = 1, n;
    double rr = 0.0;
    for (n = 1; n <= p->max_iter; ++n) {
        int rc = gummel_sweep(p, mub, phi, rho, phi_g, rho_g, mu, rb, &rr);
        if (rc && hlen > 0 && n > 1) {
            /* the state is unphysical: restart from the last plain iterate
             * g = x + f of the last recorded pair, and while the sweep from
             * there fails too, halve the step: x + theta f, theta = 1/2,
             * 1/4, ... down to 2^-AA_BACKTRACK (x itself swept cleanly) */
            double theta = 1.0;
            for (int bt = 0; rc && bt <= AA_BACKTRACK; ++bt) {
                if (bt == 0) {
                    for (long k = 0; k < N; ++k) phi[k] = g[k];
                    for (long k = 0; k < s * N; ++k) rho[k] = exp(g[N + k]);
                } else {
                    for (long k = 0; k < N; ++k) phi[k] = x[k] + theta * f[k];
                    for (long k = 0; k < s * N; ++k) rho[k] = exp(x[N + k] + theta * f[N + k]);
                }
                hlen = 0;
                rc = gummel_sweep(p, mub, phi, rho, phi_g, rho_g, mu, rb, &rr);
                theta *= 0.5;
            }
        }
        if (rc) { status = 2; break; }
        if (hist) hist[n - 1] = rr;
        if (rr < p->tol) {
            memcpy(phi, phi_g, sizeof(double) * N);
            memcpy(rho, rho_g, sizeof(double) * s * N);
            status = 0;
            break;
        }
        for (long k = 0; k < N; ++k) { x[k] = phi[k]; g[k] = phi_g[k]; }
        for (long k = 0; k < s * N; ++k) { x[N + k] = log(rho[k]); g[N + k] = log(rho_g[k]); }
        for (long k = 0; k < M; ++k) f[k] = g[k] - x[k];
        /* history ring: keep the last m+1 (x, f) pairs */
        if (hlen == m + 1) {
            memmove(X, X + M, sizeof(double) * M * m);
            memmove(F, F + M, sizeof(double) * M * m);
            hlen = m;
        }
        memcpy(X + M * hlen, x, sizeof(double) * M);
        memcpy(F + M * hlen, f, sizeof(double) * M);
        ++hlen;
        int kd = hlen - 1;
        double *xn = malloc(sizeof(double) * M);
        for (long k = 0; k < M; ++k) xn[k] = g[k];
        if (kd > 0) {
            /* dF_j = F_{j+1} - F_j, dX_j = X_{j+1} - X_j */
            double tr = 0.0;
            for (int a = 0; a < kd; ++a) {
                for (int b = 0; b <= a; ++b) {
                    double sum = 0.0;
                    for (long k = 0; k < M; ++k)
                        sum += (F[M * (a + 1) + k] - F[M * a + k]) * (F[M * (b + 1) + k] - F[M * b + k]);
                    A[a * kd + b] = A[b * kd + a] = sum;
                }
                tr += A[a * kd + a];
                double sb = 0.0;
                for (long k = 0; k < M; ++k) sb += (F[M * (a + 1) + k] - F[M * a + k]) * f[k];
                bvec[a] = sb;
            }
            for (int a = 0; a < kd; ++a) A[a * kd + a] += 1e-12 * tr + 1e-300;
            if (small_solve(kd, A, bvec) == 0) {
                for (long k = 0; k < M; ++k) {
                    double v = x[k] + f[k];
                    for (int a = 0; a < kd; ++a)
                        v -= bvec[a] * ((X[M * (a + 1) + k] - X[M * a + k]) + (F[M * (a + 1) + k] - F[M * a + k]));
                    xn[k] = v;
                }
            }
        }
        for (long k = 0; k < N; ++k) phi[k] = xn[k];
        for (long k = 0; k < s * N; ++k) rho[k] = exp(xn[N + k]);
        free(xn);
    }
    if (iters) *iters = n > p->max_iter ? p->max_iter : n;
    free(mub); free(mu); free(rb); free(x); free(g); free(f); free(X); free(F); free(phi_g); free(rho_g);
    return status;
}

/* ------------------------------------------------------------------ */
/* Equilibrium cDFT initial guess (Sec 3.2, choice of initial guess): the
 * static equilibrium of the mobile species in the potential of the
 * electrodes, which then starts the Gummel iteration.  At equilibrium every
 * species follows the Boltzmann law about its reservoir,
 *     rho_i = rho_b,i exp(mu_b,i - mu_ex,i[rho] - q_i phi),
 * and phi solves the Poisson equation with these densities (Poisson-Boltzmann
 * with the cDFT excess term).  One iteration, in this order:
 *   mu_ex from rho;  c_i = rho_b,i exp(mu_b,i - mu_ex,i);
 *   one Newton step of the Poisson-Boltzmann equation in phi at fixed c:
 *     (A + diag 4 pi lB sum_i q_i^2 c_i e^{-q_i phi}) dphi = b(phi) - A phi,
 *     b(phi) = 4 pi lB (rho_f + sum_i q_i c_i e^{-q_i phi}) + Dirichlet terms,
 *     dphi clamped to +-1 at each point, phi += dphi;
 *   rho*_i = c_i e^{-q_i phi};  rho_i <- rho_i exp(step), step = lam ln(rho*_i / rho_i)
 *     limited to +-0.2 (the step-limited geometric relaxation);
 *   stop when max(|dphi|_inf, max_i |drho_i|_inf / rho_b,i) < tol.
 * Starts from phi linear in z between the Dirichlet values and rho = rho_b.
 * Returns 0 converged, 1 not converged, 2 packing or overflow.  The linear
 * solve uses the oracle's Jacobi-PCG at the problem's lin_tol.          */
int oracle_equilibrium(const oracle_problem *p, double lam, double tol, int max_iter,
                       double *phi, double *rho, int *iters, double *res)
{
    long N = (long)p->nx * p->ny * p->nz, plane = (long)p->nx * p->ny;
    int s = p->s;
    double *mu = malloc(sizeof(double) * s * N), *c = malloc(sizeof(double) * s * N);
    double *mub = malloc(sizeof(double) * s);
    double *b = malloc(sizeof(double) * N), *Aphi = malloc(sizeof(double) * N), *dphi = malloc(sizeof(double) * N);
    fdop_t A = fd_alloc(p);
    poisson_operator(p, &A);
    oracle_bulk_mu_fmt(p->fmt, s, p->R, p->rho_b, mub);
    for (long k = 0; k < N; ++k) {
        int z = (int)(k / plane);
        phi[k] = p->phi_lo + (p->phi_hi - p->phi_lo) * (z + 1.0) / (p->nz + 1.0);
    }
    for (int i = 0; i < s; ++i)
        for (long k = 0; k < N; ++k) rho[i * N + k] = p->rho_b[i];
    int status = 1, n;
    double rr = 0.0;
    for (n = 1; n <= max_iter; ++n) {
        if (oracle_excess_mu(p, rho, mu) > 0) { status = 2; break; }
        for (int i = 0; i < s; ++i)
            for (long k = 0; k < N; ++k) c[i * N + k] = p->rho_b[i] * exp(mub[i] - mu[i * N + k]);
        /* Newton step: Jacobian = Poisson operator + diagonal screening term */
        double *shift = malloc(sizeof(double) * N);
        for (long k = 0; k < N; ++k) {
            double ch = p->rho_f ? p->rho_f[k] : 0.0, sc = 0.0;
            for (int i = 0; i < s; ++i) {
                double r = c[i * N + k] * exp(-p->q[i] * phi[k]);
                ch += p->q[i] * r;
                sc += (double)p->q[i] * p->q[i] * r;
            }
            b[k] = 4.0 * M_PI * p->lB * ch;
            shift[k] = 4.0 * M_PI * p->lB * sc;
        }
        for (long k = 0; k < plane; ++k) {
            b[k] += A.czlo[k] * p->phi_lo;
            b[N - plane + k] += A.cz[N - plane + k] * p->phi_hi;
        }
        fd_apply(&A, phi, Aphi);
        for (long k = 0; k < N; ++k) { b[k] -= Aphi[k]; dphi[k] = 0.0; }
        int bad = 0;
        for (long k = 0; k < N; ++k) if (!isfinite(b[k]) || !isfinite(shift[k])) bad = 1;
        if (bad) { free(shift); status = 2; break; }
        pcg_shifted(&A, shift, b, dphi, p->lin_tol, p->lin_max_iter);
        free(shift);
        double dmax = 0.0;
        for (long k = 0; k < N; ++k) {
            double d = dphi[k] > 1.0 ? 1.0 : (dphi[k] < -1.0 ? -1.0 : dphi[k]);
            phi[k] += d;
            if (fabs(d) > dmax) dmax = fabs(d);
        }
        rr = dmax;
        for (int i = 0; i < s; ++i) {
            double drho = 0.0;
            for (long k = 0; k < N; ++k) {
                double rs = c[i * N + k] * exp(-p->q[i] * phi[k]);
                double step = lam * log(rs / rho[i * N + k]);
                step = step > 0.2 ? 0.2 : (step < -0.2 ? -0.2 : step);
                double v = rho[i * N + k] * exp(step);
                if (!isfinite(v) || !(v > 0.0)) bad = 1;
                double d = fabs(v - rho[i * N + k]) / p->rho_b[i];
                if (d > drho) drho = d;
                rho[i * N + k] = v;
            }
            if (drho > rr) rr = drho;
        }
        if (bad) { status = 2; break; }
        if (rr < tol) { status = 0; break; }
    }
    if (iters) *iters = n > max_iter ? max_iter : n;
    if (res) *res = rr;
    free(mu); free(c); free(mub); free(b); free(Aphi); free(dphi); free(A.cx);
    return status;
}

/* Thread count of the OpenMP loops (n <= 0: one per processor). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
