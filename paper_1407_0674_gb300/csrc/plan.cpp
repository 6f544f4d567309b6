// Host-side planning: descriptor validation, padded FFT lengths, quadrature
// stencils of the weight functions and their spectra.
//
// Stencils.  Every integral over a sphere, ball or shell is the quadrature of
// Sec 3.5 (change of variables to (theta, phi)): trapezoid in theta at
// (a + 1/2) 2pi/n_theta, Gauss-Legendre in mu = cos(phi), and Gauss-Legendre in
// r with the r^2 factor for volumes; the value of a grid field at an off-grid
// node is trilinear in its 8 neighbours.  Because every output point is a grid
// point, the whole rule collapses to a translation-invariant stencil
// K[m] = sum_nodes weight * trilinear weight of offset m, applied as
// n(r) = sum_m K[m] rho(r + m) (Sec 2.3.1 correlation) and its transpose.
// Default counts: n_mu = max(8, ceil(2 pi R)), n_theta = 2 n_mu rounded up to a
// multiple of 4, n_r = max(4, ceil(2 (r_out - r_in))).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "pnp_internal.h"

namespace pnp {

bool smooth235(int n) {
    if (n < 1) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

int next_smooth(int n, bool even) {
    for (int m = std::max(n, 1);; ++m)
        if (smooth235(m) && (!even || m % 2 == 0)) return m;
}

FftAxis make_axis(int L) {
    FftAxis a{};
    a.L = L;
    int m = L, k = 0;
    while (m % 4 == 0) { a.radix[k++] = 4; m /= 4; }
    for (int p : {2, 3, 5})
        while (m % p == 0) { a.radix[k++] = p; m /= p; }
    a.nst = k;
    return a;
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method from Tricomi's
// asymptotic starting values, with P_n' carried by P'_k = P'_{k-2} + (2k-1) P_{k-1}.
void gauss_legendre_nodes(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 1; i <= n; ++i) {
        double t = (1.0 - (n - 1.0) / (8.0 * n * (double)n * n)) * std::cos(M_PI * (4.0 * i - 1.0) / (4.0 * n + 2.0));
        double dp = 1.0;
        for (int it = 0; it < 60; ++it) {
            double pkm1 = 1.0, pk = t, dkm1 = 0.0, dk = 1.0;
            for (int k = 2; k <= n; ++k) {
                double pn = ((2.0 * k - 1.0) * t * pk - (k - 1.0) * pkm1) / k;
                double dn = dkm1 + (2.0 * k - 1.0) * pk;
                pkm1 = pk; pk = pn;
                dkm1 = dk; dk = dn;
            }
            double step = pk / dk;
            t -= step;
            dp = dk;
            if (std::fabs(step) <= 1e-17 * std::max(1.0, std::fabs(t))) break;
        }
        // derivative at the converged node
        {
            double pkm1 = 1.0, pk = t, dkm1 = 0.0, dk = 1.0;
            for (int k = 2; k <= n; ++k) {
                double pn = ((2.0 * k - 1.0) * t * pk - (k - 1.0) * pkm1) / k;
                double dn = dkm1 + (2.0 * k - 1.0) * pk;
                pkm1 = pk; pk = pn;
                dkm1 = dk; dk = dn;
            }
            dp = dk;
        }
        x[i - 1] = t;
        w[i - 1] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

namespace {

struct Node {
    double p[3];
    double u[3];
    double w;
};

int rule_nmu(double r, int given) { return given > 0 ? given : std::max(8, (int)std::ceil(2.0 * M_PI * r)); }
int rule_ntheta(int nmu, int given) { return given > 0 ? given : ((2 * nmu + 3) / 4) * 4; }
int rule_nr(double len, int given) { return given > 0 ? given : std::max(4, (int)std::ceil(2.0 * len)); }

// radial nodes: radius r_out alone (surface) or Gauss-Legendre on [r_in, r_out]
// with the r^2 volume factor
std::vector<Node> nodes(bool surface, double r_in, double r_out, int nmu, int ntheta, int nr) {
    nmu = rule_nmu(r_out, nmu);
    ntheta = rule_ntheta(nmu, ntheta);
    std::vector<double> rad, radw;
    if (surface) {
        rad = {r_out};
        radw = {r_out * r_out};
    } else {
        nr = rule_nr(r_out - r_in, nr);
        std::vector<double> gx, gw;
        gauss_legendre_nodes(nr, gx, gw);
        double half = 0.5 * (r_out - r_in), mid = 0.5 * (r_out + r_in);
        for (int k = 0; k < nr; ++k) {
            double r = mid + half * gx[k];
            rad.push_back(r);
            radw.push_back(half * gw[k] * r * r);
        }
    }
    std::vector<double> mx, mw;
    gauss_legendre_nodes(nmu, mx, mw);
    const double dth = 2.0 * M_PI / ntheta;
    std::vector<Node> out;
    out.reserve(rad.size() * nmu * ntheta);
    for (size_t k = 0; k < rad.size(); ++k)
        for (int b = 0; b < nmu; ++b) {
            double sinphi = std::sqrt(std::max(0.0, 1.0 - mx[b] * mx[b]));
            for (int a = 0; a < ntheta; ++a) {
                double th = dth * (a + 0.5);
                Node n;
                n.u[0] = std::cos(th) * sinphi;
                n.u[1] = std::sin(th) * sinphi;
                n.u[2] = mx[b];
                for (int c = 0; c < 3; ++c) n.p[c] = rad[k] * n.u[c];
                n.w = radw[k] * mw[b] * dth;
                out.push_back(n);
            }
        }
    return out;
}

// add weight `wt` of a node at p to the stencil with trilinear weights
void deposit(Stencil &st, const double p[3], double wt) {
    int base[3];
    double fr[3];
    for (int c = 0; c < 3; ++c) {
        double f = std::floor(p[c]);
        base[c] = (int)f;
        fr[c] = p[c] - f;
    }
    for (int cz = 0; cz < 2; ++cz) {
        double wz = cz ? fr[2] : 1.0 - fr[2];
        for (int cy = 0; cy < 2; ++cy) {
            double wy = cy ? fr[1] : 1.0 - fr[1];
            for (int cx = 0; cx < 2; ++cx) {
                double wx = cx ? fr[0] : 1.0 - fr[0];
                double v = wt * wx * wy * wz;
                if (v == 0.0) continue;
                st.at(base[0] + cx, base[1] + cy, base[2] + cz) += v;
            }
        }
    }
}

void reset(Stencil &st, int S) {
    st.S = S;
    st.K.assign((size_t)(2 * S + 1) * (2 * S + 1) * (2 * S + 1), 0.0);
}

}  // namespace

// Shell (scalar), ball and the three vector-shell components for radius R
// (weights w2, w3, vec w2 of Sec 2.3.1; w0, w1, vec w1 are scalar multiples).
void build_fmt_stencils(double R, int nmu, int ntheta, int nr, int S, Stencil out[kNumKernels]) {
    for (int k = 0; k < kNumKernels; ++k) reset(out[k], S);
    for (const Node &n : nodes(true, 0.0, R, nmu, ntheta, nr)) {
        deposit(out[0], n.p, n.w);
        for (int c = 0; c < 3; ++c) deposit(out[2 + c], n.p, n.w * n.u[c]);
    }
    for (const Node &n : nodes(false, 0.0, R, nmu, ntheta, nr)) deposit(out[1], n.p, n.w);
}

// Square-well shell r_in <= |r| <= r_out (Sec 2.3.2), volume weight.
void build_well_stencil(double r_in, double r_out, int nmu, int ntheta, int nr, int S, Stencil &out) {
    reset(out, S);
    for (const Node &n : nodes(false, r_in, r_out, nmu, ntheta, nr)) deposit(out, n.p, n.w);
}

// MSA pair kernel of Sec 2.3.4 on the ball |r| <= sigma, deposited like the
// FMT weights: C(r) = -qq_lB [2B/sigma - (B/sigma)^2 r - 1/r], qq_lB = q_i q_j l_B.
// The quadrature weight carries r^2, so C's 1/r stays finite at every node.
void build_msa_stencil(double qq_lB, double B, double sigma, int nmu, int ntheta, int nr, int S, Stencil &out) {
    reset(out, S);
    for (const Node &n : nodes(false, 0.0, sigma, nmu, ntheta, nr)) {
        const double r = std::sqrt(n.p[0] * n.p[0] + n.p[1] * n.p[1] + n.p[2] * n.p[2]);
        const double C = -qq_lB * (2.0 * B / sigma - (B / sigma) * (B / sigma) * r - 1.0 / r);
        deposit(out, n.p, n.w * C);
    }
}

// C_ij of a problem on its own reach ceil(R_i + R_j) + 1 (Sec 2.3.4)
void build_msa_pair(const Problem &p, int i, int j, Stencil &out) {
    const double sigma = p.R[i] + p.R[j];
    double kappa2 = 0.0;
    for (int k = 0; k < p.s; ++k) kappa2 += 4.0 * M_PI * p.lB * p.rho_b[k] * p.q[k] * p.q[k];
    const double B = msa_B(std::sqrt(kappa2) * sigma);
    build_msa_stencil((double)p.q[i] * p.q[j] * p.lB, B, sigma, p.quad[0], p.quad[1], p.quad[2],
                      (int)std::ceil(sigma) + 1, out);
}

// MSA screening factor B = [xi + 1 - sqrt(1 + 2 xi)] / xi of Sec 2.3.4, taken
// as 2 xi / (1 + sqrt(1 + 2 xi))^2 (the same number) where the printed form
// cancels.
double msa_B(double xi) {
    if (xi < 1e-3) {
        const double t = 1.0 + std::sqrt(1.0 + 2.0 * xi);
        return 2.0 * xi / (t * t);
    }
    return (xi + 1.0 - std::sqrt(1.0 + 2.0 * xi)) / xi;
}

// out[kz][ky][kx] (kz <= Lz/2, ky <= Ly/2, kx <= Lx/2) =
//   scale * sum_m K[m] f_x(kx mx) f_y(ky my) f_z(kz mz),  f = cos(2 pi k m / L)
// on even axes and sin(...) on odd axes.  The stencil is even or odd in each
// axis, so this real octant determines its whole DFT:
//   DFT(K)(k) = prod over odd axes of (-i sign(k)) * out(|k|).
void octant_transform(const Stencil &st, const int L[3], const bool odd[3], double scale, double *out) {
    const int S = st.S, W = 2 * S + 1;
    int O[3];
    for (int c = 0; c < 3; ++c) O[c] = L[c] / 2 + 1;
    std::vector<double> tab[3];
    for (int c = 0; c < 3; ++c) {
        tab[c].resize((size_t)O[c] * W);
        for (int k = 0; k < O[c]; ++k)
            for (int m = -S; m <= S; ++m) {
                long r = ((long)k * m) % L[c];
                if (r < 0) r += L[c];
                double ang = 2.0 * M_PI * (double)r / L[c];
                tab[c][(size_t)k * W + (m + S)] = odd[c] ? std::sin(ang) : std::cos(ang);
            }
    }
    // stage 1: x
    std::vector<double> t1((size_t)W * W * O[0], 0.0);
    for (int mz = 0; mz < W; ++mz)
        for (int my = 0; my < W; ++my)
            for (int kx = 0; kx < O[0]; ++kx) {
                double acc = 0.0;
                const double *row = &st.K[((size_t)mz * W + my) * W];
                const double *tr = &tab[0][(size_t)kx * W];
                for (int mx = 0; mx < W; ++mx) acc += row[mx] * tr[mx];
                t1[((size_t)mz * W + my) * O[0] + kx] = acc;
            }
    // stage 2: y
    std::vector<double> t2((size_t)W * O[1] * O[0], 0.0);
    for (int mz = 0; mz < W; ++mz)
        for (int ky = 0; ky < O[1]; ++ky) {
            const double *tr = &tab[1][(size_t)ky * W];
            double *dst = &t2[((size_t)mz * O[1] + ky) * O[0]];
            for (int my = 0; my < W; ++my) {
                const double *src = &t1[((size_t)mz * W + my) * O[0]];
                double f = tr[my];
                if (f == 0.0) continue;
                for (int kx = 0; kx < O[0]; ++kx) dst[kx] += f * src[kx];
            }
        }
    // stage 3: z, split over host threads
    unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    nth = std::min<unsigned>(nth, (unsigned)O[2]);
    auto work = [&](int k0, int k1) {
        for (int kz = k0; kz < k1; ++kz) {
            const double *tr = &tab[2][(size_t)kz * W];
            double *dst = &out[(size_t)kz * O[1] * O[0]];
            std::fill(dst, dst + (size_t)O[1] * O[0], 0.0);
            for (int mz = 0; mz < W; ++mz) {
                double f = tr[mz];
                if (f == 0.0) continue;
                const double *src = &t2[(size_t)mz * O[1] * O[0]];
                for (size_t j = 0; j < (size_t)O[1] * O[0]; ++j) dst[j] += f * src[j];
            }
            for (size_t j = 0; j < (size_t)O[1] * O[0]; ++j) dst[j] *= scale;
        }
    };
    std::vector<std::thread> pool;
    int chunk = (O[2] + (int)nth - 1) / (int)nth;
    for (unsigned t = 0; t < nth; ++t) {
        int a = (int)t * chunk, b = std::min(O[2], a + chunk);
        if (a < b) pool.emplace_back(work, a, b);
    }
    for (auto &th : pool) th.join();
}

// SI constants (CODATA 2018; e and k_B exact).
static const double kCharge = 1.602176634e-19;   // C
static const double kEps0 = 8.8541878128e-12;    // F/m
static const double kBoltzmann = 1.380649e-23;   // J/K

// Bjerrum length e^2 / (4 pi eps0 eps_r k_B T) (Sec 2.3.3) from SI constants,
// expressed in grid spacings.
double bjerrum_length_h(double T, double eps_r, double h_nm) {
    double lB_m = kCharge * kCharge / (4.0 * M_PI * kEps0 * eps_r * kBoltzmann * T);
    return lB_m * 1e9 / h_nm;
}

// The unit of the reduced conductivity, e^2 D / (k_B T h^3), in S/cm.
double conductivity_unit_S_per_cm(double T, double h_nm, double D_m2_per_s) {
    const double h = h_nm * 1e-9;
    return kCharge * kCharge * D_m2_per_s / (kBoltzmann * T * h * h * h) / 100.0;
}

// Reservoir excess chemical potential: in a uniform fluid every weighted
// density is rho times the weight's integral, so mu_i = sum_alpha dPhi/dn_alpha
// * int w_i^alpha with the integrals 1, R, 4 pi R^2, 4 pi R^3 / 3 (Sec 2.3.1).
// Reservoir chemical potential mu_b,i = sum_a dPhi/dn_a(bulk n) x (integral of
// weight a of species i), for the problem's functional.
void bulk_mu_fmt(const Problem &p, std::vector<double> &mu) {
    double n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    for (int i = 0; i < p.s; ++i) {
        double R = p.R[i], r = p.rho_b[i];
        n0 += r;
        n1 += r * R;
        n2 += r * 4.0 * M_PI * R * R;
        n3 += r * 4.0 * M_PI * R * R * R / 3.0;
    }
    double g = 1.0 / (1.0 - n3);
    double d0 = -std::log1p(-n3);
    double d1 = n2 * g;
    double d2, d3;
    if (p.fmt == PNP_FMT_WHITE_BEAR) {
        // phi3 and its derivative: series below 0.05, closed form above
        double f, df;
        if (std::fabs(n3) < 0.05) {
            f = 0.0;
            df = 0.0;
            double xp = 1.0;
            for (int k = 0; k <= 24; ++k) {
                const double c = (double)(k + 1) * (k + 3) / (k + 2);
                f += c * xp;
                if (k + 1 <= 24) df += (k + 1) * ((double)(k + 2) * (k + 4) / (k + 3)) * xp;
                xp *= n3;
            }
        } else {
            const double o = 1.0 - n3, L = std::log(o);
            f = (n3 + o * o * L) / (n3 * n3 * o * o);
            df = (n3 - 2.0 * o * L) / (n3 * n3 * o * o) - 2.0 * (1.0 - 2.0 * n3) * f / (n3 * o);
        }
        d2 = n1 * g + n2 * n2 * f / (12.0 * M_PI);
        d3 = n0 * g + n1 * n2 * g * g + n2 * n2 * n2 * df / (36.0 * M_PI);
    } else {
        d2 = n1 * g + n2 * n2 * g * g / (8.0 * M_PI);
        d3 = n0 * g + n1 * n2 * g * g + n2 * n2 * n2 * g * g * g / (12.0 * M_PI);
    }
    mu.resize(p.s);
    for (int i = 0; i < p.s; ++i) {
        double R = p.R[i];
        mu[i] = d0 + R * d1 + 4.0 * M_PI * R * R * d2 + 4.0 * M_PI * R * R * R / 3.0 * d3;
    }
}

int validate_and_copy(const pnp_problem_desc *d, Problem *p, std::string *why) {
    auto bad = [&](const char *m) { if (why) *why = m; return PNP_ERR_INVALID; };
    if (!d) return bad("null descriptor");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx > 4096 || d->ny > 4096 || d->nz > 4096)
        return bad("grid size out of range");
    if (d->nspecies < 1 || d->nspecies > 8) return bad("nspecies must be 1..8");
    if (!d->valence || !d->radius || !d->rho_bulk) return bad("valence, radius and rho_bulk are required");
    for (int c = 0; c < 3; ++c)
        if (d->bc[c] < 0 || d->bc[c] > 2) return bad("bad boundary type");
    if (d->temperature_K <= 0 || d->eps_r <= 0 || d->h_nm <= 0) return bad("temperature, eps_r, h_nm must be > 0");
    if (!(d->lambda_phi > 0 && d->lambda_phi <= 1) || !(d->lambda_rho > 0 && d->lambda_rho <= 1))
        return bad("relaxation parameters must be in (0, 1]");
    if (d->rho_mix < PNP_MIX_LINEAR || d->rho_mix > PNP_MIX_ADAPTIVE) return bad("bad rho_mix");
    const bool eq = (d->flags & PNP_FLAG_EQUILIBRIUM_INIT) != 0;
    if (!(d->tol > 0) || d->max_iter < (eq ? 0 : 1))
        return bad("tol must be > 0 and max_iter >= 1 (>= 0 with the equilibrium initial guess)");
    if (d->eq_tol < 0 || d->eq_max_iter < 0) return bad("eq_tol and eq_max_iter must be >= 0");
    if (d->fmt != PNP_FMT_ROSENFELD && d->fmt != PNP_FMT_WHITE_BEAR) return bad("bad fmt");
    p->fmt = d->fmt;
    if (d->precision != PNP_PREC_FP64 && d->precision != PNP_PREC_FP32 && d->precision != PNP_PREC_DF64 &&
        d->precision != PNP_PREC_TF32SPLIT)
        return bad("bad precision");
    if (d->lin_tol < 0 || d->lin_tol >= 1) return bad("lin_tol must be in [0, 1)");
    if (d->nsites < 0 || (d->nsites > 0 && !d->site_xyz)) return bad("sites missing");
    if (d->quad_nmu < 0 || d->quad_ntheta < 0 || d->quad_nr < 0 || d->well_nmu < 0 || d->well_ntheta < 0 ||
        d->well_nr < 0 || d->quad_nmu > 256 || d->quad_ntheta > 512 || d->quad_nr > 256 || d->well_nmu > 256 ||
        d->well_ntheta > 512 || d->well_nr > 256)
        return bad("quadrature counts out of range");
    p->nx = d->nx; p->ny = d->ny; p->nz = d->nz;
    for (int c = 0; c < 3; ++c) p->bc[c] = d->bc[c];
    p->s = d->nspecies;
    p->q.assign(d->valence, d->valence + p->s);
    p->R.assign(d->radius, d->radius + p->s);
    p->rho_b.assign(d->rho_bulk, d->rho_bulk + p->s);
    p->D.assign(p->s, 1.0);
    if (d->diffusivity) p->D.assign(d->diffusivity, d->diffusivity + p->s);
    p->depth.assign(p->s, 0.0);
    if (d->well_depth) p->depth.assign(d->well_depth, d->well_depth + p->s);
    for (int i = 0; i < p->s; ++i) {
        if (!(p->R[i] > 0 && p->R[i] <= 64)) return bad("radius must be in (0, 64]");
        if (!(p->rho_b[i] >= 0) || !std::isfinite(p->rho_b[i])) return bad("rho_bulk must be finite and >= 0");
        if (!(p->D[i] > 0) || !std::isfinite(p->D[i])) return bad("diffusivity must be > 0");
        if (!std::isfinite(p->depth[i])) return bad("well depth must be finite");
        if (std::abs(p->q[i]) > 16) return bad("valence out of range");
    }
    p->has_wells = false;
    for (int i = 0; i < p->s; ++i)
        if (p->depth[i] != 0.0) p->has_wells = true;
    if (d->nsites == 0) p->has_wells = false;
    p->well_inner = d->well_inner;
    p->well_outer = d->well_outer;
    if (p->has_wells) {
        if (!(d->well_outer > d->well_inner && d->well_inner >= 0 && d->well_outer <= 64))
            return bad("well radii must satisfy 0 <= inner < outer <= 64");
        if (!(d->site_alpha > 0)) return bad("site_alpha must be > 0");
    }
    p->sites.assign(d->site_xyz, d->site_xyz + 3 * (size_t)d->nsites);
    for (double v : p->sites)
        if (!std::isfinite(v)) return bad("non-finite site coordinate");
    p->site_alpha = d->site_alpha;
    p->rho_f.clear();
    if (d->rho_fixed) {
        p->rho_f.assign(d->rho_fixed, d->rho_fixed + p->npts());
        for (double v : p->rho_f)
            if (!std::isfinite(v)) return bad("non-finite fixed charge");
    }
    p->temperature_K = d->temperature_K;
    p->eps_r = d->eps_r;
    p->h_nm = d->h_nm;
    p->lB = bjerrum_length_h(d->temperature_K, d->eps_r, d->h_nm);
    p->phi_lo = d->phi_lo;
    p->phi_hi = d->phi_hi;
    p->lambda_phi = d->lambda_phi;
    p->lambda_rho = d->lambda_rho;
    p->rho_mix = d->rho_mix;
    p->tol = d->tol;
    p->max_iter = d->max_iter;
    p->eq_init = eq;
    p->screened = (d->flags & PNP_FLAG_SCREENED_POISSON) != 0;
    p->msa = (d->flags & PNP_FLAG_MSA) != 0;
    p->phase_timing = (d->flags & PNP_FLAG_PHASE_TIMING) != 0;
    if (d->anderson_depth < 0 || d->anderson_depth > 6) return bad("anderson_depth must be in 0..6");
    if (d->anderson_depth > 0 && d->rho_mix == PNP_MIX_ADAPTIVE)
        return bad("Anderson mixing needs a relaxation without per-point state (not PNP_MIX_ADAPTIVE)");
    p->aa_depth = d->anderson_depth;
    p->eq_tol = d->eq_tol > 0 ? d->eq_tol : 1e-6;
    p->eq_max_iter = d->eq_max_iter > 0 ? d->eq_max_iter : 1000;
    p->quad[0] = d->quad_nmu; p->quad[1] = d->quad_ntheta; p->quad[2] = d->quad_nr;
    p->wquad[0] = d->well_nmu; p->wquad[1] = d->well_ntheta; p->wquad[2] = d->well_nr;
    p->sw_half = d->sw_half ? 1 : 0;
    p->precision = d->precision;
    p->lin_tol = d->lin_tol;      // 0: adaptive inner tolerance
    bulk_mu_fmt(*p, p->mu_bulk);
    double n3 = 0;
    for (int i = 0; i < p->s; ++i) n3 += p->rho_b[i] * 4.0 * M_PI * std::pow(p->R[i], 3) / 3.0;
    if (!(n3 < 1.0)) return bad("bulk packing fraction must be < 1");
    return plan_lengths(p, d->fft_len);
}

// register-FFT lengths of the mu_ex kernels
static const int kRegLengths[] = {16, 20, 24, 32, 40, 48, 64, 80, 96, 128, 256};

void length_candidates(const Problem *p, int c, std::vector<int> *out) {
    out->clear();
    const int n[3] = {p->nx, p->ny, p->nz};
    if (p->bc[c] == PNP_BC_PERIODIC) {
        out->push_back(n[c]);
        return;
    }
    const bool even = (c == 0);
    const int minL = n[c] + std::max(std::max(p->S, p->Ssw), p->Smsa);
    const int L0 = next_smooth(minL, even);
    out->push_back(L0);
    int extra = 0;
    for (int f : kRegLengths)
        if (f > L0 && f <= L0 + (6 * L0) / 10 && extra < 2) {
            out->push_back(f);
            ++extra;
        }
    if (std::find(out->begin(), out->end(), p->L[c]) == out->end()) out->push_back(p->L[c]);
    std::sort(out->begin(), out->end());
}

int plan_lengths(Problem *p, const int fft_len[3]) {
    double Rmax = 0;
    for (double r : p->R) Rmax = std::max(Rmax, r);
    p->S = (int)std::ceil(Rmax) + 1;
    p->Ssw = p->has_wells ? (int)std::ceil(p->well_outer) + 1 : 0;
    // the MSA pair kernels reach R_i + R_j
    p->Smsa = p->msa ? (int)std::ceil(2.0 * Rmax) + 1 : 0;
    int need = std::max(std::max(p->S, p->Ssw), p->Smsa);
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int c = 0; c < 3; ++c) {
        bool even = (c == 0);
        int L;
        if (p->bc[c] == PNP_BC_PERIODIC) {
            if (!smooth235(n[c]) || (even && n[c] % 2)) return PNP_ERR_INVALID;
            L = n[c];
            if (fft_len && fft_len[c] > 0 && fft_len[c] != L) return PNP_ERR_INVALID;
        } else {
            int minL = n[c] + need;
            if (fft_len && fft_len[c] > 0) {
                L = fft_len[c];
                if (L < minL || !smooth235(L) || (even && L % 2)) return PNP_ERR_INVALID;
            } else {
                // smallest legal length, or a register-FFT length when one is
                // within 30% of it
                L = next_smooth(minL, even);
                for (int f : kRegLengths)
                    if (f >= minL && f <= L + (3 * L) / 10 && f >= L) {
                        L = f;
                        break;
                    }
            }
        }
        if (L > 4096) return PNP_ERR_INVALID;
        p->L[c] = L;
        p->ax[c] = make_axis(L);
    }
    return PNP_OK;
}

}  // namespace pnp
