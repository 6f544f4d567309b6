// Internal declarations of libpnp_gb300 (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pnp.h"

namespace pnp {

constexpr int kNumWeighted = 10;   // n0, n1, n2, n3, n1x, n1y, n1z, n2x, n2y, n2z (Sec 2.3.1)
constexpr int kNumKernels = 5;     // per species: shell, ball, vector shell x, y, z
constexpr int kMaxStages = 16;

// Mixed-radix (4, 2, 3, 5) Stockham plan of one axis.
struct FftAxis {
    int L;
    int nst;
    int radix[kMaxStages];
};

bool smooth235(int n);
int next_smooth(int n, bool even);
FftAxis make_axis(int L);

// Quadrature stencil on [-S, S]^3, stored [mz][my][mx] (Sec 3.5 reading).
struct Stencil {
    int S = 0;
    std::vector<double> K;   // (2S+1)^3
    double &at(int mx, int my, int mz) {
        int w = 2 * S + 1;
        return K[((size_t)(mz + S) * w + (my + S)) * w + (mx + S)];
    }
};

struct DeviceBuffers;   // per-precision device state of the mu_ex pipeline

// scoped NVTX range (tracing tools show the library's phases on the timeline)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kNumStages = 9;
struct StageTimer {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;          // free events
    std::vector<int> stage;                 // stage id of each recorded pair
    std::vector<cudaEvent_t> ev0, ev1;      // recorded pairs
    cudaEvent_t get();
    void begin(int s, cudaStream_t st);
    void end(cudaStream_t st);
    int collect(double *ms, int *launches, int max);
    void release();
};
struct GummelState;     // device state of the Gummel solve

struct Problem {
    // ---- descriptor (copied) ----
    int nx = 0, ny = 0, nz = 0;
    int bc[3] = {0, 0, 0};
    int s = 0;
    std::vector<int> q;
    std::vector<double> R, rho_b, D, depth;
    double well_inner = 0, well_outer = 0;
    std::vector<double> sites;
    double site_alpha = 1.0;
    std::vector<double> rho_f;
    double temperature_K = 300, eps_r = 16.6, h_nm = 1.0, lB = 0;
    double phi_lo = 0, phi_hi = 0, lambda_phi = 0.3, lambda_rho = 0.3;
    int rho_mix = 0;
    double tol = 1e-8;
    int max_iter = 500;
    bool eq_init = false;             // equilibrium initial guess before the Gummel loop
    bool screened = false;            // Gummel Poisson step as one screened Newton step
    int fmt = 0;                      // PNP_FMT_ROSENFELD or PNP_FMT_WHITE_BEAR
    double eq_tol = 1e-6;
    int eq_max_iter = 1000;
    int quad[3] = {0, 0, 0}, wquad[3] = {0, 0, 0};
    int sw_half = 1;
    int precision = 0;
    double lin_tol = 0.0;             // 0: adaptive inner tolerance
    bool has_wells = false;
    bool msa = false;                 // mu_ex carries the MSA correlation term (Sec 2.3.4)
    int aa_depth = 0;                 // Anderson mixing depth of the Gummel loop (0: relaxed only)
    bool phase_timing = false;        // the solve graph marks its phase boundaries

    // ---- plan ----
    int L[3] = {0, 0, 0};
    int S = 0, Ssw = 0, Smsa = 0;     // stencil half-widths: FMT, square well, MSA pair kernels
    FftAxis ax[3];
    std::vector<double> mu_bulk;      // reservoir mu_ex (bulk Rosenfeld)

    // ---- device ----
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t last_stream = nullptr;
    int *d_flag = nullptr;            // device status bits
    double *d_U = nullptr;            // square-well field sum_m K_sw[m] rho_s(r+m)
    std::vector<double> sh_coef;      // mu_sh,i = sh_coef[i] * U
    double *d_E = nullptr;            // [s][N] MSA bulk field sum_j rho_b,j (C_ij (x) 1_Omega)
    double *d_sh_coef = nullptr;
    DeviceBuffers *buf[3] = {nullptr, nullptr, nullptr};   // FP64, FP32, double-float
    void *d_work = nullptr;           // shared FFT workspace
    size_t work_bytes = 0;
    double *d_io = nullptr;           // staging for host-pointer calls (s+1 fields)
    GummelState *gs = nullptr;
    size_t device_bytes = 0;
    int deferred = 0;                 // host-side deferred status
    StageTimer timer;
    int mg_levels = 0;
    int tile[3] = {0, 0, 0};          // register-FFT CTA tiles (x lines, y columns, z columns); 0: rule
    double tuned_ms = 0;              // mu_ex time measured by the autotuner

    size_t npts() const { return (size_t)nx * ny * nz; }
};

// plan.cpp
int validate_and_copy(const pnp_problem_desc *d, Problem *p, std::string *why);
int plan_lengths(Problem *p, const int fft_len[3]);
void length_candidates(const Problem *p, int axis, std::vector<int> *out);
void gauss_legendre_nodes(int n, std::vector<double> &x, std::vector<double> &w);
void build_fmt_stencils(double R, int nmu, int ntheta, int nr, int S, Stencil out[kNumKernels]);
void build_well_stencil(double r_in, double r_out, int nmu, int ntheta, int nr, int S, Stencil &out);
void build_msa_stencil(double qq_lB, double B, double sigma, int nmu, int ntheta, int nr, int S, Stencil &out);
double msa_B(double xi);
// MSA pair kernels of a problem: pair index of (i, j), i <= j, in the packed
// upper triangle; count s (s + 1) / 2
__host__ __device__ inline int msa_pair(int i, int j, int s) {
    if (i > j) { const int t = i; i = j; j = t; }
    return i * s - i * (i - 1) / 2 + (j - i);
}
void build_msa_pair(const Problem &p, int i, int j, Stencil &out);   // C_ij on its own reach
void octant_transform(const Stencil &st, const int L[3], const bool odd[3], double scale, double *out);
double bjerrum_length_h(double T, double eps_r, double h_nm);
double conductivity_unit_S_per_cm(double T, double h_nm, double D_m2_per_s);
void bulk_mu_fmt(const Problem &p, std::vector<double> &mu);

// ypass_tc.cu: a kernel whose bounded mbarrier wait nothing completes
int bounded_wait_probe(double limit_ms);

// autotune.cu: time candidate padded lengths and tiles, keep the fastest
int autotune_create(const pnp_problem_desc *desc, Problem **out, std::string *why);

// mu_ex.cu
int mu_ex_setup(Problem *p);                 // workspace, spectra, mu_sh
int mu_ex_prepare(Problem *p, int prec);     // lazily build one precision's buffers
int mu_ex_enqueue(Problem *p, int prec, const double *d_rho, double *d_mu, cudaStream_t st);
void mu_ex_free(Problem *p);
// F_sh (Sec 2.3.2) of device densities into d_out[0] (d_part: 512 doubles)
int square_well_energy_enqueue(Problem *p, const double *d_rho, double *d_out, double *d_part, cudaStream_t st);

// gummel.cu
int gummel_setup(Problem *p);
int gummel_run(Problem *p, const double *d_phi0, const double *d_rho0, double *d_phi, double *d_rho,
               pnp_stats *stats, cudaStream_t st);
void gummel_free(Problem *p);
int plane_flux(Problem *p, int species, const double *d_phi, const double *d_mu, const double *d_rho,
               double *d_flux, cudaStream_t st);
int gummel_launch(Problem *p, const double *d_phi0, const double *d_rho0, cudaStream_t st);
int gummel_fetch(Problem *p, double *phi, double *rho, void *dev_stats_copy, cudaStream_t st);
size_t gummel_stats_bytes();
int gummel_phase_times(Problem *p, double *ms, int max_phases);   // ms per phase of the last solve
void gummel_decode_stats(const void *raw, pnp_stats *out);
size_t estimate_device_bytes(const Problem &p);   // problem + Gummel state, from the plan

// api.cpp helpers
int cuda_status(cudaError_t e);
// Device allocations of a problem are stream-ordered (cudaMallocAsync on the
// problem's stream, completed before return; cudaFreeAsync), so freeing one
// problem never waits for work of the others.
cudaError_t dmalloc(void **ptr, size_t bytes, cudaStream_t st);
// caller arrays: kind 0 finite, 1 >= 0 and finite, 2 > 0 and finite
bool host_values_ok(const double *x, size_t n, int kind);
void dfree(void *ptr, cudaStream_t st);
int create_problem_internal(const pnp_problem_desc *desc, Problem **out, std::string *why);
void destroy_problem_internal(Problem *p);

// device status bits
enum : int { kFlagPacking = 1, kFlagOverflow = 2, kFlagNonFinite = 4, kFlagTimeout = 8 };

}  // namespace pnp

struct pnp_problem {
    pnp::Problem *impl;
};
