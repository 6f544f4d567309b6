// C ABI of libpnp_gb300 (include/pnp.h): argument checking, device state
// lifetime, host<->device staging and error mapping.
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>
#include <mutex>
#include <new>
#include <string>

#include "pnp_internal.h"

namespace pnp {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PNP_OK;
    if (e == cudaErrorMemoryAllocation) return PNP_ERR_NOMEM;
    return PNP_ERR_CUDA;
}

// Test hook, armed only through the test entry point pnp_test_fail_alloc_at:
// the k-th device allocation after arming (1-based) reports
// cudaErrorMemoryAllocation on the host without calling CUDA, so the error
// paths of every allocation site can be driven without exhausting or faulting
// a GPU.  Inert unless a caller arms it explicitly.
static std::atomic<long> g_fail_alloc_at{0};
static std::atomic<long> g_alloc_count{0};

static bool injected_alloc_failure() {
    const long at = g_fail_alloc_at.load();
    if (at <= 0) return false;
    return g_alloc_count.fetch_add(1) + 1 == at;
}

cudaError_t dmalloc(void **ptr, size_t bytes, cudaStream_t st) {
    if (injected_alloc_failure()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    static std::once_flag pool_once[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64)
        std::call_once(pool_once[dev], [dev] {
            // keep freed blocks in the pool instead of returning them at each sync
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t keep = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
        });
    cudaError_t e = cudaMallocAsync(ptr, bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        // an allocation failure is not sticky: clear it so the next launch's
        // status check does not report it again
        if (e == cudaErrorMemoryAllocation) cudaGetLastError();
        *ptr = nullptr;
    }
    return e;
}

// Checks of caller arrays on the host: branch-free scans (no early exit, so
// the compiler can vectorise them), split over threads for large arrays.
// kind 0: finite; 1: >= 0 and finite; 2: > 0 and finite (NaN fails every one).
static bool scan_values(const double *x, size_t n, int kind) {
    bool ok = true;
    const double big = std::numeric_limits<double>::max();
    if (kind == 0)
        for (size_t k = 0; k < n; ++k) ok &= (x[k] >= -big) & (x[k] <= big);
    else if (kind == 1)
        for (size_t k = 0; k < n; ++k) ok &= (x[k] >= 0.0) & (x[k] <= big);
    else
        for (size_t k = 0; k < n; ++k) ok &= (x[k] > 0.0) & (x[k] <= big);
    return ok;
}

bool host_values_ok(const double *x, size_t n, int kind) {
    const size_t kMinPerThread = (size_t)1 << 19;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned T = (unsigned)std::min<size_t>(std::min(hw, 16u), std::max<size_t>(1, n / kMinPerThread));
    if (T <= 1) return scan_values(x, n, kind);
    std::vector<std::thread> th;
    std::vector<char> ok(T, 1);
    const size_t chunk = (n + T - 1) / T;
    for (unsigned t = 0; t < T; ++t) {
        const size_t a = t * chunk, b = std::min(n, a + chunk);
        th.emplace_back([&, t, a, b] { ok[t] = a < b ? scan_values(x + a, b - a, kind) : 1; });
    }
    for (auto &h : th) h.join();
    for (char v : ok)
        if (!v) return false;
    return true;
}

void dfree(void *ptr, cudaStream_t st) {
    if (ptr) cudaFreeAsync(ptr, st);
}

void destroy_problem_internal(Problem *p) {
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    gummel_free(p);
    mu_ex_free(p);
    dfree(p->d_flag, p->stream);
    dfree(p->d_io, p->stream);
    dfree(p->d_sh_coef, p->stream);
    if (p->stream) cudaStreamDestroy(p->stream);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

int create_problem_internal(const pnp_problem_desc *desc, Problem **out, std::string *why) {
    if (desc && (desc->flags & PNP_FLAG_AUTOTUNE)) return autotune_create(desc, out, why);
    NvtxRange range("create_problem");
    Problem *p = new (std::nothrow) Problem();
    if (!p) return PNP_ERR_NOMEM;
    int rc = validate_and_copy(desc, p, why);
    if (rc) {
        delete p;
        return rc;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = dmalloc((void **)&p->d_flag, sizeof(int), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_flag, 0, sizeof(int), p->stream);
    if (e != cudaSuccess) {
        rc = cuda_status(e);
        destroy_problem_internal(p);
        return rc;
    }
    p->last_stream = p->stream;
    rc = mu_ex_setup(p);
    if (rc == PNP_OK) rc = cuda_status(cudaStreamSynchronize(p->stream));
    if (rc) {
        destroy_problem_internal(p);
        return rc;
    }
    *out = p;
    return PNP_OK;
}

static int read_flag(Problem *p, cudaStream_t st) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (h) {
        cudaMemsetAsync(p->d_flag, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
    }
    if (h & kFlagTimeout) return PNP_ERR_TIMEOUT;
    if (h & kFlagOverflow) return PNP_ERR_OVERFLOW;
    if (h & (kFlagPacking | kFlagNonFinite)) return PNP_ERR_PACKING;
    return PNP_OK;
}

static int resolve_prec(const Problem *p, int prec) {
    if (prec == PNP_PREC_DEFAULT) return p->precision;
    if (prec == PNP_PREC_FP64 || prec == PNP_PREC_FP32 || prec == PNP_PREC_DF64 || prec == PNP_PREC_TF32SPLIT)
        return prec;
    return -100;
}

}  // namespace pnp

using namespace pnp;

extern "C" {

int pnp_desc_init(pnp_problem_desc *d) {
    if (!d) return PNP_ERR_INVALID;
    std::memset(d, 0, sizeof(*d));
    d->lambda_phi = 0.3;
    d->lambda_rho = 0.3;
    d->rho_mix = PNP_MIX_LINEAR;
    d->tol = 1e-8;
    d->max_iter = 500;
    d->sw_half = 1;
    d->temperature_K = 300.0;
    d->eps_r = 16.6;
    d->h_nm = 1.0;
    d->site_alpha = 1.0;
    d->precision = PNP_PREC_FP64;
    return PNP_OK;
}

int pnp_create_problem(const pnp_problem_desc *desc, pnp_problem **out) {
    if (!desc || !out) return PNP_ERR_INVALID;
    *out = nullptr;
    Problem *impl = nullptr;
    std::string why;
    int rc = create_problem_internal(desc, &impl, &why);
    if (rc) return rc;
    pnp_problem *h = new (std::nothrow) pnp_problem{impl};
    if (!h) {
        destroy_problem_internal(impl);
        return PNP_ERR_NOMEM;
    }
    *out = h;
    return PNP_OK;
}

void pnp_destroy_problem(pnp_problem *p) {
    if (!p) return;
    destroy_problem_internal(p->impl);
    delete p;
}

int pnp_get_problem_info(const pnp_problem *h, pnp_problem_info *info) {
    if (!h || !info) return PNP_ERR_INVALID;
    const Problem *p = h->impl;
    for (int c = 0; c < 3; ++c) info->fft_len[c] = p->L[c];
    info->stencil_halfwidth = p->S;
    info->well_halfwidth = p->Ssw;
    info->device_bytes = p->device_bytes;
    info->mg_levels = p->mg_levels;
    for (int c = 0; c < 3; ++c) info->tile[c] = p->tile[c];
    info->tuned_ms = p->tuned_ms;
    info->bjerrum_h = p->lB;
    return PNP_OK;
}

int pnp_plan_problem(const pnp_problem_desc *desc, pnp_problem_info *info, double *mu_reservoir) {
    if (!desc || !info) return PNP_ERR_INVALID;
    Problem p;
    std::string why;
    const int rc = validate_and_copy(desc, &p, &why);
    if (rc) return rc;
    std::memset(info, 0, sizeof(*info));
    for (int c = 0; c < 3; ++c) info->fft_len[c] = p.L[c];
    info->stencil_halfwidth = p.S;
    info->well_halfwidth = p.Ssw;
    info->device_bytes = estimate_device_bytes(p);
    info->bjerrum_h = p.lB;
    if (mu_reservoir)
        for (int i = 0; i < p.s; ++i) mu_reservoir[i] = p.mu_bulk[i];
    return PNP_OK;
}

int pnp_conductivity(const pnp_problem_desc *desc, const double *flux, double D_m2_per_s, double *sigma) {
    if (!desc || !flux || !sigma || !(D_m2_per_s >= 0.0) || !std::isfinite(D_m2_per_s)) return PNP_ERR_INVALID;
    Problem p;
    std::string why;
    const int rc = validate_and_copy(desc, &p, &why);
    if (rc) return rc;
    const double dphi = p.phi_hi - p.phi_lo;
    if (p.bc[2] != PNP_BC_DIRICHLET || dphi == 0.0) return PNP_ERR_INVALID;
    const int faces = p.nz + 1;
    if (!host_values_ok(flux, (size_t)p.s * faces, 0)) return PNP_ERR_INVALID;
    // mean over the faces of the charge current through a plane
    double sum = 0.0;
    for (int k = 0; k < faces; ++k) {
        double c = 0.0;
        for (int i = 0; i < p.s; ++i) c += p.q[i] * flux[(size_t)i * faces + k];
        sum += c;
    }
    const double current = sum / faces / ((double)p.nx * p.ny);   // per unit area (h^2)
    const double field = -dphi / faces;                           // kT/e per h
    sigma[0] = current / field;
    sigma[1] = sigma[0] * conductivity_unit_S_per_cm(p.temperature_K, p.h_nm, D_m2_per_s);
    return PNP_OK;
}

int pnp_weight_stencil(int kind, double r_in, double r_out, int nmu, int ntheta, int nr, int S, double *out) {
    if (!out || kind < 0 || kind > 5 || !(r_out > 0) || nmu < 0 || ntheta < 0 || nr < 0 || S < 1 || S > 64)
        return PNP_ERR_INVALID;
    if ((int)std::ceil(r_out) + 1 > S || (kind == 5 && !(r_in >= 0 && r_in < r_out))) return PNP_ERR_INVALID;
    Stencil st;
    if (kind == 5) {
        build_well_stencil(r_in, r_out, nmu, ntheta, nr, S, st);
    } else {
        Stencil fmt[kNumKernels];
        build_fmt_stencils(r_out, nmu, ntheta, nr, S, fmt);
        st = fmt[kind];
    }
    std::memcpy(out, st.K.data(), sizeof(double) * st.K.size());
    return PNP_OK;
}

int pnp_msa_stencil(const pnp_problem_desc *desc, int i, int j, int S, double *out) {
    if (!desc || !out) return PNP_ERR_INVALID;
    Problem p;
    std::string why;
    const int rc = validate_and_copy(desc, &p, &why);
    if (rc) return rc;
    if (i < 0 || j < 0 || i >= p.s || j >= p.s) return PNP_ERR_INVALID;
    const double sigma = p.R[i] + p.R[j];
    if (S < (int)std::ceil(sigma) + 1 || S > 64) return PNP_ERR_INVALID;
    double kappa2 = 0.0;
    for (int k = 0; k < p.s; ++k) kappa2 += 4.0 * M_PI * p.lB * p.rho_b[k] * p.q[k] * p.q[k];
    const double B = msa_B(std::sqrt(kappa2) * sigma);
    Stencil st;
    build_msa_stencil((double)p.q[i] * p.q[j] * p.lB, B, sigma, p.quad[0], p.quad[1], p.quad[2], S, st);
    std::memcpy(out, st.K.data(), sizeof(double) * st.K.size());
    return PNP_OK;
}

int pnp_weight_spectrum(int kind, double r_in, double r_out, int nmu, int ntheta, int nr, int S, int Lx, int Ly,
                        int Lz, double *out) {
    if (!out || Lx < 2 * S + 1 || Ly < 2 * S + 1 || Lz < 2 * S + 1 || Lx > 4096 || Ly > 4096 || Lz > 4096)
        return PNP_ERR_INVALID;
    const int W = 2 * S + 1;
    std::vector<double> k((size_t)W * W * W);
    const int rc = pnp_weight_stencil(kind, r_in, r_out, nmu, ntheta, nr, S, k.data());
    if (rc) return rc;
    Stencil st;
    st.S = S;
    st.K = k;
    const int L[3] = {Lx, Ly, Lz};
    const bool odd[3] = {kind == 2, kind == 3, kind == 4};
    octant_transform(st, L, odd, 1.0, out);
    return PNP_OK;
}

int pnp_excess_mu(pnp_problem *h, const double *rho, double *mu_ex, int precision) {
    if (!h || !rho || !mu_ex) return PNP_ERR_INVALID;
    Problem *p = h->impl;
    int prec = resolve_prec(p, precision);
    if (prec < 0) return PNP_ERR_INVALID;
    const size_t n = p->npts() * p->s;
    if (!host_values_ok(rho, n, 1)) return PNP_ERR_INVALID;
    if (!p->d_io) {
        if (dmalloc((void **)&p->d_io, sizeof(double) * (2 * n + p->npts()), p->stream) != cudaSuccess)
            return PNP_ERR_NOMEM;
        p->device_bytes += sizeof(double) * (2 * n + p->npts());
    }
    cudaStream_t st = p->stream;
    p->last_stream = st;
    cudaError_t e = cudaMemcpyAsync(p->d_io, rho, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e);
    int rc = mu_ex_enqueue(p, prec, p->d_io, p->d_io + n, st);
    if (rc) return rc;
    e = cudaMemcpyAsync(mu_ex, p->d_io + n, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e);
    return read_flag(p, st);
}

int pnp_excess_mu_device(pnp_problem *h, const double *d_rho, double *d_mu_ex, int precision, void *stream) {
    if (!h || !d_rho || !d_mu_ex) return PNP_ERR_INVALID;
    Problem *p = h->impl;
    int prec = resolve_prec(p, precision);
    if (prec < 0) return PNP_ERR_INVALID;
    cudaStream_t st = stream ? (cudaStream_t)stream : p->stream;
    p->last_stream = st;
    return mu_ex_enqueue(p, prec, d_rho, d_mu_ex, st);
}

int pnp_status(pnp_problem *h) {
    if (!h) return PNP_ERR_INVALID;
    Problem *p = h->impl;
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    int rc = p->deferred;
    p->deferred = 0;
    int f = read_flag(p, p->last_stream);
    return rc ? rc : f;
}

int pnp_gummel_solve(pnp_problem *h, const double *phi0, const double *rho0, double *phi_out, double *rho_out,
                     pnp_stats *stats) {
    if (stats) *stats = pnp_stats{};
    auto fail = [&](int code) {
        if (stats) stats->status = code;
        return code;
    };
    if (!h) return fail(PNP_ERR_INVALID);
    Problem *p = h->impl;
    auto t0 = std::chrono::steady_clock::now();
    const size_t N = p->npts(), n = N * p->s;
    if (rho0 && !host_values_ok(rho0, n, 2)) return fail(PNP_ERR_INVALID);
    if (phi0 && !host_values_ok(phi0, N, 0)) return fail(PNP_ERR_INVALID);
    if (!p->d_io) {
        if (dmalloc((void **)&p->d_io, sizeof(double) * (2 * n + N), p->stream) != cudaSuccess)
            return fail(PNP_ERR_NOMEM);
        p->device_bytes += sizeof(double) * (2 * n + N);
    }
    cudaStream_t st = p->stream;
    p->last_stream = st;
    double *d_rho = p->d_io, *d_phi = p->d_io + n, *d_rho0 = nullptr, *d_phi0 = nullptr;
    cudaError_t e = cudaSuccess;
    if (rho0) {
        e = cudaMemcpyAsync(d_rho, rho0, sizeof(double) * n, cudaMemcpyHostToDevice, st);
        d_rho0 = d_rho;
    }
    if (phi0 && e == cudaSuccess) {
        e = cudaMemcpyAsync(d_phi, phi0, sizeof(double) * N, cudaMemcpyHostToDevice, st);
        d_phi0 = d_phi;
    }
    if (e != cudaSuccess) return fail(cuda_status(e));
    pnp_stats local{};
    int rc = gummel_run(p, d_phi0, d_rho0, d_phi, d_rho, &local, st);
    if (rc == PNP_OK || rc == PNP_ERR_NOT_CONVERGED) {
        if (phi_out) e = cudaMemcpyAsync(phi_out, d_phi, sizeof(double) * N, cudaMemcpyDeviceToHost, st);
        if (rho_out && e == cudaSuccess)
            e = cudaMemcpyAsync(rho_out, d_rho, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_status(e);
    }
    local.status = rc;
    local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = local;
    return rc;
}

int pnp_stage_timing(pnp_problem *h, int enable) {
    if (!h) return PNP_ERR_INVALID;
    h->impl->timer.enabled = enable != 0;
    return PNP_OK;
}

int pnp_stage_times(pnp_problem *h, double *ms, int *launches, int max_stages) {
    if (!h || max_stages < 0) return PNP_ERR_INVALID;
    return h->impl->timer.collect(ms, launches, max_stages);
}

const char *pnp_stage_name(int stage) {
    static const char *names[kNumStages] = {"x_fwd", "y_fwd", "z_mac", "y_inv", "x_fused",
                                            "y_fwd_psi", "z_back", "y_inv_mu", "x_inv"};
    if (stage < 0 || stage >= kNumStages) return "";
    return names[stage];
}

int pnp_plane_flux(pnp_problem *h, int species, const double *phi, const double *rho, double *flux) {
    if (!h || !phi || !rho || !flux) return PNP_ERR_INVALID;
    Problem *p = h->impl;
    if (species < 0 || species >= p->s || p->bc[2] != PNP_BC_DIRICHLET) return PNP_ERR_INVALID;
    const size_t N = p->npts(), n = N * p->s;
    if (!host_values_ok(rho, n, 1) || !host_values_ok(phi, N, 0)) return PNP_ERR_INVALID;
    if (!p->d_io) {
        if (dmalloc((void **)&p->d_io, sizeof(double) * (2 * n + N), p->stream) != cudaSuccess)
            return PNP_ERR_NOMEM;
        p->device_bytes += sizeof(double) * (2 * n + N);
    }
    cudaStream_t st = p->stream;
    p->last_stream = st;
    double *d_rho = p->d_io, *d_phi = p->d_io + n, *d_mu = p->d_io + n + N, *d_flux = nullptr;
    cudaError_t e = dmalloc((void **)&d_flux, sizeof(double) * (p->nz + 1), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rho, rho, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_phi, phi, sizeof(double) * N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_flag, 0, sizeof(int), st);
    int rc = cuda_status(e);
    if (rc == PNP_OK) rc = mu_ex_enqueue(p, PNP_PREC_FP64, d_rho, d_mu, st);
    if (rc == PNP_OK) rc = plane_flux(p, species, d_phi, d_mu + (size_t)species * N, d_rho + (size_t)species * N,
                                      d_flux, st);
    if (rc == PNP_OK)
        rc = cuda_status(cudaMemcpyAsync(flux, d_flux, sizeof(double) * (p->nz + 1), cudaMemcpyDeviceToHost, st));
    dfree(d_flux, st);
    const int f = read_flag(p, st);
    return rc ? rc : f;
}

int pnp_square_well_energy(pnp_problem *h, const double *rho, double *F_sh) {
    if (!h || !rho || !F_sh) return PNP_ERR_INVALID;
    Problem *p = h->impl;
    const size_t N = p->npts(), n = N * p->s;
    if (!host_values_ok(rho, n, 1)) return PNP_ERR_INVALID;
    *F_sh = 0.0;
    if (!p->has_wells) return PNP_OK;
    if (!p->d_io) {
        if (dmalloc((void **)&p->d_io, sizeof(double) * (2 * n + N), p->stream) != cudaSuccess)
            return PNP_ERR_NOMEM;
        p->device_bytes += sizeof(double) * (2 * n + N);
    }
    cudaStream_t st = p->stream;
    p->last_stream = st;
    // densities staged, then a fixed-order reduction against the well field
    // U = K_sw (x) rho_s built on the device at set-up
    double *d_rho = p->d_io, *d_red = nullptr;
    cudaError_t e = dmalloc((void **)&d_red, sizeof(double) * 520, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rho, rho, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    int rc = cuda_status(e);
    if (rc == PNP_OK) rc = square_well_energy_enqueue(p, d_rho, d_red, d_red + 8, st);
    double F = 0.0;
    if (rc == PNP_OK) rc = cuda_status(cudaMemcpyAsync(&F, d_red, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (rc == PNP_OK) rc = cuda_status(cudaStreamSynchronize(st));
    else cudaStreamSynchronize(st);
    dfree(d_red, st);
    if (rc) return rc;
    *F_sh = F;
    return PNP_OK;
}

int pnp_gummel_phase_times(pnp_problem *h, double *ms, int max_phases) {
    if (!h || !ms) return PNP_ERR_INVALID;
    return gummel_phase_times(h->impl, ms, max_phases);
}

int pnp_selftest_bounded_wait(double limit_ms) { return bounded_wait_probe(limit_ms); }

int pnp_test_fail_alloc_at(long k) {
    pnp::g_alloc_count.store(0);
    pnp::g_fail_alloc_at.store(k > 0 ? k : 0);
    return PNP_OK;
}

const char *pnp_error_string(int code) {
    switch (code) {
        case PNP_OK: return "ok";
        case PNP_PENDING: return "pending";
        case PNP_ERR_INVALID: return "invalid argument or descriptor";
        case PNP_ERR_NOMEM: return "out of memory";
        case PNP_ERR_CUDA: return "CUDA error";
        case PNP_ERR_NOT_CONVERGED: return "Gummel iteration did not converge";
        case PNP_ERR_PACKING: return "packing fraction n3 >= 1 or non-finite value in mu_ex";
        case PNP_ERR_OVERFLOW: return "Slotboom exponential overflow";
        case PNP_ERR_BUSY: return "server busy or request over the memory budget";
        case PNP_ERR_TIMEOUT: return "device wait timed out";
        case PNP_ERR_UNKNOWN_TICKET: return "unknown ticket";
        case PNP_ERR_TOO_LARGE: return "problem too large for the fixed scratch area";
        default: return "unknown error";
    }
}

}  // extern "C"
