/*
 * pnp.h -- C ABI of the GB300 PNP-cDFT library (libpnp_gb300.so).
 *
 * The library evaluates the cDFT excess chemical potentials of a mixture of
 * charged hard spheres on a uniform grid with zero-padded FFT convolutions, and
 * runs the relaxed Gummel iteration of the steady Poisson-Nernst-Planck system
 * around it on one GPU, following Meng, Zheng, Lin & Sushko, "Numerical
 * solution of 3D Poisson-Nernst-Planck equations coupled with classical density
 * functional theory ..." (arXiv:1407.0674).
 *
 * Conventions (all entry points):
 *  - Units are reduced: lengths in grid spacings h, densities in h^-3,
 *    potentials in kT/e, chemical potentials in kT.  The Bjerrum length is
 *    derived from temperature_K, eps_r and h_nm (Sec 2.3.3, Table 1).
 *  - Fields are C order [species][z][y][x] (x fastest), FP64 at the boundary
 *    for every precision variant.
 *  - Every pointer argument is owned by the caller.  Inputs are copied before
 *    the call returns; the library keeps no caller pointer.  Handles are opaque.
 *  - A pnp_problem is used by one host thread at a time.  A pnp_server is safe
 *    for concurrent pnp_submit / pnp_poll.
 *  - Errors are negative return codes (pnp_error_string gives a message); no
 *    entry point aborts the process.  Device faults surface as PNP_ERR_CUDA.
 *  - Entry points whose name ends in _device take device pointers and a
 *    cudaStream_t (passed as void*, NULL = the problem's own stream); they
 *    enqueue work and return without synchronising.  pnp_status() then
 *    synchronises and reports deferred device-side errors.
 */
#ifndef PNP_GB300_H
#define PNP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PNP_OK = 0,
    PNP_PENDING = 1,               /* pnp_poll: not finished yet */
    PNP_ERR_INVALID = -1,          /* bad argument or descriptor */
    PNP_ERR_NOMEM = -2,            /* device or host allocation failed */
    PNP_ERR_CUDA = -3,             /* CUDA runtime error */
    PNP_ERR_NOT_CONVERGED = -4,    /* Gummel reached max_iter */
    PNP_ERR_PACKING = -5,          /* n3 >= 1 or a non-finite value in mu_ex */
    PNP_ERR_OVERFLOW = -6,         /* Slotboom exponential overflowed (Sec 2.1) */
    PNP_ERR_BUSY = -7,             /* server: over the HBM budget or queue full */
    PNP_ERR_TIMEOUT = -8,          /* a bounded device wait gave up */
    PNP_ERR_UNKNOWN_TICKET = -9,   /* server: no such request */
    PNP_ERR_TOO_LARGE = -10        /* problem exceeds a fixed-size scratch area */
};

/* boundary type per axis.  For the cDFT integrals every non-periodic axis is
 * zero-extended (Sec 3.5).  The Gummel solve needs z = DIRICHLET and x, y
 * PERIODIC or NOFLUX (Sec 2.2, with the paper's y axis as z). */
enum { PNP_BC_PERIODIC = 0, PNP_BC_DIRICHLET = 1, PNP_BC_NOFLUX = 2 };

/* arithmetic of the FFT convolutions; the Gummel update, its norms and the
 * linear solves are FP64 in every variant, and so are the FMT derivatives
 * except that the FP32 and TF32SPLIT variants evaluate only their singular
 * functions of n3 (ln(1 - n3), the powers of 1/(1 - n3)) in FP64 and the
 * products with the other weighted densities in FP32.  PNP_PREC_DF64
 * carries each FFT value as an unevaluated sum of two FP32 numbers (about 48
 * significant bits) and runs the transforms on the FP32 pipes, which GB300
 * executes ~58x faster than FP64; it meets the FP64 accuracy bar of mu_ex.
 * PNP_PREC_TF32SPLIT is the FP32 variant with the y-axis transforms of length
 * 256 run as two radix-16 DFT stages on the tensor cores, each product split
 * into three TF32 products (hi*hi + lo*hi + hi*lo) accumulated in FP32; other
 * y lengths use the FP32 path. */
enum { PNP_PREC_DEFAULT = -1, PNP_PREC_FP64 = 0, PNP_PREC_FP32 = 1, PNP_PREC_DF64 = 2, PNP_PREC_TF32SPLIT = 3 };

/* descriptor flags.  PNP_FLAG_AUTOTUNE: pnp_create_problem (and the server's
 * admission of a request) times the mu_ex pipeline on the device for the
 * candidate padded lengths of each zero-extended axis (the smallest
 * 2^a 3^b 5^c length and the register-FFT lengths up to 60% above it) and for
 * the CTA tiles of the register-FFT kernels, and keeps the fastest plan; an
 * explicit fft_len entry is kept as given.  The choice is cached for the
 * process per (grid, boundaries, species count, stencil half-width, wells,
 * precision), so later problems of the same shape reuse it without timing.
 * Results do not depend on the tiles; another padded length changes mu_ex only
 * by rounding. */
#define PNP_FLAG_AUTOTUNE 1u

/* PNP_FLAG_EQUILIBRIUM_INIT: pnp_gummel_solve (without a warm start) first
 * solves the static equilibrium of the mobile species in the electrodes'
 * potential and starts the Gummel iteration from it (Sec 3.2, choice of
 * initial guess).  Equilibrium: rho_i = rho_b,i exp(mu_b,i - mu_ex,i - q_i phi)
 * with phi from the Poisson equation of these densities.  Each iteration
 * takes mu_ex from rho, one Newton step of that Poisson-Boltzmann equation in
 * phi (the Poisson operator plus the screening term 4 pi lB sum q^2 rho on
 * the diagonal, solved by the same multigrid-preconditioned CG; the step is
 * clamped to +-1 kT/e per point), and moves rho toward the Boltzmann
 * densities by the step-limited geometric relaxation with lambda_rho; it ends
 * when max(|dphi|, max_i |drho_i| / rho_b,i) < eq_tol or at eq_max_iter.
 * With this flag max_iter may be 0: the call then returns the equilibrium. */
#define PNP_FLAG_EQUILIBRIUM_INIT 2u

/* PNP_FLAG_SCREENED_POISSON: the Poisson step of each Gummel iteration keeps
 * the densities' first-order Boltzmann dependence on phi (Slotboom variables
 * and mu_ex frozen): one Newton step from the current phi,
 *   (A + diag 4 pi lB sum_i q_i^2 rho_i) dphi = 4 pi lB (rho_f + sum_i q_i rho_i) - A phi,
 * phi* = phi + dphi, then the usual relaxation.  Same fixed point as the
 * plain Poisson solve; the plain relaxed iteration is unstable once the box
 * is many Debye lengths long (the loop gain of its slowest charge mode grows
 * as lambda_phi lambda_rho kappa^2 / k^2), the screened one is not. */
#define PNP_FLAG_SCREENED_POISSON 4u

/* PNP_FLAG_MSA: mu_ex also carries the electrostatic correlations of the mean
 * spherical approximation (Sec 2.3.4):
 *   mu_el,i(r) = - sum_j int_Omega C_ij(|r - r'|) (rho_j(r') - rho_b,j) dr',
 *   C_ij(r) = -q_i q_j l_B [2B/s - (B/s)^2 r - 1/r] for r <= s, 0 beyond,
 *   s = R_i + R_j, B = [xi + 1 - sqrt(1 + 2 xi)] / xi, xi = kappa s,
 *   kappa^2 = 4 pi l_B sum_k rho_b,k q_k^2,
 * with the printed prefactor e^2/(k_B T eps) read as l_B.  The integral is
 * the ball quadrature of radius s (the FMT counts) deposited trilinearly on
 * the grid like the FMT weights, rho_j - rho_b,j zero off the domain.  The
 * bulk constant mu_el^bulk is not printed and is left out (a constant shift of
 * mu_i and of its reservoir value cancels in the Slotboom form).  Padded
 * lengths then also cover the MSA reach, ceil(2 max R) + 1.  Applied by every
 * mu_ex call and every Gummel iteration of the problem; not available through
 * pnp_excess_mu_noalloc (PNP_ERR_INVALID). */
#define PNP_FLAG_MSA 8u

/* PNP_FLAG_PHASE_TIMING (no counterpart in the paper): the solve graph also
 * marks the boundaries of the phases of every Gummel iteration with the GPU's
 * nanosecond global timer (one single-thread kernel per boundary) and sums
 * the time spent in each phase; pnp_gummel_phase_times reads the sums of the
 * last solve.  Results are unchanged; the marks add a few microseconds per
 * iteration. */
#define PNP_FLAG_PHASE_TIMING 16u

/* hard-sphere functional (Sec 2.3.1): Rosenfeld's, whose derivatives the
 * paper prints, or the White Bear (modified FMT) form it names beside it, in
 * which the n2^3 term carries phi3(n3) / (36 pi),
 * phi3(x) = [x + (1-x)^2 ln(1-x)] / [x^2 (1-x)^2], instead of
 * 1 / (24 pi (1 - n3)^2); its bulk limit is the Carnahan-Starling fluid. */
enum { PNP_FMT_ROSENFELD = 0, PNP_FMT_WHITE_BEAR = 1 };

/* density relaxation of the Gummel update (Sec 3.2): the printed linear form
 * rho <- l2 rho* + (1 - l2) rho, the geometric form rho <- rho (rho* / rho)^l2
 * (equal to first order, positive for large steps), or the geometric form
 * with its step in ln rho limited to +-0.2 per iteration (deep square wells
 * cannot push the packing fraction past 1 in one step; same fixed point);
 * PNP_MIX_ADAPTIVE is the step-limited form with a factor per point, halved
 * (down to lambda_rho / 1024) when the point's step in ln rho changes sign
 * from the previous iteration and grown by 10% (up to lambda_rho) otherwise:
 * densely packed points in deep wells, whose response is too stiff for one
 * global factor, stop alternating at the step limit. */
enum { PNP_MIX_LINEAR = 0, PNP_MIX_GEOMETRIC = 1, PNP_MIX_GEOMETRIC_LIMITED = 2, PNP_MIX_ADAPTIVE = 3 };

typedef struct {
    int nx, ny, nz;                /* grid points per axis */
    int bc[3];                     /* PNP_BC_* for x, y, z */
    int nspecies;                  /* mobile species s >= 1 */
    const int *valence;            /* [s] q_i (Sec 2.1) */
    const double *radius;          /* [s] hard-sphere radius R_i (h), Sec 2.3.1 */
    const double *rho_bulk;        /* [s] reservoir density (h^-3), Sec 2.2 */
    const double *diffusivity;     /* [s] D_i, NULL -> 1 */
    const double *well_depth;      /* [s] square-well depth eps_i (kT), NULL -> 0, Sec 2.3.2 */
    double well_inner, well_outer; /* square-well shell radii sigma_ab and gamma*sigma_ab (h) */
    int nsites;                    /* stationary sites (Sec 2.3.2) */
    const double *site_xyz;        /* [nsites][3] site centres in grid-index units */
    double site_alpha;             /* Gaussian exponent of the site density (h^-2) */
    const double *rho_fixed;       /* [nz][ny][nx] fixed charge (e h^-3), NULL -> 0 */
    double temperature_K, eps_r;   /* -> Bjerrum length (Sec 2.3.3) */
    double h_nm;                   /* grid spacing in nm */
    double phi_lo, phi_hi;         /* Dirichlet potentials on the z = 0 and z = top faces (kT/e) */
    double lambda_phi, lambda_rho; /* Gummel relaxation lambda_1, lambda_2 (Sec 3.2) */
    int rho_mix;                   /* PNP_MIX_* */
    double tol;                    /* stop when max(|dphi|, max_i |drho_i| / rho_b,i) < tol */
    int max_iter;                  /* Gummel iteration cap */
    int quad_nmu, quad_ntheta, quad_nr;   /* FMT quadrature counts, 0 = default rule */
    int well_nmu, well_ntheta, well_nr;   /* square-well quadrature counts, 0 = default */
    int sw_half;                   /* 1: mu_sh keeps the factor 1/2 of Sec 2.3.2 */
    int fft_len[3];                /* padded FFT length per axis, 0 = smallest legal */
    int precision;                 /* PNP_PREC_FP64 / FP32 / DF64 / TF32SPLIT: default for the calls below */
    double lin_tol;                /* relative residual ||r|| / ||b|| of the linear solves; 0 -> adaptive:
                                      min(1e-6, max(1e-12, 0.01 x previous Gummel residual)) */
    unsigned flags;                /* PNP_FLAG_* bits, 0 for none */
    double eq_tol;                 /* PNP_FLAG_EQUILIBRIUM_INIT: residual that ends the equilibrium stage
                                      (0 -> 1e-6) */
    int eq_max_iter;               /* and its iteration cap (0 -> 1000) */
    int fmt;                       /* hard-sphere functional, PNP_FMT_* */
    int anderson_depth;            /* 0: the relaxed Gummel iteration as printed (Sec 3.2); 1..6: that
                                      iteration accelerated by Anderson mixing of this depth (see
                                      pnp_gummel_solve); not with PNP_MIX_ADAPTIVE */
} pnp_problem_desc;

typedef struct {
    int status;                    /* PNP_OK or the error of the solve */
    int iterations;                /* Gummel iterations done */
    double residual;               /* last Gummel residual */
    long long linear_iterations;   /* PCG iterations summed over all solves */
    double seconds;                /* wall time of the call */
    int init_iterations;           /* iterations of the equilibrium initial guess (0 if not run) */
    double init_residual;          /* its last residual */
    int repeated_sweeps;           /* anderson_depth > 0: sweeps repeated from a restored or halved state after
                                      an unphysical one (not counted in iterations) */
} pnp_stats;

typedef struct {
    int fft_len[3];                /* padded lengths chosen */
    int stencil_halfwidth;         /* S of the FMT stencils (h) */
    int well_halfwidth;            /* S of the square-well stencil (h) */
    size_t device_bytes;           /* device memory held by the problem */
    int mg_levels;                 /* multigrid levels of the linear solves */
    int tile[3];                   /* CTA tiles of the register-FFT kernels (x lines, y and z
                                      columns per CTA) fixed by the autotuner; 0 = built-in rule */
    double tuned_ms;               /* mu_ex time the autotuner measured for the chosen plan, 0 if untuned */
    double bjerrum_h;              /* Bjerrum length e^2 / (4 pi eps0 eps_r kT) in units of h */
} pnp_problem_info;

typedef struct pnp_problem pnp_problem;
typedef struct pnp_server pnp_server;

/* Fill a descriptor with the defaults (all zero / NULL except lambda 0.3,
 * rho_mix LINEAR, tol 1e-8, max_iter 500, sw_half 1, temperature 300 K,
 * eps_r 16.6, h_nm 1, site_alpha 1).  Returns PNP_OK, or PNP_ERR_INVALID for NULL. */
int pnp_desc_init(pnp_problem_desc *desc);

/* Validate `desc`, plan the padded FFT lengths (each zero-extended axis needs
 * L >= n + S with S the stencil half-width, Sec 3.4), build the quadrature
 * stencils of Sec 3.5 and their spectra, the site field of Sec 2.3.2 and the
 * square-well potential mu_sh, and allocate the device state on the current
 * CUDA device.  On success *out owns all of it.
 * Errors: PNP_ERR_INVALID (descriptor), PNP_ERR_NOMEM, PNP_ERR_CUDA. */
int pnp_create_problem(const pnp_problem_desc *desc, pnp_problem **out);

/* Free everything a problem holds.  NULL is ignored. */
void pnp_destroy_problem(pnp_problem *p);

/* Report the plan of a problem. */
int pnp_get_problem_info(const pnp_problem *p, pnp_problem_info *info);

/* Validate and plan a descriptor on the host only (no device call): the padded
 * lengths the problem would use without the autotuner (Sec 3.4: L >= n + S on
 * every zero-extended axis, L = n on periodic ones), the stencil reaches and
 * the estimated device footprint into *info (mg_levels, tile and tuned_ms are
 * 0), and, when mu_reservoir is not NULL, the reservoir excess chemical
 * potentials mu_b,i of the bulk densities (nspecies values, kT) for the
 * descriptor's functional -- the Dirichlet data of the Nernst-Planck solves.
 * Errors: PNP_ERR_INVALID (descriptor rejected). */
int pnp_plan_problem(const pnp_problem_desc *desc, pnp_problem_info *info, double *mu_reservoir);

/* mu_ex,i = mu_hs,i + mu_sh,i (Sec 2.3, Eq. potential-energy-relation) for
 * the densities rho [s][nz][ny][nx] (host, FP64, >= 0).  Weighted densities
 * n_alpha (Sec 2.3.1) by zero-padded FFT correlation with the weight stencils,
 * the Rosenfeld derivatives dPhi/dn_alpha in FP64, masked to the domain, and
 * their back-convolution (Sec 2.3.1, Sec 3.4); plus the cached square-well
 * term (Sec 2.3.2).  Writes mu_ex [s][nz][ny][nx] (host).  Blocks until done.
 * Errors: PNP_ERR_INVALID, PNP_ERR_PACKING (n3 >= 1 somewhere), PNP_ERR_CUDA. */
int pnp_excess_mu(pnp_problem *p, const double *rho, double *mu_ex, int precision);

/* As pnp_excess_mu with device pointers, enqueued on `stream` (a
 * cudaStream_t, NULL = the problem's stream).  Does not synchronise; a
 * packing error is reported by the next pnp_status(). */
int pnp_excess_mu_device(pnp_problem *p, const double *d_rho, double *d_mu_ex, int precision,
                         void *stream);

/* mu_ex for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of pnp_excess_mu_device for a
 * host program whose GPU memory belongs to another allocator (for example a
 * framework whose caching allocator already holds nearly all of the device,
 * or a code that reserves its whole pool at start-up), or for a loop that
 * must not call cudaMalloc/cudaFree because they can synchronise the device.
 * It needs no pnp_problem: it validates `desc`, builds the FP64 spectra on the
 * host and runs the FP64 pipeline with every piece of device scratch taken
 * from one static 32 MiB array inside the library; it allocates no device
 * memory.  d_rho and d_mu_ex are device buffers [s][nz][ny][nx] owned by the
 * caller; `stream` is a cudaStream_t (NULL = the default stream).  Blocks
 * until the result is written.
 * Limits: hard spheres only (a descriptor with square wells is rejected with
 * PNP_ERR_INVALID); status word + twiddles + spectra + workspace must fit in
 * 32 MiB (about a 48^3 grid with three species zero-padded on every axis),
 * else PNP_ERR_TOO_LARGE.  The array is held by every GPU that loads the
 * library until the process exits.  The first call on a device looks up the
 * array's address while that device is current; make that call before any
 * stream capture.  All calls share the array, which keeps the last call's
 * contents: twiddles and spectra are uploaded (one asynchronous copy on
 * `stream`) only when the padded lengths, radii, quadrature counts or stencil
 * reach differ from the last successful call on the device.  Calls on one
 * device are serialised by a lock inside the library, and every call returns
 * only after its work on `stream` has finished, on error as well; work that
 * overlaps a call on the GPU by any other route races on the array.
 * Errors: PNP_ERR_INVALID, PNP_ERR_TOO_LARGE, PNP_ERR_PACKING, PNP_ERR_CUDA. */
int pnp_excess_mu_noalloc(const pnp_problem_desc *desc, const double *d_rho, double *d_mu_ex, void *stream);

/* Synchronise the problem's last stream and return the deferred device status
 * (PNP_OK, PNP_ERR_PACKING, PNP_ERR_OVERFLOW or PNP_ERR_CUDA), clearing it. */
int pnp_status(pnp_problem *p);

/* Per-kernel timing of the mu_ex pipeline.  While enabled, every kernel the
 * library launches for pnp_excess_mu / pnp_excess_mu_device is bracketed by
 * CUDA events on its stream.  pnp_stage_times synchronises, sums the elapsed
 * times per stage since the last reset into ms[k] and the launch counts into
 * launches[k] (k < max_stages, stage k named by pnp_stage_name), resets the
 * record and returns the number of stages.  Stage names: x_fwd, y_fwd, z_mac,
 * y_inv, x_fused, y_fwd_psi, z_back, y_inv_mu, x_inv. */
int pnp_stage_timing(pnp_problem *p, int enable);
int pnp_stage_times(pnp_problem *p, double *ms, int *launches, int max_stages);
const char *pnp_stage_name(int stage);

/* Relaxed Gummel iteration (Sec 3.2) on the device: per iteration mu_ex from
 * rho (above), the Poisson equation (Sec 2.1) for phi* and
 * phi <- l1 phi* + (1-l1) phi, then per species the Slotboom Nernst-Planck
 * equation -div(Dbar grad rhobar) = 0 (Sec 2.1) with the 7-point harmonic-mean
 * stencil of Sec 3.1, rho* = rhobar exp(-(q phi + mu_ex)) and the density
 * relaxation; both linear systems by multigrid-preconditioned CG (Sec 3.3).
 * Stops when the max-norm update is below tol.  phi0 [nz][ny][nx] and rho0
 * [s][nz][ny][nx] (host, nullable) give a warm start; the default start is
 * phi linear in z between the Dirichlet values and rho = rho_bulk.  Writes
 * phi_out and rho_out (host, nullable) and *stats (nullable).
 * Errors: PNP_ERR_NOT_CONVERGED (results still written), PNP_ERR_PACKING,
 * PNP_ERR_OVERFLOW, PNP_ERR_INVALID, PNP_ERR_CUDA. */
int pnp_gummel_solve(pnp_problem *p, const double *phi0, const double *rho0, double *phi_out,
                     double *rho_out, pnp_stats *stats);

/* Per-phase device time of the last pnp_gummel_solve of a problem created
 * with PNP_FLAG_PHASE_TIMING, summed over its Gummel iterations: ms[0] mu_ex,
 * ms[1] the Poisson step (right-hand side, multigrid-preconditioned CG, phi
 * relaxation), ms[2] the Nernst-Planck solves and density updates of every
 * species, ms[3] the end of the iteration (Anderson mixing when enabled, the
 * residual and the loop decision).  Fills min(max_phases, 4) entries and
 * returns 4; the equilibrium stage is not included.  Synchronises.  Errors:
 * PNP_ERR_INVALID (no flag, no solve yet, bad arguments), PNP_ERR_CUDA. */
int pnp_gummel_phase_times(pnp_problem *p, double *ms, int max_phases);

/* Serving: a queue of independent Gummel solves that run concurrently on one
 * GPU.  Requests are admitted as slots and the device-memory budget allow;
 * each keeps its state resident until it finishes; finished results wait in
 * host memory until polled.
 * Policies (no counterpart in the paper):
 *   PNP_SERVE_FIFO: admission in arrival order; every solve runs on its
 *     problem's stream at the default priority.
 *   PNP_SERVE_SMALLEST_FIRST: the queued request with the fewest unknowns
 *     (grid points x (species + 1)) is admitted first, and each solve runs on
 *     a stream whose CUDA priority rises as its grid shrinks (one level per
 *     factor 8 in grid points), so small solves' kernels are scheduled ahead
 *     of large ones already running: short requests are not held behind long
 *     ones, at the cost of the long ones' latency (a long request can wait as
 *     long as shorter ones keep arriving).  Results are the same bits under
 *     either policy. */
enum { PNP_SERVE_FIFO = 0, PNP_SERVE_SMALLEST_FIRST = 1 };
typedef struct {
    size_t hbm_budget_bytes;       /* device memory the server may hold, 0 -> 150 GB */
    int max_slots;                 /* concurrently resident solves, 0 -> 64 */
    int max_queue;                 /* waiting requests, 0 -> 4096 */
    int policy;                    /* PNP_SERVE_* */
} pnp_server_opts;

typedef struct {
    long long submitted, completed, failed, rejected;
    int active, queued;
    size_t bytes_in_use;
} pnp_server_stats;

int pnp_server_create(const pnp_server_opts *opts, pnp_server **out);

/* Stop the worker, drop pending requests and free everything. */
void pnp_server_destroy(pnp_server *s);

/* Enqueue a Gummel solve of `desc` (copied, including every array it points
 * to) with an optional warm start.  Non-blocking.  *ticket identifies it.
 * Errors: PNP_ERR_INVALID, PNP_ERR_BUSY (queue full, or the request alone
 * exceeds the budget). */
int pnp_submit(pnp_server *s, const pnp_problem_desc *desc, const double *phi0, const double *rho0,
               uint64_t *ticket);

/* Non-blocking.  PNP_PENDING while the request waits or runs; otherwise
 * copies phi_out [nz][ny][nx] and rho_out [s][nz][ny][nx] (nullable), fills
 * *stats, forgets the ticket and returns the solve's status.
 * PNP_ERR_UNKNOWN_TICKET for a ticket never issued or already polled. */
int pnp_poll(pnp_server *s, uint64_t ticket, double *phi_out, double *rho_out, pnp_stats *stats);

int pnp_server_get_stats(pnp_server *s, pnp_server_stats *out);

/* Nernst-Planck current of species `species` through every z face (Sec 2.1,
 * Sec 3.1; the paper's conductivity is the current over the applied field):
 * flux[k+1] = sum over the x-y plane of Dbar_face (rhobar_k - rhobar_k+1)
 * between planes k and k+1, k = -1 .. nz-1, where the planes -1 and nz are the
 * Dirichlet reservoirs (rhobar = rho_b exp(q phi_face + mu_b)),
 * Dbar = D exp(-(q phi + mu_ex)), rhobar = rho exp(q phi + mu_ex) with mu_ex
 * evaluated in FP64 from rho, and face values the harmonic mean (h = 1).  At
 * a converged steady state every entry is the same current.  phi
 * [nz][ny][nx], rho [s][nz][ny][nx] (host, FP64), flux nz + 1 doubles (host).
 * Needs a Dirichlet z axis.  Errors: PNP_ERR_INVALID (bad species, arrays,
 * boundaries), PNP_ERR_PACKING, PNP_ERR_NOMEM, PNP_ERR_CUDA. */
int pnp_plane_flux(pnp_problem *p, int species, const double *phi, const double *rho, double *flux);

/* Square-well free energy F_sh of Sec 2.3.2 (in kT), the mobile-site part:
 * the printed pair sum with its factor 1/2 counts each pair (i, s) twice, so
 * with the site density fixed
 *   F_sh = sum_i sum_r rho_i(r) sum_r' rho_s(r') Phi_is(|r - r'|) h^3
 *        = -sum_i eps_i sum_r rho_i(r) U(r),   U = K_sw (x) rho_s,
 * the well field the library builds on the device at set-up (site-site pairs
 * are a constant and mobile-mobile wells are absent).  Its derivative with
 * respect to rho_i is -eps_i U, twice mu_sh,i when sw_half keeps the 1/2.
 * rho [s][nz][ny][nx] (host, FP64, >= 0); *F_sh = 0 without wells.  The
 * densities are copied to the device and the sum is a fixed-shape device
 * reduction against U (the same bits every call).  Synchronises.
 * Errors: PNP_ERR_INVALID, PNP_ERR_NOMEM, PNP_ERR_CUDA. */
int pnp_square_well_energy(pnp_problem *p, const double *rho, double *F_sh);

/* Host-only: ionic conductivity from plane currents (Sec 4.2.1, size dependency
 * of the conductivity: the current density along the transport axis averaged
 * over its length, divided by the field).  flux [nspecies][nz+1] holds each
 * species' currents through the z faces as pnp_plane_flux returns them
 * (reduced units, h = 1, the desc's relative diffusivities).  With the charge
 * current density c_k = sum_i q_i flux_i[k] / (nx ny), its mean over the
 * nz+1 faces standing for the length average, and the applied field
 * E = -(phi_hi - phi_lo) / (nz+1) (kT/e per h):
 *   sigma[0] = mean_k c_k / E, in units of e^2 D / (k_B T h^3);
 *   sigma[1] = the same in S/cm for the diffusion scale D_m2_per_s (m^2/s;
 *              the paper's 1e-6 cm^2/s is 1e-10) and the desc's T and h_nm.
 * Needs a Dirichlet z axis and phi_hi != phi_lo.  Errors: PNP_ERR_INVALID
 * (descriptor rejected, zero bias, non-finite flux, D_m2_per_s < 0). */
int pnp_conductivity(const pnp_problem_desc *desc, const double *flux, double D_m2_per_s, double *sigma);

/* Host-only diagnostic: the discrete weight stencil K[m] the library builds
 * at set-up (Sec 2.3.1 weights by the quadrature of Sec 3.5, each node
 * deposited trilinearly on the grid; Sec 2.3.2 well shell).  kind 0: shell
 * delta(|r| - r_out) (w2); 1: ball |r| <= r_out (w3); 2, 3, 4: x, y, z
 * components of the vector shell (vec w2); 5: thick shell r_in <= |r| <= r_out
 * (the square well).  nmu, ntheta, nr: quadrature counts (0 = defaults).  out
 * gets (2S+1)^3 values, out[((mz+S)(2S+1) + my+S)(2S+1) + mx+S] for offsets
 * |m| <= S in units of h; S must reach the support (ceil(r_out) + 1).
 * Errors: PNP_ERR_INVALID. */
int pnp_weight_stencil(int kind, double r_in, double r_out, int nmu, int ntheta, int nr, int S, double *out);

/* Host-only: the discrete MSA pair kernel of Sec 2.3.4 for species i, j of
 * a descriptor, C_ij(r) = -q_i q_j l_B [2B/s - (B/s)^2 r - 1/r] on the ball
 * r <= s = R_i + R_j, B = [xi + 1 - sqrt(1 + 2 xi)] / xi, xi = kappa s,
 * kappa^2 = 4 pi l_B sum_k rho_b,k q_k^2 (l_B from the descriptor's T, eps_r
 * and h_nm), by the ball quadrature of Sec 3.5 with the descriptor's counts,
 * each node deposited trilinearly.  out gets (2S+1)^3 values in the layout
 * of pnp_weight_stencil; S >= ceil(s) + 1.  The set-up stencil of the
 * electrostatic-correlation term; the device pipeline does not apply it yet.
 * Errors: PNP_ERR_INVALID. */
int pnp_msa_stencil(const pnp_problem_desc *desc, int i, int j, int S, double *out);

/* Host-only diagnostic: the real octant of that stencil's DFT on an
 * Lx x Ly x Lz periodic grid, as the set-up stores it: out[kz][ky][kx]
 * (k <= L/2, x fastest) = sum_m K[m] f(kx mx) f(ky my) f(kz mz), f = cos on
 * even axes and sin on the vector component's own axis (odd), so the DFT is
 * out (even kernels) or -i out (vector components).  Every L must be at least
 * 2S + 1.  Errors: PNP_ERR_INVALID. */
int pnp_weight_spectrum(int kind, double r_in, double r_out, int nmu, int ntheta, int nr, int S, int Lx, int Ly,
                        int Lz, double *out);

/* Failure-path self-test with no counterpart in the paper: launches one
 * kernel that waits on an mbarrier nothing ever completes, with the same
 * globally-timed bounded wait the tensor-core kernels use, limited to
 * limit_ms (0 < limit_ms <= 1000).  Returns PNP_ERR_TIMEOUT when the wait
 * gave up and reported it (the expected result), PNP_ERR_INVALID for a bad
 * limit, PNP_ERR_CUDA on a runtime error.  The device stays usable. */
int pnp_selftest_bounded_wait(double limit_ms);

/* Failure-path test hook with no counterpart in the paper.  Arms a host-side
 * fault: counting from this call, the k-th device allocation the library
 * makes (1-based) reports PNP_ERR_NOMEM without calling CUDA; k <= 0 disarms.
 * Lets a test drive every allocation site's error path without exhausting or
 * faulting a GPU.  Nothing else arms it (no environment variable is read).
 * Process-wide; not for production callers.  Returns PNP_OK. */
int pnp_test_fail_alloc_at(long k);

/* Static message for an error code. */
const char *pnp_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* PNP_GB300_H */
