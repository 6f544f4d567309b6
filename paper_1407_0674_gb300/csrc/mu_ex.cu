// Excess chemical potential: problem set-up (spectra, twiddles, square-well
// field), per-precision buffers, dispatch, stage timing, and the fixed-scratch
// entry point.  The pipeline kernels live in mu_ex_core.cuh.
#include <mutex>

#include "mu_ex_core.cuh"

namespace pnp {

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

__global__ void k_to_dd(const double *__restrict__ a, dd *__restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = dd(a[i]);
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
        size_t bytes = (prec == PNP_PREC_FP32 ? 8 : 16) * (size_t)L;
        cudaError_t e = dmalloc(&db->tw[c], bytes, p->stream);
        if (e != cudaSuccess) return PNP_ERR_NOMEM;
        db->bytes += bytes;
        if (prec == PNP_PREC_FP64) {
            e = cudaMemcpy(db->tw[c], h.data(), bytes, cudaMemcpyHostToDevice);
        } else if (prec == PNP_PREC_DF64) {
            std::vector<dd> s(h.size());
            for (size_t k = 0; k < h.size(); ++k) s[k] = dd(h[k]);
            e = cudaMemcpy(db->tw[c], s.data(), bytes, cudaMemcpyHostToDevice);
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
    dfree(db->tc_b, st);
    delete db;
}

// FP64 spectra of every species' kernels, built on the host.
// Builds into a local set and publishes it in p->buf[0] only when complete:
// a failed build leaves nothing behind that a later call could take as ready.
static int build_fp64_into(Problem *p, DeviceBuffers *db);
static int build_fp64(Problem *p) {
    DeviceBuffers *db = new DeviceBuffers();
    db->prec = PNP_PREC_FP64;
    const int rc = build_fp64_into(p, db);
    if (rc) {
        cudaStreamSynchronize(p->stream);
        free_buffers(db, p->stream);
        return rc;
    }
    p->buf[0] = db;
    return PNP_OK;
}

static int build_fp64_into(Problem *p, DeviceBuffers *db) {
    int rc = upload_twiddles(p, db, PNP_PREC_FP64);
    if (rc) return rc;
    const Dims d = make_dims(p);
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    const size_t bytes = sizeof(double) * oct * spec_kernels(p);
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
    if (p->msa) {
        // MSA pair kernels (Sec 2.3.4), even in every axis, stored negated:
        // the z-back kernels add spec * rho_j to mu_i
        const bool even[3] = {false, false, false};
        for (int i = 0; i < p->s; ++i)
            for (int j = i; j < p->s; ++j) {
                Stencil c;
                build_msa_pair(*p, i, j, c);
                octant_transform(c, p->L, even, -scale, h.data());
                cudaError_t e = cudaMemcpy((double *)db->spec +
                                               (size_t)(p->s * kNumKernels + msa_pair(i, j, p->s)) * oct,
                                           h.data(), sizeof(double) * oct, cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return cuda_status(e);
            }
    }
    p->device_bytes += db->bytes;
    return PNP_OK;
}

int mu_ex_prepare(Problem *p, int prec) {
    if (prec == PNP_PREC_FP64) return p->buf[0] ? PNP_OK : build_fp64(p);
    if (prec == PNP_PREC_TF32SPLIT) {
        // the FP32 buffers plus the split DFT matrices of the tensor-core y pass
        int rc = mu_ex_prepare(p, PNP_PREC_FP32);
        if (rc) return rc;
        DeviceBuffers *db = p->buf[1];
        if (db->tc_b) return PNP_OK;
        std::vector<float> m(4 * 32 * 32);
        ypass_tc_matrices(m.data());
        const size_t bytes = m.size() * sizeof(float);
        if (dmalloc((void **)&db->tc_b, bytes, p->stream) != cudaSuccess) return PNP_ERR_NOMEM;
        cudaError_t e = cudaMemcpyAsync(db->tc_b, m.data(), bytes, cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) return cuda_status(e);
        db->bytes += bytes;
        p->device_bytes += bytes;
        return PNP_OK;
    }
    const int slot = prec == PNP_PREC_FP32 ? 1 : 2;
    if (p->buf[slot]) return PNP_OK;
    int rc = mu_ex_prepare(p, PNP_PREC_FP64);
    if (rc) return rc;
    // built locally, published only when complete (see build_fp64)
    DeviceBuffers *db = new DeviceBuffers();
    db->prec = prec;
    auto fail = [&](int code) {
        cudaStreamSynchronize(p->stream);
        free_buffers(db, p->stream);
        return code;
    };
    rc = upload_twiddles(p, db, prec);
    if (rc) return fail(rc);
    const Dims d = make_dims(p);
    const size_t n = (size_t)d.Ox * d.Oy * d.Oz * spec_kernels(p);
    const size_t esz = prec == PNP_PREC_FP32 ? sizeof(float) : sizeof(dd);
    if (dmalloc(&db->spec, esz * n, p->stream) != cudaSuccess) return fail(PNP_ERR_NOMEM);
    db->bytes += esz * n;
    if (prec == PNP_PREC_FP32)
        k_to_float<<<1024, 256, 0, p->stream>>>((const double *)p->buf[0]->spec, (float *)db->spec, n);
    else
        k_to_dd<<<1024, 256, 0, p->stream>>>((const double *)p->buf[0]->spec, (dd *)db->spec, n);
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(cuda_status(e));
    p->buf[slot] = db;
    p->device_bytes += db->bytes;
    return PNP_OK;
}

static __global__ void k_set(double *__restrict__ a, double v, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a[i] = v;
}

// out = K (x) in for one real field on the problem's grid (zero extension on
// the padded axes) with the FP64 Stockham kernels: x R2C, y, z multiply by the
// even real spectrum octant `d_spec` (1/(Lx Ly Lz) folded in), y, x C2R.  Uses
// the workspace; set-up only.
static int conv_even_field(Problem *p, const double *d_in, const double *d_spec, double *d_out) {
    int rc = set_smem_attrs<double>();
    if (rc == PNP_OK)
        rc = cuda_status(cudaFuncSetAttribute(k_zconv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    if (rc) return rc;
    const Dims d = make_dims(p);
    const size_t N = p->npts();
    const Launch l = launch_shape(p, PNP_PREC_FP64);
    Work w = carve(p, PNP_PREC_FP64);
    DeviceBuffers *db = p->buf[0];
    double2 *A = (double2 *)w.A, *B = (double2 *)w.B10, *B2 = (double2 *)w.Bs;
    SpeciesConst one{};
    one.s = 1;
    dim3 gx((d.npairs + l.P_x - 1) / l.P_x, d.nz, 1);
    k_xfwd<double><<<gx, 256, l.sm_x, p->stream>>>(d_in, N, A, d, p->ax[0], (const double2 *)db->tw[0], l.P_x);
    dim3 gy((d.Wx + l.TX_y - 1) / l.TX_y, d.nz, 1);
    k_ypass<double, false><<<gy, 256, l.sm_y, p->stream>>>(A, B, d, d.ny, d.ny, d.Ly, d.Ly, p->ax[1],
                                                           (const double2 *)db->tw[1], l.TX_y);
    dim3 gz((d.Wx + l.TX_z - 1) / l.TX_z, d.Ly);
    k_zconv<<<gz, 256, l.sm_zconv, p->stream>>>(B, B2, d, p->ax[2], (const double2 *)db->tw[2], d_spec, l.TX_z);
    k_ypass<double, true><<<gy, 256, l.sm_y, p->stream>>>(B2, A, d, d.Ly, d.Ly, d.ny, d.ny, p->ax[1],
                                                          (const double2 *)db->tw[1], l.TX_y);
    k_xinv<double><<<gx, 256, l.sm_x, p->stream>>>(A, d_out, N, d, p->ax[0], (const double2 *)db->tw[0], nullptr,
                                                   one, l.P_x, nullptr);
    return cuda_status(cudaGetLastError());
}

// MSA bulk field E_i = sum_j rho_b,j (C_ij (x) 1_Omega) (Sec 2.3.4): with
// mu_el,i = -sum_j C_ij (x) (rho_j - rho_b,j) on the domain, the density part
// runs through the z-back kernels every call and this fixed part is added in
// the last x pass.  One convolution of the indicator of the domain per species
// with the combined stencil sum_j rho_b,j C_ij.
static int build_msa_field(Problem *p) {
    const Dims d = make_dims(p);
    const size_t N = p->npts();
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    if (dmalloc((void **)&p->d_E, sizeof(double) * N * p->s, p->stream) != cudaSuccess) return PNP_ERR_NOMEM;
    p->device_bytes += sizeof(double) * N * p->s;
    double *d_one = nullptr, *d_spec = nullptr;
    cudaError_t e = dmalloc((void **)&d_one, sizeof(double) * N, p->stream);
    if (e == cudaSuccess) e = dmalloc((void **)&d_spec, sizeof(double) * oct, p->stream);
    int rc = cuda_status(e);
    if (rc == PNP_OK) k_set<<<1024, 256, 0, p->stream>>>(d_one, 1.0, N);
    std::vector<double> h(oct);
    const bool even[3] = {false, false, false};
    const double scale = 1.0 / ((double)d.Lx * d.Ly * d.Lz);
    for (int i = 0; i < p->s && rc == PNP_OK; ++i) {
        Stencil K;
        K.S = p->Smsa;
        K.K.assign((size_t)(2 * K.S + 1) * (2 * K.S + 1) * (2 * K.S + 1), 0.0);
        for (int j = 0; j < p->s; ++j) {
            Stencil c;
            build_msa_pair(*p, i, j, c);
            for (int mz = -c.S; mz <= c.S; ++mz)
                for (int my = -c.S; my <= c.S; ++my)
                    for (int mx = -c.S; mx <= c.S; ++mx) K.at(mx, my, mz) += p->rho_b[j] * c.at(mx, my, mz);
        }
        octant_transform(K, p->L, even, scale, h.data());
        // the previous convolution reads d_spec: copy in stream order
        e = cudaMemcpyAsync(d_spec, h.data(), sizeof(double) * oct, cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        rc = cuda_status(e);
        if (rc == PNP_OK) rc = conv_even_field(p, d_one, d_spec, p->d_E + (size_t)i * N);
    }
    if (rc == PNP_OK) rc = cuda_status(cudaStreamSynchronize(p->stream));
    else cudaStreamSynchronize(p->stream);
    dfree(d_one, p->stream);
    dfree(d_spec, p->stream);
    return rc;
}

// Workspace, FP64 spectra, the square-well field U = K_sw (x) rho_s and the
// MSA bulk field.
int mu_ex_setup(Problem *p) {
    p->work_bytes = workspace_bytes(p);
    if (dmalloc(&p->d_work, p->work_bytes, p->stream) != cudaSuccess) return PNP_ERR_NOMEM;
    p->device_bytes += p->work_bytes;
    int rc = build_fp64(p);
    if (rc) return rc;
    if (p->msa) {
        rc = build_msa_field(p);
        if (rc) return rc;
    }
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
        rc = conv_even_field(p, d_rs, d_spec, p->d_U);
        if (rc == PNP_OK) e = cudaStreamSynchronize(p->stream);
        else cudaStreamSynchronize(p->stream);
    }
    dfree(d_sites, p->stream);
    dfree(d_rs, p->stream);
    dfree(d_spec, p->stream);
    if (rc) return rc;
    return cuda_status(e);
}

// ---------------------------------------------------------------------------
// Square-well free energy F_sh = -sum_i eps_i sum_r rho_i(r) U(r) (Sec 2.3.2,
// mobile-site part) as a fixed-shape device reduction: each thread sums its
// points in grid-stride order (species inside, in order), each block a tree,
// then one block sums the block partials in a tree; the same bits every call.
constexpr int kFshBlocks = 512;

static __global__ void __launch_bounds__(256) k_fsh_partial(const double *__restrict__ U,
                                                            const double *__restrict__ rho, size_t N, int s,
                                                            SpeciesConst sc, double *__restrict__ part) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int i = 0; i < s; ++i) v += sc.c0[i] * rho[(size_t)i * N + p];
        acc += v * U[p];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

static __global__ void __launch_bounds__(kFshBlocks) k_fsh_final(const double *__restrict__ part, int nb,
                                                                double *__restrict__ out) {
    __shared__ double sh[kFshBlocks];
    sh[threadIdx.x] = (int)threadIdx.x < nb ? part[threadIdx.x] : 0.0;
    __syncthreads();
    for (int w = kFshBlocks / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// F_sh of the device densities d_rho [s][N] into d_out[0]; d_part holds
// kFshBlocks doubles.  Problems without wells get 0.
int square_well_energy_enqueue(Problem *p, const double *d_rho, double *d_out, double *d_part, cudaStream_t st) {
    const size_t N = p->npts();
    if (!p->has_wells || !p->d_U) return cuda_status(cudaMemsetAsync(d_out, 0, sizeof(double), st));
    SpeciesConst c{};
    c.s = p->s;
    for (int i = 0; i < p->s; ++i) c.c0[i] = -p->depth[i];     // coefficient of rho_i U
    const int nb = (int)std::min<size_t>(kFshBlocks, std::max<size_t>(1, (N + 255) / 256));
    k_fsh_partial<<<nb, 256, 0, st>>>(p->d_U, d_rho, N, p->s, c, d_part);
    k_fsh_final<<<1, kFshBlocks, 0, st>>>(d_part, nb, d_out);
    return cuda_status(cudaGetLastError());
}

int mu_ex_enqueue(Problem *p, int prec, const double *d_rho, double *d_mu, cudaStream_t st) {
    int rc = mu_ex_prepare(p, prec);
    if (rc) return rc;
    NvtxRange range("mu_ex");
    if (prec == PNP_PREC_FP64) return run_pipeline_fp64(p, p->buf[0], d_rho, d_mu, st);
    if (prec == PNP_PREC_DF64) return run_pipeline_df64(p, p->buf[2], d_rho, d_mu, st);
    return run_pipeline_fp32(p, p->buf[1], d_rho, d_mu, st, prec == PNP_PREC_TF32SPLIT);
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

// Every stage is also an NVTX range named after the stage (a no-op unless a
// tracing tool is attached).
static const char *const kStageNames[kNumStages] = {"x_fwd", "y_fwd", "z_mac", "y_inv", "x_fused",
                                                    "y_fwd_psi", "z_back", "y_inv_mu", "x_inv"};

void StageTimer::begin(int s, cudaStream_t st) {
    nvtxRangePushA(s >= 0 && s < kNumStages ? kStageNames[s] : "mu_ex stage");
    if (!enabled) return;
    cudaEvent_t a = get();
    cudaEventRecord(a, st);
    stage.push_back(s);
    ev0.push_back(a);
}

void StageTimer::end(cudaStream_t st) {
    nvtxRangePop();
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
    for (int k = 0; k < 3; ++k) {
        free_buffers(p->buf[k], p->stream);
        p->buf[k] = nullptr;
    }
    dfree(p->d_work, p->stream);
    dfree(p->d_U, p->stream);
    dfree(p->d_E, p->stream);
    p->d_work = nullptr;
    p->d_U = nullptr;
    p->d_E = nullptr;
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
// cleared by each call; the twiddles and spectra are uploaded again whenever
// the padded lengths, species radii, quadrature counts or stencil reach differ
// from the last successful call on that device (a per-device key, dropped on
// any error); the workspace is fully overwritten before it is read.  Calls on
// one device are serialised by a per-device lock for their whole duration, and
// each returns only after its work is done, on success and on error alike.
// Calls whose work overlaps on the GPU (from code that shares the array by
// other routes) race on it.
namespace pnp {

constexpr size_t kNoAllocBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mutex[kNoAllocDevices];
void *g_noalloc_addr[kNoAllocDevices] = {nullptr};
// what the array's twiddles and spectra were built for, per device (empty:
// nothing valid)
std::vector<double> g_noalloc_key[kNoAllocDevices];

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

// everything the twiddle tables, the spectra and their places in the array
// depend on
std::vector<double> noalloc_key(const Problem &p) {
    std::vector<double> k = {(double)p.L[0], (double)p.L[1], (double)p.L[2], (double)p.s, (double)p.S,
                             (double)p.quad[0], (double)p.quad[1], (double)p.quad[2]};
    for (int i = 0; i < p.s; ++i) k.push_back(p.R[i]);
    return k;
}

void twiddles_host(int L, double *h) {
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
    if (p.has_wells || p.msa) return PNP_ERR_INVALID;   // hard-sphere part only
    if (noalloc_bytes(p) > kNoAllocBytes) return PNP_ERR_TOO_LARGE;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kNoAllocDevices) return PNP_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex[dev]);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        g_noalloc_addr[dev] = ptr;
    }
    unsigned char *base = (unsigned char *)g_noalloc_addr[dev];
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> &key = g_noalloc_key[dev];
    // after the first enqueue every exit waits for the stream (the lock is
    // still held, so no later call can write the array under work in flight)
    // and drops the key, since the array's contents are then unknown
    auto fail = [&](int code) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        key.clear();
        return code;
    };
    const std::vector<double> want = noalloc_key(p);
    const bool fresh = key != want;
    key.clear();
    // carve: status word | twiddles x, y, z | spectra | workspace
    size_t off = 256;
    DeviceBuffers db;
    db.prec = PNP_PREC_FP64;
    const Dims d = make_dims(&p);
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz;
    size_t tw_off[3];
    for (int c = 0; c < 3; ++c) {
        tw_off[c] = off;
        db.tw[c] = base + off;
        off += round256(16 * (size_t)p.L[c]);
    }
    db.spec = base + off;
    off += round256(sizeof(double) * oct * kNumKernels * p.s);
    if (fresh) {
        // one host image of the twiddles and spectra, one copy
        std::vector<double> h((off - 256) / sizeof(double), 0.0);
        for (int c = 0; c < 3; ++c) twiddles_host(p.L[c], h.data() + (tw_off[c] - 256) / sizeof(double));
        double *hs = h.data() + ((unsigned char *)db.spec - base - 256) / sizeof(double);
        const double scale = 1.0 / ((double)d.Lx * d.Ly * d.Lz);
        const bool odd[kNumKernels][3] = {{false, false, false}, {false, false, false}, {true, false, false},
                                          {false, true, false}, {false, false, true}};
        for (int i = 0; i < p.s; ++i) {
            Stencil stn[kNumKernels];
            build_fmt_stencils(p.R[i], p.quad[0], p.quad[1], p.quad[2], p.S, stn);
            for (int k = 0; k < kNumKernels; ++k)
                octant_transform(stn[k], p.L, odd[k], scale, hs + (size_t)(i * kNumKernels + k) * oct);
        }
        // from pageable memory the copy has read `h` when the call returns
        e = cudaMemcpyAsync(base + 256, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(cuda_status(e));
    }
    p.d_work = base + off;
    p.d_flag = (int *)base;
    e = cudaMemsetAsync(p.d_flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return fail(cuda_status(e));
    rc = run_pipeline_fp64(&p, &db, d_rho, d_mu_ex, st);
    if (rc) return fail(rc);
    int flag = 0;
    e = cudaMemcpyAsync(&flag, p.d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_status(e));
    p.d_work = nullptr;
    p.d_flag = nullptr;
    key = want;
    return (flag & (kFlagPacking | kFlagNonFinite)) ? PNP_ERR_PACKING : PNP_OK;
}

namespace pnp {

// Device memory a problem will hold once its Gummel state exists: FFT
// workspace, spectra (FP64, plus FP32 when that is the problem's precision),
// square-well field, staging buffers and the multigrid hierarchy.
size_t estimate_device_bytes(const Problem &p) {
    const Dims d = make_dims(&p);
    const size_t N = p.npts();
    const size_t oct = (size_t)d.Ox * d.Oy * d.Oz * spec_kernels(&p);
    size_t b = workspace_bytes(&p) + oct * sizeof(double);
    if (p.precision == PNP_PREC_FP32 || p.precision == PNP_PREC_TF32SPLIT) b += oct * sizeof(float);
    if (p.precision == PNP_PREC_DF64) b += oct * sizeof(dd);
    if (p.has_wells) b += N * sizeof(double);
    if (p.msa) b += N * p.s * sizeof(double);               // MSA bulk field
    b += sizeof(double) * (2 * N * p.s + N);                 // host-call staging
    b += sizeof(double) * N * 11 * 8 / 7;                    // multigrid levels
    b += sizeof(double) * N * (2 * (size_t)p.s + 7);         // solve state and CG vectors
    if (p.aa_depth > 0) b += sizeof(double) * N * (1 + (size_t)p.s) * 2 * (p.aa_depth + 2);   // Anderson history
    return b + b / 16 + (1 << 20);
}

}  // namespace pnp
