// Split-precision DFT stage on the 5th-generation tensor cores: the y pass of
// the FP32 pipeline (Sec 3.4: one axis of the zero-padded 3D transforms) with
// its two radix-16 DFT stages written as dense matrix products.
//
// A length-256 line is x[n1 + 16 n2].  Stage A forms, for every (column c, n1),
// the 16-point DFT over n2; the result is multiplied by W_256^(n1 k2); stage B
// forms the 16-point DFT over n1, giving X[k2 + 16 k1].  A CTA takes 8
// adjacent half-spectrum columns of one (field, z) plane, so both stages are
//     D (128 x 32) = A (128 x 32) * B (32 x 32)
// with complex values as interleaved (re, im) pairs: rows of A are the 128
// (column, n1) [stage A] or (k2, column) [stage B] lines, B is the real form
// of the 16-point DFT matrix.  Each product runs as three TF32 MMAs,
//     A_hi B_hi + A_lo B_hi + A_hi B_lo,
// where x = x_hi + x_lo with x_hi the value rounded to TF32 (10-bit mantissa)
// and x_lo the rounded remainder, accumulated in FP32 in tensor memory (about
// 21 significant bits in the products; the dropped A_lo B_lo term is below
// 2^-21 relative).
//
// tcgen05 usage: one elected thread issues the MMAs (kind::tf32, M 128, N 32,
// K 8 per instruction, both operands K-major in 128-byte-swizzled shared
// memory), tcgen05.commit signals an mbarrier, and the four warps read the
// accumulator back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31).
// Every wait on the mbarrier is bounded by the global timer; on expiry the CTA
// sets the timeout flag, stops issuing work and still frees its tensor memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "mu_ex_core.cuh"

namespace pnp {
namespace tcy {

constexpr int kThreads = 128;
constexpr int kCols = 8;                    // half-spectrum columns per tile
constexpr int kRowBytes = 128;              // 32 FP32 values: one swizzle row
constexpr int kAbytes = 128 * kRowBytes;    // one A operand (hi or lo)
constexpr int kBbytes = 32 * kRowBytes;     // one B operand (hi or lo)
constexpr int kTmemCols = 32;
constexpr int kSmemBytes = 2 * kAbytes + 2 * kBbytes + 64 + 1024;   // + barrier, slot, alignment
constexpr unsigned long long kWaitLimitNs = 1000000000ull;           // 1 s per wait

// instruction descriptor: D F32, A and B TF32, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of FP32 element k of row r in a K-major tile with the 128-byte
// swizzle (16-byte chunk index XOR row mod 8; tile base 1024-byte aligned)
__device__ __forceinline__ uint32_t swz(int r, int k) {
    return (uint32_t)(r * kRowBytes + ((((k >> 2) ^ (r & 7))) << 4) + (k & 3) * 4);
}

// shared-memory matrix descriptor: start address, leading offset 16 B (unused
// for swizzled K-major), stride 1024 B between 8-row groups, descriptor
// version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// round to the nearest TF32 value (ties away from zero)
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void put_split(unsigned char *sm, uint32_t off, float2 v) {
    const float hx = tf32_round(v.x), hy = tf32_round(v.y);
    *reinterpret_cast<float2 *>(sm + off) = make_float2(hx, hy);
    *reinterpret_cast<float2 *>(sm + kAbytes + off) = make_float2(tf32_round(v.x - hx), tf32_round(v.y - hy));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity,
                                           unsigned long long limit_ns = kWaitLimitNs) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) return false;
    }
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// the three split products of one stage, then a commit to the mbarrier
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t aHi, uint32_t aLo, uint32_t bHi, uint32_t bLo,
                                            uint32_t bar) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {          // K = 32 in steps of 8 TF32 (32 bytes)
        const uint32_t o = ks * 32;
        mma(tmem, sdesc(aHi + o), sdesc(bHi + o), ks > 0);
        mma(tmem, sdesc(aLo + o), sdesc(bHi + o), 1);
        mma(tmem, sdesc(aHi + o), sdesc(bLo + o), 1);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// in: rows j < n_in of planes with rows_in rows (others zero); out: rows j <
// n_out of planes with rows_out rows; F fields x nz planes x Wx columns.
// bmat: [hi, lo][32][32] real form of the 16-point DFT of this direction,
// element [j][k] = B(k, j).  tw[m] = exp(-2 pi i m / 256).
template <bool INV>
__global__ void __launch_bounds__(kThreads) k_ypass_tc(const float2 *__restrict__ in, float2 *__restrict__ out, Dims d,
                                                      int rows_in, int n_in, int rows_out, int n_out, int F,
                                                      const float2 *__restrict__ tw, const float *__restrict__ bmat,
                                                      int *__restrict__ flag) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sm = smem_raw + (base - raw);
    const uint32_t aHi = base, aLo = base + kAbytes, bHi = base + 2 * kAbytes, bLo = bHi + kBbytes;
    uint64_t *bar_p = reinterpret_cast<uint64_t *>(sm + 2 * kAbytes + 2 * kBbytes);
    uint32_t *slot_p = reinterpret_cast<uint32_t *>(sm + 2 * kAbytes + 2 * kBbytes + 8);
    const uint32_t bar = smem_addr(bar_p);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int c = tid & (kCols - 1), q = tid >> 3;

    for (int e = tid; e < 2 * 32 * 32; e += kThreads) {
        const int h = e >> 10, j = (e >> 5) & 31, k = e & 31;
        *reinterpret_cast<float *>(sm + 2 * kAbytes + h * kBbytes + swz(j, k)) = bmat[e];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot_p)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *slot_p;
    const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);

    const int tilesX = (d.Wx + kCols - 1) / kCols;
    const long ntiles = (long)tilesX * d.nz * F;
    auto plane = [&](long tl, int &kx) -> size_t {
        const int bx = (int)(tl % tilesX);
        const long rest = tl / tilesX;
        kx = bx * kCols + c;
        return (size_t)rest;      // f * nz + z
    };
    float2 x[16];
    auto load = [&](long tl) {
        int kx;
        const size_t pl = plane(tl, kx);
        const float2 *src = in + pl * rows_in * d.Wx + kx;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) {
            const int y = q + 16 * n2;
            x[n2] = (kx < d.Wx && y < n_in) ? __ldg(&src[(size_t)y * d.Wx]) : make_float2(0.f, 0.f);
        }
    };

    long tile = blockIdx.x;
    if (tile < ntiles) load(tile);
    uint32_t parity = 0;
    bool ok = true;
    while (tile < ntiles && ok) {
        // stage A operand: row tid = (n1 = q, column c), K index n2
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) put_split(sm, swz(tid, 2 * n2), x[n2]);
        const long cur = tile;
        tile += gridDim.x;
        if (tile < ntiles) load(tile);          // in flight during this tile's MMAs

        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) issue_stage(tmem, aHi, aLo, bHi, bLo, bar);
        ok = __syncthreads_and(wait_phase(bar, parity));
        parity ^= 1;
        if (!ok) break;
        fence_after();
        float acc[32];
        tmem_ld32(tlane, acc);

        // twiddle W_256^(n1 k2), then stage B operand: row (k2, c), K index n1 = q
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            float2 w = __ldg(&tw[q * k2]);
            if (INV) w.y = -w.y;
            const float2 v = make_float2(acc[2 * k2] * w.x - acc[2 * k2 + 1] * w.y,
                                         acc[2 * k2] * w.y + acc[2 * k2 + 1] * w.x);
            put_split(sm, swz(k2 * kCols + c, 2 * q), v);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) issue_stage(tmem, aHi, aLo, bHi, bLo, bar);
        ok = __syncthreads_and(wait_phase(bar, parity));
        parity ^= 1;
        if (!ok) break;
        fence_after();
        tmem_ld32(tlane, acc);

        // row tid = (k2 = q, column c) holds X[k2 + 16 k1], k1 < 16
        int kx;
        const size_t pl = plane(cur, kx);
        if (kx < d.Wx) {
            float2 *dst = out + pl * rows_out * d.Wx + kx;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const int y = q + 16 * k1;
                if (y < n_out) dst[(size_t)y * d.Wx] = make_float2(acc[2 * k1], acc[2 * k1 + 1]);
            }
        }
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (!ok && tid == 0) atomicOr(flag, kFlagTimeout);
    // a timed-out wait leaves the MMAs possibly in flight: give them one more
    // bounded wait before the tensor memory is released
    if (!ok) wait_phase(bar, parity ^ 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Failure-path check of the bounded wait: one thread waits on an mbarrier
// that nothing arrives on, gives up after limit_ns and records the timeout
// the way the pipeline kernels do.
__global__ void k_bounded_wait_probe(unsigned long long limit_ns, int *flag) {
    __shared__ uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1) : "memory");
    if (!wait_phase(b, 0, limit_ns)) atomicOr(flag, kFlagTimeout);
}

}  // namespace tcy

int bounded_wait_probe(double limit_ms) {
    if (!(limit_ms > 0) || limit_ms > 1000.0) return PNP_ERR_INVALID;
    int *d_flag = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = dmalloc((void **)&d_flag, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flag, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        tcy::k_bounded_wait_probe<<<1, 1, 0, st>>>((unsigned long long)(limit_ms * 1e6), d_flag);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_flag) dfree(d_flag, st);
    if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    if (e != cudaSuccess) return cuda_status(e);
    return (h & kFlagTimeout) ? PNP_ERR_TIMEOUT : PNP_OK;
}

// Real form of the 16-point DFT (forward: exp(-2 pi i n k / 16); inverse:
// conjugate) split into TF32 hi and lo parts: out[dir][hi/lo][j][k] with
// j = 2 k_out + {re, im}, k = 2 n_in + {re, im}.  4096 floats.
void ypass_tc_matrices(float *out) {
    auto tf32 = [](float v) {
        uint32_t u;
        std::memcpy(&u, &v, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        float r;
        std::memcpy(&r, &u, 4);
        return r;
    };
    for (int dir = 0; dir < 2; ++dir) {
        for (int kk = 0; kk < 16; ++kk) {
            for (int n = 0; n < 16; ++n) {
                const double ang = 2.0 * M_PI * (double)((kk * n) % 16) / 16.0;
                const double cr = std::cos(ang), si = dir == 0 ? -std::sin(ang) : std::sin(ang);
                // out_re = sum a cr - b si ; out_im = sum a si + b cr
                const double m[2][2] = {{cr, -si}, {si, cr}};   // [out comp][in comp]
                for (int oc = 0; oc < 2; ++oc)
                    for (int ic = 0; ic < 2; ++ic) {
                        const int j = 2 * kk + oc, k = 2 * n + ic;
                        const float v = (float)m[oc][ic];
                        const float hi = tf32(v);
                        const float lo = tf32((float)((double)m[oc][ic] - (double)hi));
                        out[((dir * 2 + 0) * 32 + j) * 32 + k] = hi;
                        out[((dir * 2 + 1) * 32 + j) * 32 + k] = lo;
                    }
            }
        }
    }
}

bool ypass_tc_supported(const Dims &d) { return d.Ly == 256; }

int launch_ypass_tc(bool inv, const float2 *in, float2 *out, const Dims &d, int rows_in, int n_in, int rows_out,
                    int n_out, int F, const float2 *tw, const float *bmat, int *flag, cudaStream_t st) {
    // resident CTAs per SM and SM count, once per device
    static std::mutex mu;
    static int cached_per_sm[64] = {0}, cached_sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = 1, sms = 1;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && cached_per_sm[dev]) {
            per_sm = cached_per_sm[dev];
            sms = cached_sms[dev];
        } else {
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            for (int k = 0; k < 2; ++k) {
                auto fn = k ? tcy::k_ypass_tc<true> : tcy::k_ypass_tc<false>;
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, tcy::kSmemBytes);
                // without a carveout preference the occupancy query assumes the
                // smallest shared-memory split that fits one CTA
                cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
            }
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tcy::k_ypass_tc<false>, tcy::kThreads,
                                                              tcy::kSmemBytes) != cudaSuccess)
                per_sm = 0;
            // the same bound from the kernel's registers and the SM's shared memory
            cudaFuncAttributes fa;
            int smem_sm = 0;
            if (cudaFuncGetAttributes(&fa, tcy::k_ypass_tc<false>) == cudaSuccess &&
                cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
                fa.numRegs > 0) {
                const int by_regs = 65536 / (fa.numRegs * tcy::kThreads);
                const int by_smem = smem_sm / (tcy::kSmemBytes + 1024);
                per_sm = std::max(per_sm, std::min(by_regs, by_smem));
            }
            per_sm = std::min(std::max(per_sm, 1), 8);
            sms = std::max(sms, 1);
            cudaGetLastError();
            if (dev >= 0 && dev < 64) {
                cached_per_sm[dev] = per_sm;
                cached_sms[dev] = sms;
            }
        }
    }
    const long ntiles = (long)((d.Wx + tcy::kCols - 1) / tcy::kCols) * d.nz * F;
    if (ntiles == 0) return PNP_OK;
    const int grid = (int)std::min<long>(ntiles, (long)sms * per_sm);
    const float *b = bmat + (inv ? 2 * 32 * 32 : 0);
    if (inv)
        tcy::k_ypass_tc<true><<<grid, tcy::kThreads, tcy::kSmemBytes, st>>>(in, out, d, rows_in, n_in, rows_out,
                                                                              n_out, F, tw, b, flag);
    else
        tcy::k_ypass_tc<false><<<grid, tcy::kThreads, tcy::kSmemBytes, st>>>(in, out, d, rows_in, n_in, rows_out,
                                                                               n_out, F, tw, b, flag);
    return cuda_status(cudaGetLastError());
}

}  // namespace pnp
