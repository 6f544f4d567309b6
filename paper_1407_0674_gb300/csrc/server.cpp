// Serving loop: a queue of independent Gummel solves running concurrently on
// one GPU (pnp_server_* in include/pnp.h).
//
// A worker thread admits queued requests (in arrival order, or smallest first
// with PNP_SERVE_SMALLEST_FIRST) while a slot is free and the request's device footprint (estimated
// from its plan before anything is allocated) fits the memory budget; a
// preparer thread per admitted request builds the problem and launches its
// whole solve -- one CUDA graph whose loops end on the device -- on the
// problem's own stream, followed by copies of the result into pinned host
// memory and an event.  Solves therefore overlap on
// the GPU; requests that arrive while others run are admitted as soon as a
// slot and memory free up.  Completion is detected with cudaEventQuery (the
// worker never blocks on one solve); finished results wait in host memory
// until pnp_poll takes them.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "pnp_internal.h"

namespace pnp {

struct Request {
    uint64_t ticket = 0;
    pnp_problem_desc desc{};
    // owned copies of every array the descriptor points to
    std::vector<int> q;
    std::vector<double> R, rho_b, D, depth, sites, rho_f, phi0, rho0;
    size_t bytes = 0;
    size_t npts = 0;
    int s = 0;
    // running state
    Problem *prob = nullptr;
    cudaStream_t own_stream = nullptr;           // priority stream (PNP_SERVE_SMALLEST_FIRST)
    cudaEvent_t done_ev = nullptr;
    double *h_phi = nullptr, *h_rho = nullptr;   // pinned
    void *h_stats = nullptr;                     // pinned
    // result
    bool finished = false;
    int status = PNP_PENDING;
    std::vector<double> phi, rho;
    pnp_stats stats{};
    std::chrono::steady_clock::time_point t_submit, t_start, t_end;
};

}  // namespace pnp

namespace pnp {
// Pinned host buffers are recycled: cudaFreeHost would wait for the whole
// device, stalling every running solve.  Freed only when the server goes.
struct PinnedPool {
    std::mutex mu;
    std::multimap<size_t, void *> idle;
    std::map<void *, size_t> size_of;
    void *get(size_t n) {
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = idle.lower_bound(n);
            if (it != idle.end() && it->first <= 2 * n + 4096) {
                void *p = it->second;
                idle.erase(it);
                return p;
            }
        }
        void *p = nullptr;
        if (cudaMallocHost(&p, n) != cudaSuccess) return nullptr;
        std::lock_guard<std::mutex> lk(mu);
        size_of[p] = n;
        return p;
    }
    void put(void *p) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        idle.emplace(size_of[p], p);
    }
    ~PinnedPool() {
        for (auto &kv : size_of) cudaFreeHost(kv.first);
    }
};
}  // namespace pnp

struct pnp_server {
    pnp_server_opts opts{};
    pnp::PinnedPool pinned;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<pnp::Request *> queue;
    std::vector<pnp::Request *> running;   // launched, not yet retired (worker and preparers, under mu)
    int preparing = 0;                     // admitted requests whose problem is being built
    std::condition_variable prepared;      // signalled when a preparer ends
    std::map<uint64_t, pnp::Request *> all;
    size_t bytes_in_use = 0;
    long long submitted = 0, completed = 0, failed = 0, rejected = 0;
};

namespace pnp {

static void deep_copy(const pnp_problem_desc *d, Request *r, const double *phi0, const double *rho0) {
    r->desc = *d;
    const int s = d->nspecies;
    const size_t N = (size_t)d->nx * d->ny * d->nz;
    r->q.assign(d->valence, d->valence + s);
    r->R.assign(d->radius, d->radius + s);
    r->rho_b.assign(d->rho_bulk, d->rho_bulk + s);
    if (d->diffusivity) r->D.assign(d->diffusivity, d->diffusivity + s);
    if (d->well_depth) r->depth.assign(d->well_depth, d->well_depth + s);
    if (d->nsites > 0) r->sites.assign(d->site_xyz, d->site_xyz + 3 * (size_t)d->nsites);
    if (d->rho_fixed) r->rho_f.assign(d->rho_fixed, d->rho_fixed + N);
    if (phi0) r->phi0.assign(phi0, phi0 + N);
    if (rho0) r->rho0.assign(rho0, rho0 + N * s);
    r->desc.valence = r->q.data();
    r->desc.radius = r->R.data();
    r->desc.rho_bulk = r->rho_b.data();
    r->desc.diffusivity = r->D.empty() ? nullptr : r->D.data();
    r->desc.well_depth = r->depth.empty() ? nullptr : r->depth.data();
    r->desc.site_xyz = r->sites.empty() ? nullptr : r->sites.data();
    r->desc.rho_fixed = r->rho_f.empty() ? nullptr : r->rho_f.data();
    r->npts = N;
    r->s = s;
}

static void release(pnp_server *s, Request *r) {
    if (r->prob) destroy_problem_internal(r->prob);
    r->prob = nullptr;
    if (r->own_stream) cudaStreamDestroy(r->own_stream);
    r->own_stream = nullptr;
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    r->done_ev = nullptr;
    s->pinned.put(r->h_phi);
    s->pinned.put(r->h_rho);
    s->pinned.put(r->h_stats);
    r->h_phi = r->h_rho = nullptr;
    r->h_stats = nullptr;
}

// start one admitted request: build the problem and enqueue its whole solve
static int start(pnp_server *s, Request *r) {
    NvtxRange range("server_admit");
    std::string why;
    int rc = create_problem_internal(&r->desc, &r->prob, &why);
    if (rc) return rc;
    Problem *p = r->prob;
    const size_t N = r->npts;
    cudaError_t e = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
    r->h_phi = (double *)s->pinned.get(sizeof(double) * N);
    r->h_rho = (double *)s->pinned.get(sizeof(double) * N * r->s);
    r->h_stats = s->pinned.get(gummel_stats_bytes());
    if (!r->h_phi || !r->h_rho || !r->h_stats) return PNP_ERR_NOMEM;
    cudaStream_t st = p->stream;
    if (s->opts.policy == PNP_SERVE_SMALLEST_FIRST) {
        // one priority level per factor 8 in grid points: 32^3 and smaller
        // highest, up to the lowest level the device offers
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e != cudaSuccess) return cuda_status(e);
        const int level = std::max(0, (int)std::floor(std::log2((double)std::max<size_t>(N, 1)) / 3.0) - 5);
        const int prio = std::min(least, greatest + level);
        e = cudaStreamCreateWithPriority(&r->own_stream, cudaStreamNonBlocking, prio);
        if (e != cudaSuccess) return cuda_status(e);
        st = r->own_stream;
    }
    const double *d_phi0 = nullptr, *d_rho0 = nullptr;
    if (!r->phi0.empty() || !r->rho0.empty()) {
        const size_t n = N * r->s;
        if (dmalloc((void **)&p->d_io, sizeof(double) * (2 * n + N), st) != cudaSuccess) return PNP_ERR_NOMEM;
        if (!r->rho0.empty()) {
            e = cudaMemcpyAsync(p->d_io, r->rho0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
            d_rho0 = p->d_io;
        }
        if (!r->phi0.empty() && e == cudaSuccess) {
            e = cudaMemcpyAsync(p->d_io + n, r->phi0.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st);
            d_phi0 = p->d_io + n;
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    rc = gummel_launch(p, d_phi0, d_rho0, st);
    if (rc) return rc;
    rc = gummel_fetch(p, r->h_phi, r->h_rho, r->h_stats, st);
    if (rc) return rc;
    return cuda_status(cudaEventRecord(r->done_ev, st));
}

static void finish(pnp_server *s, Request *r, int status) {
    NvtxRange range("server_retire");
    r->t_end = std::chrono::steady_clock::now();
    if (status == PNP_PENDING) {
        gummel_decode_stats(r->h_stats, &r->stats);
        status = r->stats.status;
        r->phi.assign(r->h_phi, r->h_phi + r->npts);
        r->rho.assign(r->h_rho, r->h_rho + r->npts * r->s);
    } else {
        r->stats.status = status;
    }
    r->stats.seconds = std::chrono::duration<double>(r->t_end - r->t_start).count();
    r->status = status;
    release(s, r);
    std::lock_guard<std::mutex> lk(s->mu);
    s->bytes_in_use -= r->bytes;
    r->finished = true;
    if (status == PNP_OK || status == PNP_ERR_NOT_CONVERGED) s->completed++;
    else s->failed++;
}

// Build an admitted request's problem and launch its solve on a thread of its
// own: problem creation (validation, spectra, set-up kernels, graph
// recording) is host-heavy and waits for its own set-up work on a busy GPU,
// so several run side by side while the worker keeps retiring solves.
static void prepare(pnp_server *s, Request *r) {
    cudaSetDevice(s->device);
    r->t_start = std::chrono::steady_clock::now();
    const int rc = start(s, r);
    if (rc) finish(s, r, rc);
    std::lock_guard<std::mutex> lk(s->mu);
    if (!rc) s->running.push_back(r);
    s->preparing--;
    s->prepared.notify_all();
}

static void worker_main(pnp_server *s) {
    cudaSetDevice(s->device);
    while (true) {
        // admit while a slot is free and the budget allows; each admitted
        // request is prepared on its own thread
        std::vector<Request *> done;
        bool idle = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->running.empty() && s->queue.empty() && s->preparing == 0)
                s->cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->stop || !s->queue.empty(); });
            if (s->stop) break;
            while (!s->queue.empty() && (int)s->running.size() + s->preparing < s->opts.max_slots) {
                auto it = s->queue.begin();
                if (s->opts.policy == PNP_SERVE_SMALLEST_FIRST)
                    it = std::min_element(s->queue.begin(), s->queue.end(), [](const Request *a, const Request *b) {
                        const size_t wa = a->npts * (a->s + 1), wb = b->npts * (b->s + 1);
                        return wa != wb ? wa < wb : a->ticket < b->ticket;
                    });
                Request *r = *it;
                if (s->bytes_in_use + r->bytes > s->opts.hbm_budget_bytes) break;
                s->queue.erase(it);
                s->bytes_in_use += r->bytes;
                s->preparing++;
                std::thread(prepare, s, r).detach();
            }
            // retire finished solves without blocking on any one of them
            for (size_t k = 0; k < s->running.size();) {
                Request *r = s->running[k];
                if (cudaEventQuery(r->done_ev) == cudaErrorNotReady) {
                    ++k;
                    continue;
                }
                done.push_back(r);
                s->running[k] = s->running.back();
                s->running.pop_back();
            }
            idle = done.empty();
        }
        for (Request *r : done) {
            const cudaError_t q = cudaEventQuery(r->done_ev);
            finish(s, r, q == cudaSuccess ? PNP_PENDING : PNP_ERR_CUDA);
        }
        if (idle) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    // drain: wait for the preparers, then for what is on the device, and drop it
    std::vector<Request *> left;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->prepared.wait(lk, [&] { return s->preparing == 0; });
        left.swap(s->running);
    }
    for (Request *r : left) {
        if (r->done_ev) cudaEventSynchronize(r->done_ev);
        finish(s, r, PNP_ERR_CUDA);
    }
}

}  // namespace pnp

using namespace pnp;

extern "C" {

int pnp_server_create(const pnp_server_opts *opts, pnp_server **out) {
    if (!out) return PNP_ERR_INVALID;
    *out = nullptr;
    pnp_server *s = new (std::nothrow) pnp_server();
    if (!s) return PNP_ERR_NOMEM;
    if (opts) s->opts = *opts;
    if (s->opts.hbm_budget_bytes == 0) s->opts.hbm_budget_bytes = (size_t)150 << 30;
    if (s->opts.max_slots <= 0) s->opts.max_slots = 64;
    if (s->opts.max_queue <= 0) s->opts.max_queue = 4096;
    if (s->opts.policy != PNP_SERVE_FIFO && s->opts.policy != PNP_SERVE_SMALLEST_FIRST) {
        delete s;
        return PNP_ERR_INVALID;
    }
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return PNP_ERR_CUDA;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return PNP_OK;
}

void pnp_server_destroy(pnp_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->all) {
        release(s, kv.second);
        delete kv.second;
    }
    delete s;
}

int pnp_submit(pnp_server *s, const pnp_problem_desc *desc, const double *phi0, const double *rho0,
               uint64_t *ticket) {
    if (!s || !desc || !ticket) return PNP_ERR_INVALID;
    // validate and size on the host; nothing touches the device here
    Problem probe;
    std::string why;
    int rc = validate_and_copy(desc, &probe, &why);
    if (rc) return rc;
    if (probe.bc[2] != PNP_BC_DIRICHLET || probe.bc[0] == PNP_BC_DIRICHLET || probe.bc[1] == PNP_BC_DIRICHLET)
        return PNP_ERR_INVALID;
    const size_t N = probe.npts();
    if (rho0 && !host_values_ok(rho0, N * probe.s, 2)) return PNP_ERR_INVALID;
    if (phi0 && !host_values_ok(phi0, N, 0)) return PNP_ERR_INVALID;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return PNP_ERR_NOMEM;
    deep_copy(desc, r.get(), phi0, rho0);
    r->bytes = estimate_device_bytes(probe);
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (r->bytes > s->opts.hbm_budget_bytes || (int)s->queue.size() >= s->opts.max_queue) {
            s->rejected++;
            return PNP_ERR_BUSY;
        }
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->all[r->ticket] = r.get();
        s->queue.push_back(r.release());
        s->submitted++;
    }
    s->cv.notify_all();
    return PNP_OK;
}

int pnp_poll(pnp_server *s, uint64_t ticket, double *phi_out, double *rho_out, pnp_stats *stats) {
    if (!s) return PNP_ERR_INVALID;
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return PNP_ERR_UNKNOWN_TICKET;
        r = it->second;
        if (!r->finished) return PNP_PENDING;
        s->all.erase(it);
    }
    if (phi_out && !r->phi.empty()) std::memcpy(phi_out, r->phi.data(), sizeof(double) * r->phi.size());
    if (rho_out && !r->rho.empty()) std::memcpy(rho_out, r->rho.data(), sizeof(double) * r->rho.size());
    if (stats) *stats = r->stats;
    const int status = r->status;
    delete r;
    return status;
}

int pnp_server_get_stats(pnp_server *s, pnp_server_stats *out) {
    if (!s || !out) return PNP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->rejected = s->rejected;
    out->queued = (int)s->queue.size();
    out->active = (int)s->running.size() + s->preparing;
    out->bytes_in_use = s->bytes_in_use;
    return PNP_OK;
}

}  // extern "C"
