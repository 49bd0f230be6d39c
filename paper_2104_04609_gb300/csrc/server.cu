// server.cu -- continuous-batching serving loop for OSRC-PMCHWT solve
// requests (resident state kept across requests, admission by device memory).
//
// A worker thread owns the GPU work.  A request with one right-hand side is
// one GMRES job; a request with several is one block job (same-mesh
// right-hand sides batched): matrix-free requests run GMRES in lockstep over
// their right-hand sides with one several-right-hand-side far-field launch
// per iteration, FP64-dense requests the batched mixed-precision solve.
// Jobs are admitted into a fixed number of slots as slots free up and as the
// context's device-memory budget allows; each slot has its own CUDA stream
// and its own workspace (a clone of a resident problem), so the kernels of
// different jobs overlap on the device while each job's result stays
// bit-identical to a solve of the same request alone (every kernel is
// deterministic and no launch configuration depends on the mix).  Problems
// (mesh topology, near-field CSR, M, S, Pade constants) are cached by mesh
// and parameters: right-hand sides of one request, and requests on the same
// mesh and frequency, reuse them.  Unreferenced cache entries are evicted in
// least-recently-used order when memory is needed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "osrc_internal.cuh"

extern "C" int osrc_dense_batched_solve(osrc_problem *pb, const void *b, void *x, int nrhs, double tol,
                                        int max_refine, double inner_tol, int inner_maxit, double precond_tol,
                                        osrc_batched_info *info, void *stream);
extern "C" int osrc_dense_precond_build(osrc_problem *pb, double tol, int maxit, void *stream);

namespace {

constexpr int BATCH_MAX = 128;        // right-hand sides per batched block
constexpr int BATCH_INNER_MAXIT = 400;
constexpr double BATCH_INNER_TOL = 1e-3;
constexpr int BATCH_MAX_REFINE = 10;

using Clock = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    std::vector<double> verts;
    std::vector<int> tris;
    int nv = 0, nt = 0;
    osrc_params params{};
    int kind = 0;
    std::vector<double> src;
    int nrhs = 0;
    double tol = 1e-5;
    int maxit = 500;
    std::string key;
    Clock::time_point t_submit, t_start, t_done;
    bool started = false;  // t_start set (first job admitted)
    int next_rhs = 0;
    int rhs_done = 0;
    int inflight = 0;  // jobs of this request running in slots
    int status = OSRC_OK;
    bool finished = false;
    std::vector<double2> x;  // nrhs x 2nv
    osrc_solve_info info{};
};

struct CacheEntry {
    osrc_mesh *mesh = nullptr;
    osrc_problem *pb = nullptr;
    int refs = 0;
    uint64_t last_use = 0;
    bool precond_built = false;  // explicit preconditioner matrix of the batched solve
    bool batched_busy = false;   // a batched job is using this problem's batched state
};

struct Slot {
    osrc_problem *work = nullptr;  // workspace clone of entry->pb
    CacheEntry *entry = nullptr;
    std::string entry_key;
    cudaStream_t st = nullptr;
    GmresRun run;
    Request *req = nullptr;
    int rhs = -1;
    DBuf<double2> d_b, d_x;
    bool busy = false;
    // a batched job (all right-hand sides of one request) runs on its own host
    // thread with this slot's stream; bdone is set under the server mutex
    bool batched = false;
    std::thread bth;
    CacheEntry *bentry = nullptr;
    bool bdone = false;
    int bstatus = OSRC_OK;
    osrc_solve_info binfo{};
    bool lockstep = false;  // the block is a matrix-free lockstep GMRES, not the dense batched solve
};

constexpr int ADMIT_WAIT = -1;  // the head of the queue must wait (its problem is busy)

uint64_t fnv1a(const void *data, size_t n, uint64_t h) {
    const unsigned char *p = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

std::string request_key(const Request &r) {
    uint64_t h = 1469598103934665603ULL;
    h = fnv1a(r.verts.data(), r.verts.size() * sizeof(double), h);
    h = fnv1a(r.tris.data(), r.tris.size() * sizeof(int), h);
    const osrc_params &p = r.params;
    const double d[] = {p.k_ext, p.k_int, p.rho_ratio, p.theta, p.damping_R, p.inner_tol, p.k_int_im};
    const int i[] = {p.n_pade, p.osrc_side, p.n_ss, p.precision, p.inner_maxit, p.precond, p.formulation,
                     p.dense_assembly, r.nv, r.nt};
    h = fnv1a(d, sizeof(d), h);
    h = fnv1a(i, sizeof(i), h);
    char buf[32];
    snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
    return std::string(buf);
}

}  // namespace

struct osrc_server {
    osrc_ctx *ctx = nullptr;
    int max_active = 1;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;  // requests with right-hand sides not yet started
    std::map<long long, std::unique_ptr<Request>> reqs;
    std::map<std::string, CacheEntry> cache;
    std::vector<Slot> slots;
    std::thread worker;
    std::atomic<bool> stop{false};
    long long next_id = 1;
    uint64_t tick = 0;
    osrc_server_stats stats{};
    int worker_error = OSRC_OK;

    void run();
    int admit_one(Slot &slot);
    int start_batched(Slot &slot, Request *r);
    void batched_body(Slot &slot, Request *r, CacheEntry *entry);
    void lockstep_body(Slot &slot, Request *r, CacheEntry *entry);
    void finish_batched(Slot &slot);
    int acquire_entry(Request *r, CacheEntry **out, cudaStream_t st);
    void release_slot_workspace(Slot &slot);
    bool evict_one();
    void finish_job(Slot &slot, int status);
    void reclaim_all();
};

// Frees every idle slot's workspace and every unreferenced resident problem.
void osrc_server::reclaim_all() {
    for (Slot &s : slots)
        if (!s.busy) release_slot_workspace(s);
    while (evict_one()) {
    }
}

bool osrc_server::evict_one() {
    auto victim = cache.end();
    for (auto it = cache.begin(); it != cache.end(); ++it)
        if (it->second.refs == 0 && (victim == cache.end() || it->second.last_use < victim->second.last_use))
            victim = it;
    if (victim == cache.end()) return false;
    osrc_problem_destroy(victim->second.pb);
    osrc_mesh_destroy(victim->second.mesh);
    cache.erase(victim);
    stats.evictions++;
    return true;
}

void osrc_server::release_slot_workspace(Slot &slot) {
    if (slot.work) {
        osrc_problem_destroy(slot.work);
        slot.work = nullptr;
    }
    if (slot.entry) {
        slot.entry->refs--;
        slot.entry = nullptr;
    }
    slot.entry_key.clear();
    slot.d_b.release();
    slot.d_x.release();
}

int osrc_server::acquire_entry(Request *r, CacheEntry **out, cudaStream_t st) {
    auto it = cache.find(r->key);
    if (it != cache.end()) {
        stats.cache_hits++;
        *out = &it->second;
        return OSRC_OK;
    }
    const size_t need = estimate_problem_bytes(r->nv, r->nt, r->params);
    while (ctx->budget && ctx->used + need > ctx->budget)
        if (!evict_one()) return OSRC_OUT_OF_MEMORY;
    CacheEntry e;
    int s = osrc_mesh_create(ctx, r->verts.data(), r->nv, r->tris.data(), r->nt, &e.mesh);
    if (s != OSRC_OK) return s;
    s = osrc_problem_create(e.mesh, &r->params, &e.pb, st);
    if (s != OSRC_OK) {
        osrc_mesh_destroy(e.mesh);
        return s;
    }
    stats.cache_misses++;
    auto res = cache.emplace(r->key, e);
    *out = &res.first->second;
    return OSRC_OK;
}

// Starts the next right-hand side of the oldest pending request in `slot`.
// Returns OSRC_OK if a job was started, OSRC_OUT_OF_MEMORY if it must wait,
// another status if the request failed.
int osrc_server::admit_one(Slot &slot) {
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        while (!pending.empty() && (pending.front()->finished || pending.front()->status != OSRC_OK))
            pending.pop_front();
        if (pending.empty()) return OSRC_TIMEOUT;  // nothing to do
        r = pending.front();
    }
    if (r->params.precision == OSRC_FP64_DENSE) return start_batched(slot, r);
    if (r->nrhs > 1 && r->params.precond != OSRC_PRECOND_CALDERON) return start_batched(slot, r);
    // workspace: reuse the slot's clone if it serves the same problem
    CacheEntry *entry = nullptr;
    if (slot.entry && slot.entry_key == r->key) {
        entry = slot.entry;
    } else {
        release_slot_workspace(slot);
        int s = acquire_entry(r, &entry, slot.st);
        if (s != OSRC_OK) return s;
        const size_t need = estimate_work_bytes(r->nv, r->nt, r->params, r->maxit);
        while (ctx->budget && ctx->used + need > ctx->budget) {
            entry->refs++;  // keep the entry this job needs
            const bool ok = evict_one();
            entry->refs--;
            if (!ok) return OSRC_OUT_OF_MEMORY;
        }
        osrc_problem *w = nullptr;
        s = problem_clone(entry->pb, &w);
        if (s != OSRC_OK) return s;
        slot.work = w;
        slot.entry = entry;
        slot.entry_key = r->key;
        entry->refs++;
        if ((s = slot.d_b.alloc(ctx, 2 * (size_t)r->nv)) || (s = slot.d_x.alloc(ctx, 2 * (size_t)r->nv))) {
            release_slot_workspace(slot);
            return s;
        }
        int s2 = ensure_gmres_workspace(slot.work, r->maxit);
        if (s2 != OSRC_OK) {
            release_slot_workspace(slot);
            return s2;
        }
    }
    entry->last_use = ++tick;
    int rhs;
    {
        std::lock_guard<std::mutex> lock(mu);
        rhs = r->next_rhs++;
        r->inflight++;
        if (!r->started) {
            r->started = true;
            r->t_start = Clock::now();
        }
        if (r->next_rhs >= r->nrhs) pending.pop_front();
    }
    slot.req = r;
    slot.rhs = rhs;
    slot.busy = true;
    int s = rhs_build(slot.work, r->kind, r->src.data() + 3 * rhs, slot.d_b.p, slot.st);
    if (s == OSRC_OK) s = slot.run.start(slot.work, slot.st, slot.d_b.p, slot.d_x.p, r->tol, r->maxit);
    if (s != OSRC_OK) {
        finish_job(slot, s);
        return OSRC_OK;
    }
    stats.jobs_started++;
    if (ctx->used > stats.mem_peak) stats.mem_peak = ctx->used;
    return OSRC_OK;
}

// Starts a batched job: every right-hand side of request r, as blocks of up
// to BATCH_MAX, by the batched mixed-precision solve on the cached problem.
// The GPU work runs on a host thread of its own (the worker keeps advancing
// the other slots); one batched job per resident problem at a time.  Returns
// OSRC_OUT_OF_MEMORY or ADMIT_WAIT (request left queued) if it cannot start
// yet.
int osrc_server::start_batched(Slot &slot, Request *r) {
    release_slot_workspace(slot);  // the block runs on the resident problem, not on a clone
    auto it = cache.find(r->key);
    if (it != cache.end() && it->second.batched_busy) return ADMIT_WAIT;
    CacheEntry *entry = nullptr;
    int s = acquire_entry(r, &entry, slot.st);
    if (s != OSRC_OK) return s;
    entry->refs++;
    const bool lockstep = r->params.precision != OSRC_FP64_DENSE;
    const int blk = std::min(r->nrhs, BATCH_MAX);
    size_t need, have;
    if (lockstep) {  // one GMRES workspace per right-hand side in flight, and the block's vectors
        need = (size_t)std::min(r->nrhs, 16) * estimate_work_bytes(r->nv, r->nt, r->params, r->maxit) +
               (size_t)r->nrhs * 2 * r->nv * 32;
        have = need;
    } else {
        need = estimate_batched_bytes(r->nv, r->params.n_pade, blk, BATCH_INNER_MAXIT) +
               (size_t)blk * 2 * r->nv * 32;
        have = entry->pb->batched ? 0 : need;  // state of an earlier block is reused
    }
    while (ctx->budget && ctx->used + have > ctx->budget)
        if (!evict_one()) {
            entry->refs--;
            return OSRC_OUT_OF_MEMORY;
        }
    {
        std::lock_guard<std::mutex> lock(mu);
        r->next_rhs = r->nrhs;
        r->inflight++;
        pending.pop_front();
        if (!r->started) {
            r->started = true;
            r->t_start = Clock::now();
        }
    }
    entry->last_use = ++tick;
    entry->batched_busy = true;
    stats.jobs_started++;
    stats.batched_jobs++;
    slot.req = r;
    slot.busy = true;
    slot.batched = true;
    slot.bentry = entry;
    slot.bdone = false;
    slot.lockstep = lockstep;
    if (lockstep) slot.bth = std::thread([this, &slot, r, entry] { lockstep_body(slot, r, entry); });
    else slot.bth = std::thread([this, &slot, r, entry] { batched_body(slot, r, entry); });
    return OSRC_OK;
}

// The GPU work of a matrix-free request with several right-hand sides: GMRES
// advanced in lockstep over all of them (osrc_gmres_solve), sharing one
// far-field launch per iteration for the right-hand sides still iterating.
// Runs on its own host thread with the slot's stream, like a batched job.
void osrc_server::lockstep_body(Slot &slot, Request *r, CacheEntry *entry) {
    cudaSetDevice(ctx->device);
    const int n2 = 2 * r->nv;
    int status = OSRC_OK, s;
    osrc_solve_info info{};
    if ((s = slot.d_b.alloc(ctx, (size_t)r->nrhs * n2)) || (s = slot.d_x.alloc(ctx, (size_t)r->nrhs * n2)))
        status = s;
    for (int i = 0; i < r->nrhs && status == OSRC_OK; ++i)
        status = rhs_build(entry->pb, r->kind, r->src.data() + 3 * (size_t)i, slot.d_b.p + (size_t)i * n2, slot.st);
    if (status == OSRC_OK) {
        entry->pb->cancel = &stop;  // server shutdown ends the solve at its next iteration
        const int gs = osrc_gmres_solve(entry->pb, slot.d_b.p, slot.d_x.p, r->nrhs, r->tol, r->maxit, 0, &info,
                                        slot.st);
        entry->pb->cancel = nullptr;
        if (gs != OSRC_OK && gs != OSRC_NOT_CONVERGED) status = gs;
        if (status == OSRC_OK &&
            (cudaMemcpyAsync(r->x.data(), slot.d_x.p, (size_t)r->nrhs * n2 * sizeof(double2),
                             cudaMemcpyDeviceToHost, slot.st) != cudaSuccess ||
             cudaStreamSynchronize(slot.st) != cudaSuccess))
            status = OSRC_CUDA_ERROR;
    }
    std::lock_guard<std::mutex> lock(mu);
    slot.bstatus = status;
    slot.binfo = info;
    slot.bdone = true;
}

// The GPU work of a batched job (its own host thread; touches only the job's
// slot buffers, stream and problem, and the request's result).
void osrc_server::batched_body(Slot &slot, Request *r, CacheEntry *entry) {
    cudaSetDevice(ctx->device);
    const int blk = std::min(r->nrhs, BATCH_MAX);
    const int n2 = 2 * r->nv;
    int status = OSRC_OK, s;
    osrc_solve_info agg{};
    agg.converged = 1;
    if ((s = slot.d_b.alloc(ctx, (size_t)blk * n2)) || (s = slot.d_x.alloc(ctx, (size_t)blk * n2))) status = s;
    if (status == OSRC_OK && !entry->precond_built) {
        status = osrc_dense_precond_build(entry->pb, 1e-3, 500, slot.st);
        entry->precond_built = status == OSRC_OK;
    }
    for (int r0 = 0; status == OSRC_OK && r0 < r->nrhs; r0 += BATCH_MAX) {
        const int nb = std::min(BATCH_MAX, r->nrhs - r0);
        for (int i = 0; i < nb && status == OSRC_OK; ++i)
            status = rhs_build(entry->pb, r->kind, r->src.data() + 3 * (size_t)(r0 + i), slot.d_b.p + (size_t)i * n2,
                               slot.st);
        if (status != OSRC_OK) break;
        osrc_batched_info bi{};
        const int bs = osrc_dense_batched_solve(entry->pb, slot.d_b.p, slot.d_x.p, nb, r->tol, BATCH_MAX_REFINE,
                                                BATCH_INNER_TOL, BATCH_INNER_MAXIT, 0.0, &bi, slot.st);
        if (bs != OSRC_OK && bs != OSRC_NOT_CONVERGED) {
            status = bs;
            break;
        }
        if (bs == OSRC_NOT_CONVERGED) agg.converged = 0;
        if (cudaMemcpyAsync(r->x.data() + (size_t)r0 * n2, slot.d_x.p, (size_t)nb * n2 * sizeof(double2),
                            cudaMemcpyDeviceToHost, slot.st) != cudaSuccess ||
            cudaStreamSynchronize(slot.st) != cudaSuccess) {
            status = OSRC_CUDA_ERROR;
            break;
        }
        agg.iterations += bi.inner_iterations;
        agg.total_iterations += bi.inner_iterations;
        agg.true_residual = fmax(agg.true_residual, bi.residual);
    }
    std::lock_guard<std::mutex> lock(mu);
    slot.bstatus = status;
    slot.binfo = agg;
    slot.bdone = true;
}

// Worker side of a finished batched job: joins its thread, releases its
// buffers and finishes the request.
void osrc_server::finish_batched(Slot &slot) {
    if (slot.bth.joinable()) slot.bth.join();
    slot.d_b.release();
    slot.d_x.release();
    CacheEntry *entry = slot.bentry;
    entry->refs--;
    entry->batched_busy = false;
    if (ctx->used > stats.mem_peak) stats.mem_peak = ctx->used;
    Request *r = slot.req;
    int status = slot.bstatus;
    const osrc_solve_info &agg = slot.binfo;
    {
        std::lock_guard<std::mutex> lock(mu);
        r->info.iterations = agg.iterations;
        r->info.total_iterations = agg.total_iterations;
        r->info.true_residual = agg.true_residual;
        r->info.precond_residual = slot.lockstep ? agg.precond_residual : agg.true_residual;
        r->info.converged = agg.converged;
        r->info.ms_matvec = agg.ms_matvec;
        r->info.ms_precond = agg.ms_precond;
        r->info.ms_arnoldi = agg.ms_arnoldi;
        if (status == OSRC_OK && !agg.converged) status = OSRC_NOT_CONVERGED;
        r->status = status;
        r->rhs_done = r->nrhs;
        r->inflight--;
        r->finished = true;
        r->t_done = Clock::now();
        r->info.ms_total = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        r->info.ms_queued =
            r->started ? std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count() : r->info.ms_total;
        stats.completed++;
        if (status != OSRC_OK) stats.failed++;
        cv.notify_all();
    }
    slot.req = nullptr;
    slot.bentry = nullptr;
    slot.batched = false;
    slot.lockstep = false;
    slot.bdone = false;
    slot.busy = false;
}

void osrc_server::finish_job(Slot &slot, int status) {
    Request *r = slot.req;
    const int n = 2 * r->nv;
    if (status == OSRC_OK || status == OSRC_NOT_CONVERGED) {
        cudaMemcpyAsync(r->x.data() + (size_t)n * slot.rhs, slot.d_x.p, n * sizeof(double2),
                        cudaMemcpyDeviceToHost, slot.st);
        if (cudaStreamSynchronize(slot.st) != cudaSuccess) status = OSRC_CUDA_ERROR;
    }
    std::lock_guard<std::mutex> lock(mu);
    const osrc_solve_info &ri = slot.run.info;
    r->info.iterations = ri.iterations;
    r->info.precond_residual = fmax(r->info.precond_residual, ri.precond_residual);
    r->info.true_residual = fmax(r->info.true_residual, ri.true_residual);
    r->info.ms_matvec += ri.ms_matvec;
    r->info.ms_precond += ri.ms_precond;
    r->info.ms_arnoldi += ri.ms_arnoldi;
    r->info.total_iterations += ri.iterations;
    if (!slot.run.converged) r->info.converged = 0;
    const bool hard_error = status != OSRC_OK && status != OSRC_NOT_CONVERGED;
    if (status != OSRC_OK && (r->status == OSRC_OK || hard_error)) r->status = status;
    r->rhs_done++;
    r->inflight--;
    // a request finishes when every right-hand side is done, or after an
    // error once none of its jobs is still running (no more are started)
    const bool failed = r->status != OSRC_OK && r->status != OSRC_NOT_CONVERGED;
    if (r->inflight == 0 && (r->rhs_done >= r->nrhs || failed)) {
        if (!r->finished) {
            r->finished = true;
            r->t_done = Clock::now();
            r->info.ms_total = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
            r->info.ms_queued =
            r->started ? std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count() : r->info.ms_total;
            stats.completed++;
            if (r->status != OSRC_OK) stats.failed++;
        }
        cv.notify_all();
    }
    slot.req = nullptr;
    slot.rhs = -1;
    slot.busy = false;
}

void osrc_server::run() {
    cudaSetDevice(ctx->device);
    while (!stop.load()) {
        bool progress = false;
        int busy = 0;
        for (Slot &s : slots) busy += s.busy ? 1 : 0;
        for (Slot &s : slots) {
            if (s.busy) continue;
            const int a = admit_one(s);
            if (a == OSRC_OK) {
                progress = true;
                ++busy;
                continue;
            }
            if (a == OSRC_TIMEOUT || a == ADMIT_WAIT) break;  // queue empty, or its head must wait
            if (a == OSRC_OUT_OF_MEMORY && busy > 0) break;  // wait for memory
            if (a == OSRC_OUT_OF_MEMORY) {
                // nothing runs: free everything idle and try once more
                reclaim_all();
                const int b = admit_one(s);
                if (b == OSRC_OK) {
                    progress = true;
                    ++busy;
                    continue;
                }
            }
            // the request at the head of the queue cannot be served
            std::lock_guard<std::mutex> lock(mu);
            Request *r = pending.empty() ? nullptr : pending.front();
            if (r) {
                pending.pop_front();
                r->status = a;
                if (!r->finished) {
                    r->finished = true;
                    r->t_done = Clock::now();
                    stats.completed++;
                    stats.failed++;
                }
                cv.notify_all();
            }
            progress = true;
        }
        if (busy > stats.active_peak) stats.active_peak = busy;
        for (Slot &s : slots) {
            if (s.busy && s.batched) {
                bool done;
                {
                    std::lock_guard<std::mutex> lock(mu);
                    done = s.bdone;
                }
                if (done) {
                    finish_batched(s);
                    progress = true;
                }
                continue;
            }
            if (!s.busy || !s.run.ready()) continue;
            const int st = s.run.advance();
            progress = true;
            if (st != OSRC_OK) {
                finish_job(s, st);
            } else if (s.run.done()) {
                const int fs = s.run.status != OSRC_OK ? s.run.status
                                                       : (s.run.converged ? OSRC_OK : OSRC_NOT_CONVERGED);
                finish_job(s, fs);
            }
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int osrc_server_create(osrc_ctx *ctx, int max_active, osrc_server **out) {
    if (!ctx || !out || max_active < 1 || max_active > 64) return OSRC_INVALID_ARG;
    *out = nullptr;
    OSRC_CK(cudaSetDevice(ctx->device));
    osrc_server *sv = new osrc_server;
    sv->ctx = ctx;
    sv->max_active = max_active;
    sv->slots.resize(max_active);
    for (Slot &s : sv->slots) {
        if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess) {
            for (Slot &t : sv->slots)
                if (t.st) cudaStreamDestroy(t.st);
            delete sv;
            return OSRC_CUDA_ERROR;
        }
    }
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return OSRC_OK;
}

extern "C" int osrc_server_submit(osrc_server *sv, const osrc_request *rq, long long *id_out) {
    if (!sv || !rq || !id_out || !rq->verts || !rq->tris || !rq->src || rq->nrhs < 1 ||
        !(rq->tol > 0.0) || rq->maxit < 1 || (rq->rhs_kind != 0 && rq->rhs_kind != 1))
        return OSRC_INVALID_ARG;
    OSRC_TRY(osrc_mesh_validate(rq->verts, rq->nv, rq->tris, rq->nt));
    auto r = std::make_unique<Request>();
    r->verts.assign(rq->verts, rq->verts + 3 * (size_t)rq->nv);
    r->tris.assign(rq->tris, rq->tris + 3 * (size_t)rq->nt);
    r->nv = rq->nv;
    r->nt = rq->nt;
    r->params = rq->params;
    r->kind = rq->rhs_kind;
    r->src.assign(rq->src, rq->src + 3 * (size_t)rq->nrhs);
    r->nrhs = rq->nrhs;
    r->tol = rq->tol;
    r->maxit = rq->maxit;
    r->key = request_key(*r);
    r->x.assign((size_t)rq->nrhs * 2 * rq->nv, cd(0, 0));
    r->info.converged = 1;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(sv->mu);
    r->id = sv->next_id++;
    *id_out = r->id;
    sv->pending.push_back(r.get());
    sv->reqs.emplace(r->id, std::move(r));
    sv->stats.submitted++;
    return OSRC_OK;
}

extern "C" int osrc_server_poll(osrc_server *sv, long long id, int *done, double *latency_ms,
                                osrc_solve_info *info) {
    if (!sv || !done) return OSRC_INVALID_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return OSRC_INVALID_ARG;
    Request *r = it->second.get();
    *done = r->finished ? 1 : 0;
    if (r->finished) {
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        if (info) *info = r->info;
        return r->status;
    }
    return OSRC_OK;
}

extern "C" int osrc_server_wait(osrc_server *sv, long long id, double timeout_s) {
    if (!sv || !(timeout_s >= 0.0)) return OSRC_INVALID_ARG;
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return OSRC_INVALID_ARG;
    Request *r = it->second.get();
    const bool ok = sv->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), [r] { return r->finished; });
    if (!ok) return OSRC_TIMEOUT;
    return r->status;
}

extern "C" int osrc_server_result(osrc_server *sv, long long id, void *x_host) {
    if (!sv || !x_host) return OSRC_INVALID_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return OSRC_INVALID_ARG;
    Request *r = it->second.get();
    if (!r->finished) return OSRC_TIMEOUT;
    std::memcpy(x_host, r->x.data(), r->x.size() * sizeof(double2));
    const int s = r->status;
    sv->reqs.erase(it);
    return s;
}

extern "C" int osrc_server_get_stats(osrc_server *sv, osrc_server_stats *out) {
    if (!sv || !out) return OSRC_INVALID_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    *out = sv->stats;
    out->mem_used = sv->ctx->used;
    return OSRC_OK;
}

extern "C" void osrc_server_destroy(osrc_server *sv) {
    if (!sv) return;
    sv->stop.store(true);
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot &s : sv->slots)  // batched jobs still running finish first
        if (s.bth.joinable()) s.bth.join();
    cudaSetDevice(sv->ctx->device);
    for (Slot &s : sv->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        sv->release_slot_workspace(s);
    }
    for (auto &kv : sv->cache) {
        osrc_problem_destroy(kv.second.pb);
        osrc_mesh_destroy(kv.second.mesh);
    }
    sv->cache.clear();
    for (Slot &s : sv->slots)
        if (s.st) cudaStreamDestroy(s.st);
    delete sv;
}
