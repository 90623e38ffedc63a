// Solve server: continuous batching of independent solves on one GPU.
//
// Requests (L, mode, rtol, host s and b) are queued by cg_batch_submit and
// admitted when a worker slot is free and the device-memory budget holds the
// request's plan.  A slot that admits a request also takes the other queued
// requests of the same size, mode and preconditioning (up to kMaxBatch, as
// the budget allows) and runs them as one batched solve (cg_solve_batch's
// graph: every pass over all of them at once, each with its own tolerance).
// Each slot is a host thread with its own non-blocking CUDA stream; slots
// run their batches concurrently, so requests that arrive while others are
// on the GPU overlap with them.  Plans (spectrum, tables, workspaces) stay
// resident and are reused by later requests of the same L (at most two plans
// per size: a request whose size's plans are all busy waits and joins the
// next batch);
// idle plans of other sizes are evicted when the budget requires it.  Each result is the
// same whether a request runs alone or in a mix: a problem's arithmetic in a
// batched solve depends only on its own inputs and its plan's launch shapes
// (reductions run in a fixed order inside each problem), not on the batch.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fftconv.h"
#include "fc_alloc.h"

// cg_solve_batch with a tolerance per problem (fc_lib.cu).
int fc_batch_solve_rtols(fftconv_plan* p, int nb, const double* s, const double* b, double* x, const cg_opts* o,
                         const double* rtols, cg_result* r, cudaStream_t st);

namespace {

constexpr int kMaxBatch = 64;  // requests one slot takes into one batched solve
// Requests up to this size run on the slots' higher-priority streams: their
// short passes are scheduled ahead of the long ones of large solves, so that
// a small request is not held behind a large one sharing the GPU.
constexpr int kSmallL = 256;

// Plans one size may hold (busy ones included): 2, or FC_SERVER_PLANS_PER_SIZE.
int plans_per_size() {
    static const int n = [] {
        const char* e = getenv("FC_SERVER_PLANS_PER_SIZE");
        const int v = e ? atoi(e) : 0;
        return v >= 1 && v <= 16 ? v : 2;
    }();
    return n;
}

// FC_SERVER_TRACE=1: one line per batched solve on stderr (size, plan made or
// kept, and the wall time of set-up, input copies, solve and output copies).
bool trace_on() {
    static const bool on = [] {
        const char* e = getenv("FC_SERVER_TRACE");
        return e && strcmp(e, "0");
    }();
    return on;
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t ticket = 0;
    cg_request rq{};
    std::vector<double> s, b;  // host copies taken at submit (empty with FC_REQ_BORROW)
    const double* sp() const { return s.empty() ? rq.s : s.data(); }
    const double* bp() const { return b.empty() ? rq.b : b.data(); }
    size_t est = 0;            // device bytes reserved: its plan (if one must be made) and its
                               // share of the plan's batch workspace
    int state = 0;             // 0 queued, 1 running, 2 done
    int rc = 0;
    cg_result res{};
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct Slot {
    std::thread th;
    cudaStream_t stream = nullptr;     // lower priority: requests of L > kSmallL (and staging growth)
    cudaStream_t stream_hi = nullptr;  // higher priority: requests of L <= kSmallL
    cudaEvent_t done = nullptr;  // blocking-sync event: a waiting slot thread sleeps
    double *ds = nullptr, *db = nullptr, *dx = nullptr;  // device staging (stream-ordered)
    long cap = 0;
    std::vector<double> rtols;
    std::vector<cg_result> res;
};

int padded_side(int L) {
    int m = 2;
    while (m < 2 * L) m *= 2;
    return m;
}

// Device bytes of an FC_F32|FC_F64 plan for side L (its allocations, rounded
// up by 1 MiB for tables), plus the slot's staging vectors.
size_t estimate_bytes(int L) {
    const size_t N = (size_t)L * L, M = padded_side(L), Q = M / 2 + 1;
    size_t b = (size_t)L * (M / 2) * (16 + 8);   // FP64 and FP32 half-spectrum intermediates
    b += N * (6 * 8 + 1 + 5 * 4);                // CG vectors and mask
    b += Q * Q * (8 + 4);                        // spectrum quarters
    b += 1 << 20;
    return b;
}

// Device bytes one problem adds to a plan's batch workspace in the given
// mode (as cg_solve_batch allocates it: FP64 iterate, residual, b, s, mask,
// FP64 intermediate, state and partial sums; the mode's inner vectors,
// preconditioner spectrum and, mixed, the FP32 intermediate), plus staging.
size_t batch_bytes(int L, int mode) {
    const size_t N = (size_t)L * L, M = padded_side(L), Q = M / 2 + 1, zs = (M / 2) * (size_t)L;
    size_t b = N * (4 * 8 + 1) + 16 * zs + 512 + 8 * 3 * ((size_t)L + 1);
    if (mode == FC_MODE_MIXED)
        b += N * 6 * 4 + 4 * Q * Q + 8 * zs;
    else
        b += N * 3 * 8 + 8 * Q * Q;
    return b + 3 * 8 * N;  // the slot's device staging of s, b, x
}

}  // namespace

struct cg_server {
    int dev = 0;
    size_t budget = 0, used = 0, peak = 0;
    long long batches = 0, solves = 0;  // batched solves run and the requests they held
    int max_batch = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req*> queue;
    std::unordered_map<uint64_t, Req*> reqs;
    std::multimap<int, fftconv_plan*> idle;      // idle plans by L
    std::map<fftconv_plan*, size_t> plan_bytes;  // every plan held
    std::map<int, int> plans_of;                 // plans held (idle, busy or being made) per L
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<Slot*> slots;
};

namespace {

// Pick the first queued request that can run now: an idle plan of its size
// exists, or its plan fits the budget (possibly after evicting idle plans of
// other sizes).  Called with the lock held.  Returns the request and the plan
// to use (nullptr: create one) and the idle plans to destroy.  The request's
// reservation (r->est) covers its plan when one is made and one problem of
// the plan's batch workspace.
Req* admit_one_locked(cg_server* sv, fftconv_plan** plan, std::vector<fftconv_plan*>& evict) {
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
        Req* r = *it;
        auto ip = sv->idle.find(r->rq.L);
        const bool have = ip != sv->idle.end();
        // every plan this size may hold is busy: the request waits for one
        // (and joins its next batch) rather than making another
        if (!have && sv->plans_of[r->rq.L] >= plans_per_size()) continue;
        const size_t need = have ? batch_bytes(r->rq.L, r->rq.mode) : r->est;
        size_t freeable = 0;
        for (auto& kv : sv->idle)
            if (!have || kv.second != ip->second) freeable += sv->plan_bytes[kv.second];
        if (sv->used + need > sv->budget && sv->used - freeable + need > sv->budget) continue;
        fftconv_plan* keep = have ? ip->second : nullptr;
        if (have) sv->idle.erase(ip);
        while (sv->used + need > sv->budget && !sv->idle.empty()) {
            auto v = sv->idle.begin();
            evict.push_back(v->second);
            sv->used -= sv->plan_bytes[v->second];
            sv->plan_bytes.erase(v->second);
            sv->plans_of[v->first] -= 1;
            sv->idle.erase(v);
        }
        if (!have) sv->plans_of[r->rq.L] += 1;  // the plan this slot will make
        r->est = need;  // reserved until the batch ends
        sv->used += need;
        if (sv->used > sv->peak) sv->peak = sv->used;
        *plan = keep;
        sv->queue.erase(it);
        return r;
    }
    return nullptr;
}

// Admit a request (admit_one_locked) and the queued requests that can join
// its batch: same L, mode and preconditioning, each reserving one problem's
// share of the batch workspace while the budget holds it.
bool admit_locked(cg_server* sv, std::vector<Req*>& batch, fftconv_plan** plan, std::vector<fftconv_plan*>& evict) {
    batch.clear();
    Req* r = admit_one_locked(sv, plan, evict);
    if (!r) return false;
    batch.push_back(r);
    const size_t per = batch_bytes(r->rq.L, r->rq.mode);
    for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)batch.size() < kMaxBatch;) {
        Req* q = *it;
        if (q->rq.L == r->rq.L && q->rq.mode == r->rq.mode && q->rq.precond == r->rq.precond &&
            sv->used + per <= sv->budget) {
            q->est = per;
            sv->used += per;
            batch.push_back(q);
            it = sv->queue.erase(it);
        } else {
            ++it;
        }
    }
    if (sv->used > sv->peak) sv->peak = sv->used;
    return true;
}

// Device staging for n doubles per vector, grown geometrically with
// stream-ordered allocations (no device-wide synchronisation while other
// slots run).  There is no pinned host staging: allocating pinned memory
// takes a driver lock for a long time (measured: 100-250 ms per growth,
// stalling every slot), so the copies go straight from and to the
// requests' own host arrays.
int ensure_staging(Slot* sl, long n) {
    if (n <= sl->cap) return FC_OK;
    long cap = sl->cap > 0 ? sl->cap : n;
    while (cap < n) cap *= 2;
    // nothing of the slot's may still use the old buffers, on either stream
    if (cudaStreamSynchronize(sl->stream_hi) != cudaSuccess || cudaStreamSynchronize(sl->stream) != cudaSuccess)
        return FC_ECUDA;
    fc::dev_free_async(sl->ds, sl->stream);
    fc::dev_free_async(sl->db, sl->stream);
    fc::dev_free_async(sl->dx, sl->stream);
    sl->ds = sl->db = sl->dx = nullptr;
    sl->cap = 0;
    const size_t bytes = sizeof(double) * (size_t)cap;
    if (fc::dev_malloc_async((void**)&sl->ds, bytes, sl->stream) != cudaSuccess ||
        fc::dev_malloc_async((void**)&sl->db, bytes, sl->stream) != cudaSuccess ||
        fc::dev_malloc_async((void**)&sl->dx, bytes, sl->stream) != cudaSuccess)
        return FC_ENOMEM;
    // the buffers may be used on the slot's other stream: their allocation done
    if (cudaStreamSynchronize(sl->stream) != cudaSuccess) return FC_ECUDA;
    sl->cap = cap;
    return FC_OK;
}

void worker(cg_server* sv, Slot* sl) {
    cudaSetDevice(sv->dev);
    std::vector<Req*> batch;
    for (;;) {
        fftconv_plan* plan = nullptr;
        std::vector<fftconv_plan*> evict;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] { return sv->stop || admit_locked(sv, batch, &plan, evict); });
            if (batch.empty()) return;  // stopping
            const double t = now_s();
            for (Req* q : batch) {
                q->state = 1;
                q->t_start = t;
            }
            sv->batches += 1;
            sv->solves += (long long)batch.size();
            if ((int)batch.size() > sv->max_batch) sv->max_batch = (int)batch.size();
        }
        for (fftconv_plan* e : evict) fftconv_plan_destroy(e);
        Req* r = batch[0];
        const int L = r->rq.L, nb = (int)batch.size();
        cudaStream_t st = L <= kSmallL ? sl->stream_hi : sl->stream;
        const long N = (long)L * L;
        const bool created = plan == nullptr;
        int rc = FC_OK;
        if (created) {
            rc = fftconv_plan_create(&plan, L, FC_F32 | FC_F64, nullptr);
            // many slot threads wait at once: let them sleep, not spin
            if (rc == FC_OK) rc = fftconv_plan_sync_mode(plan, 1);
        }
        if (rc == FC_OK) rc = ensure_staging(sl, (long)nb * N);
        sl->rtols.resize(nb);
        sl->res.assign(nb, cg_result{});
        const double t_in = now_s();
        if (rc == FC_OK) {
            for (int k = 0; k < nb && rc == FC_OK; ++k) {
                sl->rtols[k] = batch[k]->rq.rtol;
                if (cudaMemcpyAsync(sl->ds + (size_t)k * N, batch[k]->sp(), sizeof(double) * N,
                                    cudaMemcpyHostToDevice, st) != cudaSuccess ||
                    cudaMemcpyAsync(sl->db + (size_t)k * N, batch[k]->bp(), sizeof(double) * N,
                                    cudaMemcpyHostToDevice, st) != cudaSuccess)
                    rc = FC_ECUDA;
            }
        }
        const double t_solve = now_s();
        double t_out = t_solve;
        if (rc == FC_OK) {
            cg_opts o{};
            o.rtol = r->rq.rtol;
            o.mode = r->rq.mode;
            o.x0_zero = 1;
            o.precond = r->rq.precond;
            rc = fc_batch_solve_rtols(plan, nb, sl->ds, sl->db, sl->dx, &o, sl->rtols.data(), sl->res.data(),
                                      st);
            t_out = now_s();
            if (rc == FC_OK || rc == FC_ENOCONV || rc == FC_ENANINF) {
                rc = FC_OK;
                for (int k = 0; k < nb && rc == FC_OK; ++k)
                    if (batch[k]->rq.x &&
                        cudaMemcpyAsync(batch[k]->rq.x, sl->dx + (size_t)k * N, sizeof(double) * N,
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
                        rc = FC_ECUDA;
                if (rc == FC_OK && (cudaEventRecord(sl->done, st) != cudaSuccess ||
                                    cudaEventSynchronize(sl->done) != cudaSuccess))
                    rc = FC_ECUDA;
            }
        }
        if (trace_on()) {
            const double t_end = now_s();
            fprintf(stderr, "[fftconv server] L=%d nb=%d plan=%s set-up %.2f ms, inputs %.2f ms, solve %.2f ms, "
                    "outputs %.2f ms\n", L, nb, created ? "new" : "kept", (t_in - batch[0]->t_start) * 1e3,
                    (t_solve - t_in) * 1e3, (t_out - t_solve) * 1e3, (t_end - t_out) * 1e3);
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            const double t = now_s();
            for (int k = 0; k < nb; ++k) {
                Req* q = batch[k];
                sv->used -= q->est;  // reservations end; the plan's bytes are counted below
                q->res = sl->res[k];
                q->rc = rc != FC_OK ? rc : q->res.status;
                q->res.status = q->rc;
                q->t_done = t;
                q->res.latency_s = q->t_done - q->t_submit;
                q->res.run_s = q->t_done - q->t_start;
                q->state = 2;
            }
            if (!plan && created) sv->plans_of[L] -= 1;  // the plan could not be made
            if (plan) {
                size_t nbytes = 0;
                fftconv_plan_info(plan, nullptr, nullptr, nullptr, &nbytes);
                size_t& held = sv->plan_bytes[plan];  // 0 for a plan made here
                sv->used += nbytes - held;
                held = nbytes;
                if (sv->used > sv->peak) sv->peak = sv->used;
                sv->idle.emplace(L, plan);
            }
        }
        sv->cv.notify_all();
    }
}

}  // namespace

extern "C" int cg_server_create(cg_server** out, size_t mem_budget_bytes, int max_slots, fc_stream_t stream) {
    (void)stream;  // each slot runs on its own non-blocking stream
    if (!out || max_slots < 1 || max_slots > 256 || mem_budget_bytes == 0) return FC_EINVAL;
    *out = nullptr;
    cg_server* sv = new (std::nothrow) cg_server();
    if (!sv) return FC_ENOMEM;
    if (cudaGetDevice(&sv->dev) != cudaSuccess) {
        delete sv;
        return FC_ECUDA;
    }
    sv->budget = mem_budget_bytes;
    sv->max_slots = max_slots;
    for (int i = 0; i < max_slots; ++i) {
        Slot* sl = new (std::nothrow) Slot();
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (!sl || cudaStreamCreateWithPriority(&sl->stream, cudaStreamNonBlocking, lo) != cudaSuccess ||
            cudaStreamCreateWithPriority(&sl->stream_hi, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl->done, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
            if (sl && sl->stream) cudaStreamDestroy(sl->stream);
            if (sl && sl->stream_hi) cudaStreamDestroy(sl->stream_hi);
            delete sl;
            cg_server_destroy(sv);
            return FC_ECUDA;
        }
        sv->slots.push_back(sl);
    }
    for (Slot* sl : sv->slots) sl->th = std::thread(worker, sv, sl);
    *out = sv;
    return FC_OK;
}

extern "C" int cg_server_reserve(cg_server* sv, int L, int nplans) {
    if (!sv || L < 1 || L > 4096 || nplans < 1) return FC_EINVAL;
    const int want = nplans < plans_per_size() ? nplans : plans_per_size();
    for (;;) {
        const size_t need = estimate_bytes(L);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (sv->plans_of[L] >= want) return FC_OK;
            if (sv->used + need > sv->budget) return FC_EBUDGET;
            sv->plans_of[L] += 1;  // the plan made below
            sv->used += need;
            if (sv->used > sv->peak) sv->peak = sv->used;
        }
        fftconv_plan* plan = nullptr;
        int rc = fftconv_plan_create(&plan, L, FC_F32 | FC_F64, nullptr);
        if (rc == FC_OK) rc = fftconv_plan_sync_mode(plan, 1);
        size_t nbytes = 0;
        if (rc == FC_OK) fftconv_plan_info(plan, nullptr, nullptr, nullptr, &nbytes);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->used -= need;
            if (rc != FC_OK) {
                sv->plans_of[L] -= 1;
            } else {
                sv->plan_bytes[plan] = nbytes;
                sv->used += nbytes;
                if (sv->used > sv->peak) sv->peak = sv->used;
                sv->idle.emplace(L, plan);
            }
        }
        if (rc != FC_OK) {
            if (plan) fftconv_plan_destroy(plan);
            return rc;
        }
        sv->cv.notify_all();
    }
}

extern "C" int cg_batch_submit(cg_server* sv, const cg_request* rq, uint64_t* ticket) {
    if (!sv || !rq || !ticket || !rq->s || !rq->b || rq->L < 1 || rq->L > 4096 || !(rq->rtol >= 0) ||
        (rq->mode != FC_MODE_F64 && rq->mode != FC_MODE_MIXED) || (rq->flags & ~FC_REQ_BORROW))
        return FC_EINVAL;
    const size_t est = estimate_bytes(rq->L) + batch_bytes(rq->L, rq->mode);
    if (est > sv->budget) return FC_EBUDGET;
    Req* r = new (std::nothrow) Req();
    if (!r) return FC_ENOMEM;
    const size_t N = (size_t)rq->L * rq->L;
    try {
        if (!(rq->flags & FC_REQ_BORROW)) {
            r->s.assign(rq->s, rq->s + N);
            r->b.assign(rq->b, rq->b + N);
        }
    } catch (...) {
        delete r;
        return FC_ENOMEM;
    }
    r->rq = *rq;
    r->est = est;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->ticket = sv->next_ticket++;
        sv->reqs[r->ticket] = r;
        sv->queue.push_back(r);
        *ticket = r->ticket;
    }
    sv->cv.notify_all();
    return FC_OK;
}

extern "C" int cg_poll(cg_server* sv, uint64_t ticket, cg_result* res, int* done) {
    if (!sv || !done) return FC_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return FC_ENOTFOUND;
    Req* r = it->second;
    *done = r->state == 2;
    if (*done) {
        if (res) *res = r->res;
        const int rc = r->rc;
        sv->reqs.erase(it);
        delete r;
        return rc == FC_ENOCONV || rc == FC_ENANINF ? FC_OK : rc;
    }
    return FC_OK;
}

extern "C" int cg_server_batches(cg_server* sv, long long* batches, long long* solves, int* max_batch) {
    if (!sv) return FC_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (batches) *batches = sv->batches;
    if (solves) *solves = sv->solves;
    if (max_batch) *max_batch = sv->max_batch;
    return FC_OK;
}

extern "C" int cg_server_stats(cg_server* sv, size_t* used, size_t* peak, int* queued, int* plans) {
    if (!sv) return FC_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (used) *used = sv->used;
    if (peak) *peak = sv->peak;
    if (queued) *queued = (int)sv->queue.size();
    if (plans) *plans = (int)sv->plan_bytes.size();
    return FC_OK;
}

extern "C" int cg_server_destroy(cg_server* sv) {
    if (!sv) return FC_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    for (Slot* sl : sv->slots)
        if (sl->th.joinable()) sl->th.join();
    for (auto& kv : sv->plan_bytes) fftconv_plan_destroy(kv.first);
    for (Slot* sl : sv->slots) {
        if (sl->stream_hi) {
            cudaStreamSynchronize(sl->stream_hi);
            cudaStreamDestroy(sl->stream_hi);
        }
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        if (sl->stream) {
            fc::dev_free_async(sl->ds, sl->stream);
            fc::dev_free_async(sl->db, sl->stream);
            fc::dev_free_async(sl->dx, sl->stream);
            cudaStreamSynchronize(sl->stream);
            cudaStreamDestroy(sl->stream);
        }
        if (sl->done) cudaEventDestroy(sl->done);
        delete sl;
    }
    for (auto& kv : sv->reqs) delete kv.second;  // every request, queued or not, is in reqs
    delete sv;
    return FC_OK;
}
