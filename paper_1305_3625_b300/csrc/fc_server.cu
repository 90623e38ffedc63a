// Solve server: continuous batching of independent solves on one GPU.
//
// Requests (L, mode, rtol, host s and b) are queued by cg_batch_submit and
// admitted when a worker slot is free and the device-memory budget holds the
// request's plan.  Each slot is a host thread with its own non-blocking CUDA
// stream; slots run their solves concurrently, so requests that arrive while
// others are on the GPU overlap with them.  Plans (spectrum, tables,
// workspaces) stay resident and are reused by later requests of the same L;
// idle plans of other sizes are evicted when the budget requires it.  Each
// result is the same whether a request runs alone or in a mix: a solve's
// arithmetic depends only on its own inputs and its plan (reductions run in a
// fixed order inside each solve).
#include <cuda_runtime.h>
#include <stdio.h>
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

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t ticket = 0;
    cg_request rq{};
    std::vector<double> s, b;  // host copies taken at submit
    size_t est = 0;            // device bytes the request's plan needs
    int state = 0;             // 0 queued, 1 running, 2 done
    int rc = 0;
    cg_result res{};
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct Slot {
    std::thread th;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;  // blocking-sync event: a waiting slot thread sleeps
    double *ds = nullptr, *db = nullptr, *dx = nullptr;  // device staging
    double *hs = nullptr, *hb = nullptr, *hx = nullptr;  // pinned host staging
    long cap = 0;
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

}  // namespace

struct cg_server {
    int dev = 0;
    size_t budget = 0, used = 0, peak = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req*> queue;
    std::unordered_map<uint64_t, Req*> reqs;
    std::multimap<int, fftconv_plan*> idle;      // idle plans by L
    std::map<fftconv_plan*, size_t> plan_bytes;  // every plan held
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<Slot*> slots;
};

namespace {

// Pick the first queued request that can run now: an idle plan of its size
// exists, or its plan fits the budget (possibly after evicting idle plans of
// other sizes).  Called with the lock held.  Returns the request and the plan
// to use (nullptr: create one) and the idle plans to destroy.
Req* admit_locked(cg_server* sv, fftconv_plan** plan, std::vector<fftconv_plan*>& evict) {
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
        Req* r = *it;
        auto ip = sv->idle.find(r->rq.L);
        if (ip != sv->idle.end()) {
            *plan = ip->second;
            sv->idle.erase(ip);
            sv->queue.erase(it);
            return r;
        }
        size_t freeable = 0;
        for (auto& kv : sv->idle) freeable += sv->plan_bytes[kv.second];
        if (sv->used + r->est <= sv->budget || sv->used - freeable + r->est <= sv->budget) {
            while (sv->used + r->est > sv->budget && !sv->idle.empty()) {
                auto v = sv->idle.begin();
                evict.push_back(v->second);
                sv->used -= sv->plan_bytes[v->second];
                sv->plan_bytes.erase(v->second);
                sv->idle.erase(v);
            }
            sv->used += r->est;  // reserved until the plan exists
            if (sv->used > sv->peak) sv->peak = sv->used;
            *plan = nullptr;
            sv->queue.erase(it);
            return r;
        }
    }
    return nullptr;
}

int ensure_staging(Slot* sl, long n) {
    if (n <= sl->cap) return FC_OK;
    cudaStreamSynchronize(sl->stream);
    cudaFree(sl->ds);
    cudaFree(sl->db);
    cudaFree(sl->dx);
    cudaFreeHost(sl->hs);
    cudaFreeHost(sl->hb);
    cudaFreeHost(sl->hx);
    sl->ds = sl->db = sl->dx = sl->hs = sl->hb = sl->hx = nullptr;
    sl->cap = 0;
    const size_t bytes = sizeof(double) * (size_t)n;
    if (cudaMalloc(&sl->ds, bytes) != cudaSuccess || cudaMalloc(&sl->db, bytes) != cudaSuccess ||
        cudaMalloc(&sl->dx, bytes) != cudaSuccess || cudaMallocHost(&sl->hs, bytes) != cudaSuccess ||
        cudaMallocHost(&sl->hb, bytes) != cudaSuccess || cudaMallocHost(&sl->hx, bytes) != cudaSuccess)
        return FC_ENOMEM;
    sl->cap = n;
    return FC_OK;
}

void worker(cg_server* sv, Slot* sl) {
    cudaSetDevice(sv->dev);
    for (;;) {
        Req* r = nullptr;
        fftconv_plan* plan = nullptr;
        std::vector<fftconv_plan*> evict;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] {
                if (sv->stop) return true;
                r = admit_locked(sv, &plan, evict);
                return r != nullptr;
            });
            if (!r) return;  // stopping
            r->state = 1;
            r->t_start = now_s();
        }
        for (fftconv_plan* e : evict) fftconv_plan_destroy(e);
        const int L = r->rq.L;
        const long N = (long)L * L;
        int rc = FC_OK;
        if (!plan) {
            rc = fftconv_plan_create(&plan, L, FC_F32 | FC_F64, nullptr);
            // many slot threads wait at once: let them sleep, not spin
            if (rc == FC_OK) rc = fftconv_plan_sync_mode(plan, 1);
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->used -= r->est;
            if (rc == FC_OK) {
                size_t nb = 0;
                fftconv_plan_info(plan, nullptr, nullptr, nullptr, &nb);
                sv->plan_bytes[plan] = nb;
                sv->used += nb;
                if (sv->used > sv->peak) sv->peak = sv->used;
            }
        }
        if (rc == FC_OK) rc = ensure_staging(sl, N);
        if (rc == FC_OK) {
            memcpy(sl->hs, r->s.data(), sizeof(double) * N);
            memcpy(sl->hb, r->b.data(), sizeof(double) * N);
            cudaMemcpyAsync(sl->ds, sl->hs, sizeof(double) * N, cudaMemcpyHostToDevice, sl->stream);
            cudaMemcpyAsync(sl->db, sl->hb, sizeof(double) * N, cudaMemcpyHostToDevice, sl->stream);
            cg_opts o{};
            o.rtol = r->rq.rtol;
            o.mode = r->rq.mode;
            o.x0_zero = 1;
            o.precond = r->rq.precond;
            rc = cg_solve(plan, sl->ds, sl->db, sl->dx, nullptr, &o, &r->res, sl->stream);
            if (rc == FC_OK || rc == FC_ENOCONV || rc == FC_ENANINF) {
                cudaMemcpyAsync(sl->hx, sl->dx, sizeof(double) * N, cudaMemcpyDeviceToHost, sl->stream);
                if (cudaEventRecord(sl->done, sl->stream) != cudaSuccess || cudaEventSynchronize(sl->done) != cudaSuccess)
                    rc = FC_ECUDA;
                if (r->rq.x) memcpy(r->rq.x, sl->hx, sizeof(double) * N);
            }
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->rc = rc;
            r->res.status = rc;
            r->t_done = now_s();
            r->res.latency_s = r->t_done - r->t_submit;
            r->res.run_s = r->t_done - r->t_start;
            r->state = 2;
            if (plan) sv->idle.emplace(L, plan);
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
        if (!sl || cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl->done, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
            if (sl && sl->stream) cudaStreamDestroy(sl->stream);
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

extern "C" int cg_batch_submit(cg_server* sv, const cg_request* rq, uint64_t* ticket) {
    if (!sv || !rq || !ticket || !rq->s || !rq->b || rq->L < 1 || rq->L > 4096 || !(rq->rtol >= 0) ||
        (rq->mode != FC_MODE_F64 && rq->mode != FC_MODE_MIXED))
        return FC_EINVAL;
    const size_t est = estimate_bytes(rq->L);
    if (est > sv->budget) return FC_EBUDGET;
    Req* r = new (std::nothrow) Req();
    if (!r) return FC_ENOMEM;
    const size_t N = (size_t)rq->L * rq->L;
    try {
        r->s.assign(rq->s, rq->s + N);
        r->b.assign(rq->b, rq->b + N);
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
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        cudaFree(sl->ds);
        cudaFree(sl->db);
        cudaFree(sl->dx);
        cudaFreeHost(sl->hs);
        cudaFreeHost(sl->hb);
        cudaFreeHost(sl->hx);
        if (sl->stream) cudaStreamDestroy(sl->stream);
        if (sl->done) cudaEventDestroy(sl->done);
        delete sl;
    }
    for (auto& kv : sv->reqs) delete kv.second;  // every request, queued or not, is in reqs
    delete sv;
    return FC_OK;
}
