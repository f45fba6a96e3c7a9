// Serving form: a continuous-batching request loop over one forest (the
// cc_server_* entry points of include/cc.h).
//
// Threads and streams:
//  - callers enqueue requests (any thread); each gets a ticket and an arrival
//    time;
//  - one worker thread cuts the arrived, not yet launched requests into
//    groups of consecutive same-kind requests, reserves a contiguous range of
//    the device staging ring for each group, copies the group's host data in
//    on the h2d stream, and launches ONE Bulk-Update or Bulk-Query over the
//    range on the compute stream (after the copy). Query answers go back on
//    the d2h stream. An event recorded after the group's last operation is
//    watched by a completion thread, which stamps the completion time and
//    frees the group's ring range;
//  - groups compute in arrival order on the single compute stream, so a
//    query sees exactly the updates that arrived before it. Merging adjacent
//    updates is exact because the graph is the union of the edge sets.
// Neither thread holds the lock while it calls CUDA, so neither can wait on
// the other.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "cc.h"
#include "cc_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    int32_t kind;
    const int32_t* data;
    int64_t k;
    uint8_t* out;
    double t_arrive = 0, t_done = -1;
    int64_t off = 0;  // ring position (pairs)
    bool done = false;
};

struct Group {
    cc_server* srv;
    int64_t first, last;  // requests [first, last)
    int64_t b, e;         // ring range [b, e) in pairs
    cudaEvent_t ev = nullptr;  // recorded after the group's last operation
    bool launched = false;     // ev has been recorded
    bool done = false;
};

}  // namespace

struct cc_server {
    cc_ctx* ctx = nullptr;
    cudaStream_t prev_stream = nullptr;
    int device = 0;
    cudaStream_t compute = nullptr, h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_in = nullptr, ev_q = nullptr;
    int32_t* ring = nullptr;
    uint8_t* ring_out = nullptr;
    int64_t cap = 0, max_group = 0;
    bool merge = true;

    std::mutex mu;
    // one condition per kind of waiter, so that a notification wakes only
    // the thread that can act on it
    std::condition_variable cv_work;  // worker: new requests, ring space, stop
    std::condition_variable cv_reap;  // completion thread: launched groups, stop
    std::condition_variable cv_done;  // cc_server_wait / drain / destroy: completions
    std::deque<Req> reqs;
    int64_t next_launch = 0, completed = 0, groups = 0;
    int64_t n_upd = 0, n_qry = 0, edges = 0, pairs = 0;
    int64_t head = 0;
    int64_t used = 0;  // ring pairs held by in-flight groups
    std::deque<Group*> inflight;
    bool stop = false;
    cc_status err = CC_OK;
    std::string errmsg;
    std::thread worker;
    std::thread reaper;                 // completion thread
    std::vector<cudaEvent_t> spare_events;
};

namespace {

void fail_worker(cc_server* s, cudaError_t e, const char* what) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err == CC_OK) {
        s->err = CC_ERR_CUDA;
        s->errmsg = std::string(what) + ": " + cudaGetErrorString(e);
    }
    s->cv_work.notify_all();
    s->cv_reap.notify_all();
    s->cv_done.notify_all();
}

// A group's work is complete: stamp its requests, free ring ranges in order.
// Called with the lock held.
void mark_done(cc_server* s, Group* g, double t) {
    for (int64_t i = g->first; i < g->last; i++) {
        s->reqs[i].t_done = t;
        s->reqs[i].done = true;
    }
    s->completed += g->last - g->first;
    g->done = true;
    while (!s->inflight.empty() && s->inflight.front()->done) {
        Group* f = s->inflight.front();
        s->used -= f->e - f->b;
        s->spare_events.push_back(f->ev);
        delete f;
        s->inflight.pop_front();
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();  // ring space for a group that did not fit
}

// Completion thread: takes the oldest launched group that is not done under
// the lock, then polls its event with the lock released (the worker and the
// enqueuing threads never wait behind the poll), so the time from completion
// to notice stays at a few microseconds. Groups complete in launch order
// except that an update group may finish while an earlier query group's
// answers are still being copied out; such a group is noticed right after
// that copy. Only this thread marks groups done, and a group is freed only
// once done, so the pointer stays valid while it is polled.
void reaper_loop(cc_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        Group* g = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto oldest = [&]() -> Group* {
                for (Group* x : s->inflight)
                    if (!x->done) return x->launched ? x : nullptr;
                return nullptr;
            };
            s->cv_reap.wait(lk, [&] {
                if (s->err != CC_OK || oldest()) return true;
                return s->stop && s->next_launch >= (int64_t)s->reqs.size() && s->inflight.empty();
            });
            if (s->err != CC_OK) return;
            g = oldest();
            if (!g) return;  // stopping, nothing left
        }
        // poll every ~2 us: often enough for latency, rarely enough that the
        // driver calls of the worker thread do not queue behind the queries
        cudaError_t q;
        while ((q = cudaEventQuery(g->ev)) == cudaErrorNotReady) {
            const double t_next = now_s() + 2e-6;
            while (now_s() < t_next) std::this_thread::yield();
        }
        if (q != cudaSuccess) {
            fail_worker(s, q, "serve: completion");
            return;
        }
        const double t = now_s();
        std::lock_guard<std::mutex> lk(s->mu);
        mark_done(s, g, t);
    }
}

// Reserve [b, b+k) of the ring (FIFO). Called with the lock held.
//
// Groups take ranges in launch order and free them in the same order, so the
// occupied part is one arc from the oldest non-empty in-flight group's start
// (tail) to head, possibly wrapping past the end. Emptiness is decided by the
// number of pairs held, not by head == tail: a group of zero pairs sits at
// head without occupying anything, and when it is the oldest in flight while
// later groups have filled the ring all the way round, head == tail means
// full.
bool ring_alloc(cc_server* s, int64_t k, int64_t* b) {
    if (s->used == 0) s->head = 0;
    if (k == 0) {
        *b = s->head;
        return true;
    }
    if (s->used == 0) {
        if (k > s->cap) return false;
        *b = 0;
        return true;
    }
    int64_t tail = s->head;
    for (const Group* g : s->inflight)
        if (g->e > g->b) {
            tail = g->b;
            break;
        }
    if (s->head > tail) {
        // occupied [tail, head): free space at the end, then at the start
        if (s->cap - s->head >= k) { *b = s->head; return true; }
        if (tail >= k) { *b = 0; return true; }
        return false;
    }
    // wrapped: occupied [tail, cap) and [0, head); free [head, tail)
    if (tail - s->head >= k) { *b = s->head; return true; }
    return false;
}


void worker_loop(cc_server* s) {
    cudaSetDevice(s->device);
    std::vector<Req> batch;
    for (;;) {
        int64_t first, last, b = 0, total = 0;
        int32_t kind;
        Group* g = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || s->err != CC_OK || s->next_launch < (int64_t)s->reqs.size(); });
            if (s->err != CC_OK) return;
            if (s->next_launch >= (int64_t)s->reqs.size()) return;  // stop, nothing left
            for (;;) {
                // the longest run of same-kind requests that fits one launch
                first = s->next_launch;
                kind = s->reqs[first].kind;
                last = first;
                total = 0;
                while (last < (int64_t)s->reqs.size() && s->reqs[last].kind == kind &&
                       (last == first || (s->merge && total + s->reqs[last].k <= s->max_group))) {
                    total += s->reqs[last].k;
                    last++;
                }
                // shrink it until its staging range fits; else wait for room
                while (!ring_alloc(s, total, &b) && last - first > 1) total -= s->reqs[--last].k;
                if (ring_alloc(s, total, &b)) break;
                s->cv_work.wait(lk);
                if (s->err != CC_OK) return;
            }
            g = new Group{s, first, last, b, b + total};
            if (!s->spare_events.empty()) {
                g->ev = s->spare_events.back();
                s->spare_events.pop_back();
            }
            s->inflight.push_back(g);
            s->head = b + total;
            s->used += total;
            s->next_launch = last;
            s->groups++;
            batch.clear();
            int64_t off = b;
            for (int64_t i = first; i < last; i++) {
                s->reqs[i].off = off;
                off += s->reqs[i].k;
                batch.push_back(s->reqs[i]);
            }
        }
        // --- device work for the group (no lock held) ---
        cudaError_t e = cudaSuccess;
        if (!g->ev) e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming);
        // copy in: one copy per run of requests whose host data is contiguous;
        // if the driver refuses a run (it spans two separate host
        // allocations), copy its requests one by one
        for (size_t i = 0; i < batch.size() && e == cudaSuccess;) {
            size_t j = i + 1;
            int64_t pairs = batch[i].k;
            while (j < batch.size() && batch[j].data == batch[i].data + 2 * pairs) pairs += batch[j++].k;
            if (pairs > 0) {
                e = cudaMemcpyAsync(s->ring + 2 * batch[i].off, batch[i].data, sizeof(int32_t) * 2 * (size_t)pairs,
                                    cudaMemcpyHostToDevice, s->h2d);
                if (e == cudaErrorInvalidValue && j > i + 1) {
                    cudaGetLastError();
                    e = cudaSuccess;
                    for (size_t r = i; r < j && e == cudaSuccess; r++)
                        if (batch[r].k > 0)
                            e = cudaMemcpyAsync(s->ring + 2 * batch[r].off, batch[r].data,
                                                sizeof(int32_t) * 2 * (size_t)batch[r].k, cudaMemcpyHostToDevice, s->h2d);
                }
            }
            i = j;
        }
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_in, s->h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->compute, s->ev_in, 0);
        if (e != cudaSuccess) { fail_worker(s, e, "serve: staging copy"); return; }
        if (kind == CC_OP_UPDATE) {
            cc_status st = total ? cc_bulk_update(s->ctx, s->ring + 2 * b, total) : CC_OK;
            if (st != CC_OK) { fail_worker(s, cudaErrorUnknown, "serve: bulk update"); return; }
            e = cudaEventRecord(g->ev, s->compute);
        } else {
            cc_status st = total ? cc_bulk_query(s->ctx, s->ring + 2 * b, total, s->ring_out + b) : CC_OK;
            if (st != CC_OK) { fail_worker(s, cudaErrorUnknown, "serve: bulk query"); return; }
            e = cudaEventRecord(s->ev_q, s->compute);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->d2h, s->ev_q, 0);
            for (size_t i = 0; i < batch.size() && e == cudaSuccess;) {  // contiguous outputs: one copy
                size_t j = i + 1;
                int64_t pairs = batch[i].k;
                while (j < batch.size() && batch[j].out == batch[i].out + pairs) pairs += batch[j++].k;
                if (pairs > 0) {
                    e = cudaMemcpyAsync(batch[i].out, s->ring_out + batch[i].off, (size_t)pairs,
                                        cudaMemcpyDeviceToHost, s->d2h);
                    if (e == cudaErrorInvalidValue && j > i + 1) {  // spans two allocations
                        cudaGetLastError();
                        e = cudaSuccess;
                        for (size_t r = i; r < j && e == cudaSuccess; r++)
                            if (batch[r].k > 0)
                                e = cudaMemcpyAsync(batch[r].out, s->ring_out + batch[r].off, (size_t)batch[r].k,
                                                    cudaMemcpyDeviceToHost, s->d2h);
                    }
                }
                i = j;
            }
            if (e == cudaSuccess) e = cudaEventRecord(g->ev, s->d2h);
        }
        if (e != cudaSuccess) { fail_worker(s, e, "serve: launch"); return; }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            g->launched = true;
            s->cv_reap.notify_one();
        }
    }
}

cc_status server_fail(cc_status st, const char* msg) { return cc::record_error(st, msg); }

}  // namespace

extern "C" {

cc_status cc_server_create(cc_ctx* ctx, const cc_server_config* cfg, cc_server** out) {
    if (!ctx || !out) return server_fail(CC_ERR_ARG, "cc_server_create: null argument");
    *out = nullptr;
    if (cc::ctx_graphs(ctx) > 1) return server_fail(CC_ERR_UNSUPPORTED, "cc_server_create: segmented handle");
    cc_server* s = new (std::nothrow) cc_server();
    if (!s) return server_fail(CC_ERR_OOM, "cc_server_create: host allocation");
    s->ctx = ctx;
    s->device = cc::ctx_device(ctx);
    s->prev_stream = cc::ctx_stream(ctx);
    s->cap = (cfg && cfg->ring_pairs > 0) ? cfg->ring_pairs : (int64_t)1 << 25;
    s->max_group = (cfg && cfg->max_group_pairs > 0) ? cfg->max_group_pairs : (int64_t)1 << 22;
    s->merge = cfg ? cfg->merge != 0 : true;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_q, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&s->ring, sizeof(int32_t) * 2 * (size_t)s->cap);
    if (e == cudaSuccess) e = cudaMalloc(&s->ring_out, (size_t)s->cap);
    // the new streams do not wait for the handle's old stream: order them once
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->prev_stream);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->ring);
        cudaFree(s->ring_out);
        if (s->ev_in) cudaEventDestroy(s->ev_in);
        if (s->ev_q) cudaEventDestroy(s->ev_q);
        if (s->compute) cudaStreamDestroy(s->compute);
        if (s->h2d) cudaStreamDestroy(s->h2d);
        if (s->d2h) cudaStreamDestroy(s->d2h);
        delete s;
        return server_fail(e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA, "cc_server_create: CUDA setup failed");
    }
    cc_set_stream(ctx, s->compute);
    s->worker = std::thread(worker_loop, s);
    s->reaper = std::thread(reaper_loop, s);
    *out = s;
    return CC_OK;
}

cc_status cc_server_enqueue(cc_server* s, int32_t kind, const int32_t* data, int64_t k,
                            uint8_t* out, uint64_t* ticket) {
    if (!s) return server_fail(CC_ERR_ARG, "cc_server_enqueue: null server");
    if (kind != CC_OP_UPDATE && kind != CC_OP_QUERY) return server_fail(CC_ERR_ARG, "cc_server_enqueue: unknown kind");
    if (k < 0 || k > s->cap || k > INT32_MAX) return server_fail(CC_ERR_ARG, "cc_server_enqueue: k out of range (larger than the staging ring?)");
    if (k > 0 && (!data || (kind == CC_OP_QUERY && !out))) return server_fail(CC_ERR_ARG, "cc_server_enqueue: null array");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err != CC_OK) return server_fail(s->err, s->errmsg.c_str());
    if (s->stop) return server_fail(CC_ERR_ARG, "cc_server_enqueue: server is stopping");
    Req r;
    r.kind = kind;
    r.data = data;
    r.k = k;
    r.out = out;
    r.t_arrive = now_s();
    s->reqs.push_back(r);
    if (kind == CC_OP_UPDATE) { s->n_upd++; s->edges += k; } else { s->n_qry++; s->pairs += k; }
    if (ticket) *ticket = (uint64_t)(s->reqs.size() - 1);
    s->cv_work.notify_one();
    return CC_OK;
}

cc_status cc_server_enqueue_many(cc_server* s, int64_t n, const int32_t* kinds,
                                 const int32_t* const* data, const int64_t* k, uint8_t* const* out,
                                 uint64_t* first_ticket) {
    if (!s) return server_fail(CC_ERR_ARG, "cc_server_enqueue_many: null server");
    if (n < 0) return server_fail(CC_ERR_ARG, "cc_server_enqueue_many: n < 0");
    if (n > 0 && (!kinds || !data || !k)) return server_fail(CC_ERR_ARG, "cc_server_enqueue_many: null array");
    char msg[160];
    for (int64_t i = 0; i < n; i++) {  // everything is checked before anything is accepted
        const char* why = nullptr;
        if (kinds[i] != CC_OP_UPDATE && kinds[i] != CC_OP_QUERY) why = "unknown kind";
        else if (k[i] < 0 || k[i] > s->cap || k[i] > INT32_MAX) why = "k out of range (larger than the staging ring?)";
        else if (k[i] > 0 && !data[i]) why = "null data";
        else if (k[i] > 0 && kinds[i] == CC_OP_QUERY && (!out || !out[i])) why = "null out for a query";
        if (why) {
            snprintf(msg, sizeof msg, "cc_server_enqueue_many: request %lld: %s", (long long)i, why);
            return server_fail(CC_ERR_ARG, msg);
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err != CC_OK) return server_fail(s->err, s->errmsg.c_str());
    if (s->stop) return server_fail(CC_ERR_ARG, "cc_server_enqueue_many: server is stopping");
    const double t = now_s();
    if (first_ticket) *first_ticket = (uint64_t)s->reqs.size();
    for (int64_t i = 0; i < n; i++) {
        Req r;
        r.kind = kinds[i];
        r.data = data[i];
        r.k = k[i];
        r.out = kinds[i] == CC_OP_QUERY ? out[i] : nullptr;
        r.t_arrive = t;
        s->reqs.push_back(r);
        if (r.kind == CC_OP_UPDATE) { s->n_upd++; s->edges += r.k; } else { s->n_qry++; s->pairs += r.k; }
    }
    if (n > 0) s->cv_work.notify_one();
    return CC_OK;
}

cc_status cc_server_wait(cc_server* s, uint64_t ticket, double* latency_s) {
    if (!s) return server_fail(CC_ERR_ARG, "cc_server_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket >= s->reqs.size()) return server_fail(CC_ERR_ARG, "cc_server_wait: unknown ticket");
    s->cv_done.wait(lk, [&] { return s->reqs[ticket].done || s->err != CC_OK; });
    if (s->err != CC_OK) return server_fail(s->err, s->errmsg.c_str());
    if (latency_s) *latency_s = s->reqs[ticket].t_done - s->reqs[ticket].t_arrive;
    return CC_OK;
}

cc_status cc_server_drain(cc_server* s) {
    if (!s) return server_fail(CC_ERR_ARG, "cc_server_drain: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->completed == (int64_t)s->reqs.size() || s->err != CC_OK; });
    if (s->err != CC_OK) return server_fail(s->err, s->errmsg.c_str());
    return CC_OK;
}

cc_status cc_server_get_stats(cc_server* s, cc_server_stats* out) {
    if (!s || !out) return server_fail(CC_ERR_ARG, "cc_server_get_stats: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->requests = (int64_t)s->reqs.size();
    out->updates = s->n_upd;
    out->queries = s->n_qry;
    out->completed = s->completed;
    out->groups = s->groups;
    out->edges = s->edges;
    out->pairs = s->pairs;
    return CC_OK;
}

cc_status cc_server_latencies(cc_server* s, double* out, int64_t n, int64_t* written) {
    if (!s || (n > 0 && !out)) return server_fail(CC_ERR_ARG, "cc_server_latencies: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t m = n < (int64_t)s->reqs.size() ? n : (int64_t)s->reqs.size();
    for (int64_t i = 0; i < m; i++)
        out[i] = s->reqs[i].done ? s->reqs[i].t_done - s->reqs[i].t_arrive : -1.0;
    if (written) *written = m;
    return CC_OK;
}

cc_status cc_server_destroy(cc_server* s) {
    if (!s) return CC_OK;
    cc_status st = CC_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->completed == (int64_t)s->reqs.size() || s->err != CC_OK; });
        s->stop = true;
        s->cv_work.notify_all();
        s->cv_reap.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->cv_reap.notify_all();
    }
    if (s->reaper.joinable()) s->reaper.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    if (cudaStreamSynchronize(s->compute) != cudaSuccess || cudaStreamSynchronize(s->d2h) != cudaSuccess)
        st = server_fail(CC_ERR_CUDA, "cc_server_destroy: sync");
    cudaStreamSynchronize(s->h2d);
    cc_set_stream(s->ctx, s->prev_stream);
    for (Group* g : s->inflight) {
        if (g->ev) cudaEventDestroy(g->ev);
        delete g;
    }
    for (cudaEvent_t ev : s->spare_events) cudaEventDestroy(ev);
    cudaFree(s->ring);
    cudaFree(s->ring_out);
    cudaEventDestroy(s->ev_in);
    cudaEventDestroy(s->ev_q);
    cudaStreamDestroy(s->compute);
    cudaStreamDestroy(s->h2d);
    cudaStreamDestroy(s->d2h);
    cudaSetDevice(prev);
    if (s->err != CC_OK && st == CC_OK) st = server_fail(s->err, s->errmsg.c_str());
    delete s;
    return st;
}

}  // extern "C"
